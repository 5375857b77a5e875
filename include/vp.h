/*
 * vp.h -- C ABI of the GB300 volume-potential library.
 *
 * The library computes volume potentials phi = g_k * f on a uniform N^d grid
 * with the truncated-Green's-function method of Vico, Greengard & Ferrando,
 * "Fast convolution with free-space Green's functions" (arXiv:1604.03155):
 *
 *   phi(x) = int_D g_k(x - y) f(y) dy,  D = [-1/2, 1/2]^d        (Section 1, eq. volint)
 *
 * where g_k is the free-space Green's function of -(Delta + k^2): e^{ikr}/(4 pi r)
 * in 3D, (i/4) H_0^(1)(kr) in 2D, 1/(4 pi r) and -log(r)/(2 pi) for k = 0
 * (Tables 1-2), or the biharmonic g_b of -Delta^2: r/(8 pi) in 3D and
 * -r^2 (log r - 1)/(8 pi) in 2D (Tables 1-2, row Delta^2).  The kernel is cut off at r = L (Section 1, g^L) so that its
 * Fourier transform G^L is smooth; G^L is sampled on the 4N-oversampled grid
 * and inverse transformed once to the discrete kernel T (Section 4, the
 * "precomputation step"); every apply is then a zero-padded (2N)^d FFT
 * convolution (Section 4), optionally with gradients by spectral
 * differentiation (Section 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid (Section 4): N even, h = 1/N; storage index p_j in [0, N) on each axis
 *   maps to grid index i_j = p_j - N/2 + 1 and coordinate x_j = i_j h, so the
 *   origin is a node.  Arrays are C order (last axis fastest), N^d elements.
 * Result: phi_p = sum_{p'} T(p - p') f_{p'}, the quadrature weight h^d included,
 *   so phi approximates the integral above to spectral accuracy for smooth f.
 * Pointers: f, phi and grad may be device pointers (asynchronous on the
 *   plan's stream) or host pointers (pinned buffers are read and written in
 *   place through their device mappings, others are staged through device
 *   memory; the call returns when the host result is written).  phi may not
 *   alias f.
 * Complex data is interleaved (re, im).  grad holds d contiguous N^d blocks,
 *   block j = d phi / d x_j.
 * Errors: every call returns a vp_status and never aborts; argument errors are
 *   reported before any device work.  vp_last_error() gives a message.
 * Environment: VP_LOG=1 also writes every recorded error message to stderr
 *   ("vp: <object>: <message>"), VP_LOG=2 the pass autotuner's choices too;
 *   VP_TIMEOUT_MS sets the default wait budget of batches and networks;
 *   VP_AUTOTUNE_CACHE names the autotuners' cache file.
 */
#ifndef VP_H
#define VP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vp_plan_s* vp_plan; /* opaque; owned by the library */

typedef enum {
  VP_OK = 0,
  VP_ERR_INVALID_ARG = 1, /* bad argument (NULL, out of range, wrong dtype) */
  VP_ERR_UNSUPPORTED = 2, /* valid but not built (grid size without an FFT plan) */
  VP_ERR_OOM = 3,         /* device allocation failed */
  VP_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  VP_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  VP_ERR_NUMERICAL = 6    /* non-finite value where a finite one is required */
} vp_status;

typedef enum { VP_LAPLACE = 0, VP_HELMHOLTZ = 1, VP_BIHARMONIC = 2 } vp_kernel;

/* Arithmetic of the apply.  The precompute is always FP64.
 *  VP_FP32, VP_FP64   every pass in that precision (FP32 / FP64 data types).
 *  VP_TC_*            FP32 data and FP32 passes, except the fused axis-0 pass
 *                     of the 3D apply (forward 2N transform, multiplier,
 *                     inverse 2N transform), whose 2N = 16 x N2 transforms run
 *                     as radix-16 and radix-N2 complex GEMMs on the tensor
 *                     cores with the FP32 operands split into 16-bit parts
 *                     and FP32 accumulation (a project addition; the paper's
 *                     apply is FP64):
 *                       BF16X2  x = x0 + x1 (BF16), 3 partial products
 *                       FP16X2  x = x0 + x1 (FP16, power-of-two scaled), 3 products
 *                       BF16X3  x = x0 + x1 + x2 (BF16), 6 partial products
 *                     Only 3D plans with 2N in {256, 512} (N = 128, 256) and
 *                     only vp_apply (not vp_apply_grad); otherwise
 *                     VP_ERR_UNSUPPORTED. */
typedef enum {
  VP_FP32 = 0,
  VP_FP64 = 1,
  VP_TC_BF16X2 = 2,
  VP_TC_FP16X2 = 3,
  VP_TC_BF16X3 = 4
} vp_precision;

/* Gradient definition (Section 3, spectral differentiation):
 *  VP_GRAD_EXACT      derivative kernels T_j = inverse 4N transform of i s_j G^L
 *                     (the Nyquist sample zeroed), cropped and transformed like
 *                     T; the exact derivative of the discretised integral.
 *  VP_GRAD_SPECTRAL2N multiply the (2N)^d product by i pi m_j (the 2N grid's own
 *                     frequencies, Nyquist zeroed); agrees with EXACT to
 *                     spectral accuracy when f is negligible at the box edge. */
typedef enum { VP_GRAD_EXACT = 0, VP_GRAD_SPECTRAL2N = 1 } vp_grad_mode;

/* Element type of f, phi and grad.  Complex types work for every kernel; real
 * types only for VP_LAPLACE (real kernel, real potential).  The type must
 * match the plan's precision: R32/C64 for FP32, R64/C128 for FP64. */
typedef enum { VP_R32 = 0, VP_C64 = 1, VP_R64 = 2, VP_C128 = 3 } vp_dtype;

/* Precomputed arrays that can be read back (FP64, complex128 octants). */
typedef enum {
  VP_ARRAY_T = 0,     /* T(n), n in [0, N]^d                      (Section 4) */
  VP_ARRAY_GHAT = 1,  /* multiplier at m in [0, N]^d, unscaled       (Section 4) */
  VP_ARRAY_TJ = 2,    /* T_j(n), n in [0, N]^d, axis j = `axis`      (Section 3) */
  VP_ARRAY_GHATJ = 3  /* gradient multiplier octant, axis j          (Section 3) */
} vp_array;

/* Creates a plan and runs the FP64 precompute on the device (Sections 2 and 4):
 * samples G^L(|s_m|) for s_m = (pi/2) m, m in [0, 2N]^d (the octant of the
 * 4N grid; G^L is radial), reduces it to T by separable cosine sums (the
 * inverse 4N DFT of an even array), crops to (-N, N]^d and transforms to the
 * (2N)^d multiplier, stored as its [0, N]^d octant in FP64 and FP32.
 *   d       2 or 3
 *   N       even, >= 4; 2N must be a supported FFT length (VP_ERR_UNSUPPORTED)
 *   kernel  VP_LAPLACE or VP_BIHARMONIC (k must be 0), VP_HELMHOLTZ (k > 0)
 *   L       truncation radius; L <= 0 selects 1.8 (3D) / 1.5 (2D) (Section 2);
 *           otherwise sqrt(d) < L <= 3 (3 keeps the 4N grid alias-free).
 * The plan owns all device memory it allocates; workspace for applies is
 * allocated on first use.  Synchronous: returns after the precompute. */
vp_status vp_plan_create(vp_plan* out, int d, int N, vp_kernel kernel, double k, double L);

/* The same on a grid with N[j] points along axis j (axis 0 slowest; each N[j]
 * even, >= 4, 2 N[j] a built length): h_j = 1/N[j] on the same unit box.  The
 * spectrum is sampled at s_m = (pi/2) m on the per-axis 4 N[j] grids (the
 * frequency step is pi/2 on every axis) and every transform of Section 4 runs
 * per axis with that axis's length; arrays are C order [N0][N1]([N2]), octants
 * [N0+1][N1+1]([N2+1]).  Serves vp_apply, vp_apply_grad, vp_apply_noalloc, the
 * batch, the Nystrom entries and the Bi-CGStab solvers; the tensor-core
 * precisions and the FGMRES/U-Net solver take cubic plans only
 * (VP_ERR_UNSUPPORTED / VP_ERR_INVALID_ARG). */
vp_status vp_plan_create_aniso(vp_plan* out, int d, const int* N, vp_kernel kernel, double k, double L);
/* Points per axis (d ints). */
vp_status vp_plan_dims(vp_plan plan, int* N);

/* Saved plans: the precompute (Sections 2 and 4: sampling G^L, the 4N inverse
 * transform to T, the 2N multiplier) run once and kept on disk.
 *   vp_plan_save writes the plan's FP64 results to `path`: T and the unscaled
 *     multiplier octant, and the derivative kernels T_j with their multipliers
 *     when a gradient apply has built them (a 96-byte header: magic "VPPLAN01",
 *     version 1, d, N per axis, kernel, k, L, octant size, payload size and a
 *     64-bit FNV-1a hash of the payload's 8-byte words; then each octant as
 *     complex128, axis 0 slowest; host byte order).  Synchronises the plan's
 *     stream.
 *   vp_plan_load creates a plan on the current device from such a file
 *     without running the precompute: the uploaded arrays are scaled and
 *     rounded by the same kernel as at creation, so every apply equals that
 *     of the saved plan bit for bit.  The settings (precision, gradient mode,
 *     stream, host access, tile shapes) start at their defaults.
 *   vp_plan_kernel reports the plan's kernel.
 * Errors: VP_ERR_INVALID_ARG for a NULL argument, a file that cannot be
 * opened, written or read, a wrong magic, version or size, a truncated file,
 * trailing bytes or a hash mismatch (all checked before any device work);
 * the errors of vp_plan_create otherwise. */
vp_status vp_plan_save(vp_plan plan, const char* path);
vp_status vp_plan_load(vp_plan* out, const char* path);
vp_status vp_plan_kernel(vp_plan plan, vp_kernel* kernel);

/* Nystrom matrix entries on the fly (Section 4, the remark after the discrete
 * convolution): T is the matrix of a high-order Nystrom discretisation of the
 * volume integral, phi_p = sum_{p'} T(p - p') f_{p'} (weight h^d included).
 *   which, axis: VP_ARRAY_T (the potential; axis ignored) or VP_ARRAY_TJ with
 *     axis j (the derivative kernel of Section 3, odd in x_j; built on first use)
 *   vp_kernel_entries: out[i] = T(n_i) for count integer offsets n_i, given as
 *     count x d int32 (row i = n_i), each |n_ij| <= N
 *   vp_matrix_block: out[i][j] = T(p(rows[i]) - p(cols[j])), row-major
 *     nrows x ncols, rows/cols flat C-order grid indices in [0, N^d) (int64)
 *   dtype: VP_C128 (the FP64 octant as is) or VP_C64 (rounded); out complex.
 * All arrays are device pointers; asynchronous work on the plan's stream, the
 * call returns after it.  An offset or index out of range writes zero there
 * and returns VP_ERR_INVALID_ARG. */
vp_status vp_kernel_entries(vp_plan plan, int which, int axis, const int* offsets, long long count, void* out,
                            vp_dtype dtype);
vp_status vp_matrix_block(vp_plan plan, int which, int axis, const long long* rows, long long nrows,
                          const long long* cols, long long ncols, void* out, vp_dtype dtype);

/* Host pointers to page-locked (pinned) memory: direct = 1 lets the first
 * pass read f and the last pass write phi/grad in host memory through their
 * device mappings (over the CPU-GPU link, no staging copies); direct = 0
 * stages them through a plan-owned device buffer, as for pageable memory.
 * The default, set at plan creation, is 1 where the device reports coherent
 * access to host memory through the host's page tables
 * (cudaDevAttrPageableMemoryAccessUsesHostPageTables: a link such as
 * NVLink-C2C), else 0.  The call returns after the host result is written
 * either way. */
vp_status vp_plan_set_host_access(vp_plan plan, int direct);

/* Tile shapes of the FP32 passes (the four-step engine, 2N in {64, 128, 256,
 * 512, 1024}).  Each pass has up to 4 candidate shapes (pencils per CTA,
 * staging depth, exchange in the staging slot or in its own buffer; for the
 * fused pass of 2N = 512, candidate 0 is the TMA kernel); candidate 0 is the
 * measured default.  pass: 0 fwd_rows, 1 fwd_axis1, 2 fused_axis0, 3 inv_axis1,
 * 4 inv_rows (2D plans have no axis-1 passes).
 *   vp_plan_autotune times every candidate of every four-step pass on the
 *     plan's workspace and stream (CUDA events, 10 applies each after 2
 *     warm-ups), keeps the fastest per pass, and caches the choice on disk per
 *     device, driver and grid (VP_AUTOTUNE_CACHE, default
 *     $HOME/.cache/vp_autotune.txt); a cached choice is reused unless
 *     flags & 1.  Candidates are timed inside whole applies, pass by pass; one
 *     replaces the current choice when the apply gets more than 1% faster.
 *     The plan's precision must be VP_FP32 (else VP_ERR_UNSUPPORTED).
 *     Synchronises the plan's stream; allocates two grid-sized scratch
 *     buffers for the duration of the call.
 *   vp_plan_pass_config reports a pass's candidate count (0: the pass runs on
 *     the Stockham engine; the name is then "stockham", or "absent"), its
 *     current choice and that candidate's name ("W8 S4 alias": 8 pencils per
 *     CTA, 4 staging slots, aliased exchange), NUL-terminated within cap bytes.
 *   vp_plan_set_pass_config sets the choice (VP_ERR_INVALID_ARG for an index
 *     out of range, VP_ERR_UNSUPPORTED for a shape above a CTA's shared memory).
 * Every candidate computes the same result up to FP32 rounding order. */
vp_status vp_plan_autotune(vp_plan plan, int flags);
vp_status vp_plan_pass_config(vp_plan plan, int pass, int* cfg, int* count, char* name, size_t cap);
vp_status vp_plan_set_pass_config(vp_plan plan, int pass, int cfg);

/* Stream for subsequent calls (cudaStream_t as void*; NULL = legacy default).
 * One plan serves one stream at a time. */
vp_status vp_plan_set_stream(vp_plan plan, void* stream);

/* Apply arithmetic (default VP_FP32). */
vp_status vp_plan_set_precision(vp_plan plan, vp_precision precision);

/* Gradient definition (default VP_GRAD_EXACT).  EXACT builds the derivative
 * multipliers on the first gradient apply (FP64 precompute, synchronous). */
vp_status vp_plan_set_grad_mode(vp_plan plan, vp_grad_mode mode);

/* phi = T * f (Section 4): zero-pad to (2N)^d, forward FFT, multiply, inverse
 * FFT, crop.  f, phi: N^d elements of `dtype`. */
vp_status vp_apply(vp_plan plan, const void* f, void* phi, vp_dtype dtype);

/* phi = T * f (phi may be NULL) and grad_j = T_j * f (or the 2N-mode
 * derivative), all from one forward transform (Section 3: "any derivative
 * ... at the cost of an additional FFT").  grad: d * N^d elements. */
vp_status vp_apply_grad(vp_plan plan, const void* f, void* phi, void* grad, vp_dtype dtype);

/* The apply of vp_apply / vp_apply_grad on `count` densities in host memory,
 * pipelined: density i + 1 is copied to the device and the fields of density
 * i - 1 are copied back on two copy streams of the plan (the GPU's copy
 * engines) while density i is transformed on the plan's stream, so the
 * transfers hide behind the transforms.  f[i], phi[i], grad[i]: the N^d (phi)
 * and d * N^d (grad) element arrays of density i, `dtype` as for vp_apply;
 * page-locked host memory overlaps (pageable memory works, but its copies do
 * not overlap); device pointers are copied like host ones.  phi or grad may
 * be NULL (not both): NULL phi skips the potential, NULL grad the gradient.
 * The call returns when every output is in the caller's memory, also after a
 * failure part-way.  On first use the plan allocates 3 device slots of
 * (1 + fields) * N^d elements (or count slots when count < 3) and keeps them
 * until vp_destroy.  Errors: VP_ERR_INVALID_ARG for count < 0, a NULL array
 * or entry, phi[i] == f[i] or a dtype that does not match the plan;
 * VP_ERR_UNSUPPORTED for grad with a tensor-core precision; VP_ERR_OOM when
 * the slots do not fit.  Each output equals that of vp_apply / vp_apply_grad
 * on the same density bit for bit (the same kernels on the same workspace). */
vp_status vp_apply_pipeline(vp_plan plan, int count, const void* const* f, void* const* phi, void* const* grad,
                            vp_dtype dtype);

/* Copies a precomputed FP64 octant (prod_j (N_j+1) complex128 = 2 prod_j (N_j+1) doubles) to
 * host memory.  `axis` selects j for the gradient arrays (ignored otherwise);
 * `count` is the number of doubles available at host_dst. */
vp_status vp_plan_get_array(vp_plan plan, vp_array which, int axis, double* host_dst, size_t count);

/* Plan parameters and the device bytes it currently holds (N: the points of
 * axis 0; vp_plan_dims gives every axis). */
vp_status vp_plan_info(vp_plan plan, int* d, int* N, double* k, double* L, size_t* device_bytes);

/* Per-pass device timing with CUDA events recorded on the plan's stream
 * around every kernel launch (off by default).  vp_plan_get_timing
 * synchronises the stream, returns for each pass its name, launch count and
 * summed milliseconds since the last read, and resets the counters.
 * Up to `cap` passes are written; *npass receives the number of passes. */
vp_status vp_plan_set_timing(vp_plan plan, int enable);
vp_status vp_plan_get_timing(vp_plan plan, int cap, int* npass, const char** names, int* launches,
                             double* total_ms);

/* Number of kernel launches one vp_apply / vp_apply_grad issues. */
vp_status vp_plan_launch_count(vp_plan plan, int grad, int* launches);

/* Synchronises the plan's stream and reports the first device-side error:
 * a CUDA error, or VP_ERR_TIMEOUT when a bounded wait of a pass kernel gave
 * up -- the tensor-core pass's MMA completion or the FP32 fused pass's TMA
 * and multiplier pipeline (the error word is then cleared). */
vp_status vp_plan_status(vp_plan plan);

/* Message of the last failing call on this plan (plan may be NULL for
 * vp_plan_create failures; the message is then per thread). */
const char* vp_last_error(vp_plan plan);

const char* vp_status_string(vp_status status);

/* Every entry point that works on a device makes the plan's device current
 * for the call and restores the caller's current device before returning. */

/* Frees every device allocation of the plan.  NULL-safe. */
vp_status vp_destroy(vp_plan plan);

/* Whether 2N is a built FFT length (1) or not (0). */
int vp_fft_length_supported(int n2);


/* ---------------------------------------------------------------------------
 * Batched apply: many densities of different N, kernel and k in one persistent
 * launch (a batched form of the Section 4 apply; the paper has no batch).
 *
 * vp_batch_create takes `count` (<= 128) FP32 plans on one device (else
 * VP_ERR_INVALID_ARG) (d = 3 or 2, 2N in
 * {16, 24, 32, 48, 64, 96, 128, 192, 256}); the plans are borrowed and must
 * outlive the batch.  The batch owns one workspace per density.
 * vp_batch_apply computes phi_i = T_i * f_i for every i (device pointers,
 * complex64, N_i^d elements each; asynchronous on the batch's stream).  Every
 * pass of every density becomes tiles in one global work list, cut into work
 * items of `chunk` consecutive tiles of one pass; persistent CTAs take items in
 * pass-major order, wait (bounded) until the previous pass of the same density
 * has completed, and run an item's tiles with each tile's input staged while
 * the one before it is computed.  The launch and its counter reset run as one
 * CUDA graph, replayed per call.
 * Strategy: VP_BATCH_AUTO (default) times, on the first call, the persistent
 * kernel with chunks of 4, 8, 16 and 32 tiles on all resident CTAs and with
 * chunks of 8 at one CTA per SM, against per-density vp_apply launches
 * (serial, and forked over eight streams inside one CUDA graph), keeps the
 * fastest and caches the choice on disk (file $VP_AUTOTUNE_CACHE, default
 * ~/.cache/vp_autotune.txt) keyed by device, driver and the batch's sizes.
 * vp_batch_set_chunk fixes the chunk size (1..256; 0 = the autotuner's
 * choice, 8 before tuning); vp_batch_get_chunk reports the one in use.
 * Failure detection: a wait longer than the batch timeout (default about 2 s,
 * or VP_TIMEOUT_MS milliseconds from the environment at vp_batch_create;
 * vp_batch_set_timeout) records an error and lets the kernel finish;
 * vp_batch_status then returns VP_ERR_TIMEOUT.  vp_batch_withhold(b, i, p)
 * (p >= 1) makes pass p of density i wait for one tile more than its
 * predecessor has, so that path can be tested without a device fault;
 * p <= 0 restores every dependency.
 * ------------------------------------------------------------------------- */
typedef struct vp_batch_s* vp_batch;
typedef enum {
  VP_BATCH_AUTO = 0,
  VP_BATCH_PERSISTENT = 1,        /* persistent kernel, all resident CTAs */
  VP_BATCH_PERSISTENT_ONE_PER_SM = 2,
  VP_BATCH_PER_DENSITY = 3,       /* one vp_apply per density, for comparison */
  VP_BATCH_GRAPH_STREAMS = 4      /* per-density applies over 8 streams, one CUDA graph */
} vp_batch_strategy;
vp_status vp_batch_create(vp_batch* out, int count, const vp_plan* plans);
vp_status vp_batch_set_stream(vp_batch b, void* stream);
vp_status vp_batch_set_strategy(vp_batch b, int strategy);
vp_status vp_batch_get_strategy(vp_batch b, int* strategy);
vp_status vp_batch_set_chunk(vp_batch b, int chunk);
vp_status vp_batch_get_chunk(vp_batch b, int* chunk);
vp_status vp_batch_set_timeout(vp_batch b, double seconds);
vp_status vp_batch_withhold(vp_batch b, int density, int pass);
vp_status vp_batch_apply(vp_batch b, const void* const* f, void* const* phi);
vp_status vp_batch_status(vp_batch b);
vp_status vp_batch_info(vp_batch b, long long* items, int* passes, size_t* device_bytes);
const char* vp_batch_last_error(vp_batch b);
vp_status vp_batch_destroy(vp_batch b);

/* ---------------------------------------------------------------------------
 * Lippmann-Schwinger scattering on the volume potential (Section 5.3).
 *
 * For contrast q (real, N^3 floats) and incident field u_inc the scattered
 * field solves  A u = u - k^2 V[q u] = k^2 V[q u_inc] = b  with V the plan's
 * volume potential (3D Helmholtz plan, FP32 precision; complex64 vectors,
 * device pointers).  The paper solves the dual density form with Bi-CGStab;
 * vp_ls_solve runs right-preconditioned flexible GMRES(restart) (classical
 * Gram-Schmidt with one re-orthogonalisation; inner products from FP32
 * products and per-thread partial sums, summed across threads in FP64).  `precond`
 * (may be NULL) maps a residual r to z ~ A^-1 r on `stream`; if a
 * preconditioned cycle fails to reduce the residual the solve continues as
 * plain GMRES (stats->used_fallback).  The solve stops when the recurrence
 * residual is below tol or after maxit iterations; stats->true_residual is
 * ||b - A u|| / ||b|| with A (and b from u_inc, when given) evaluated in FP64.
 * ------------------------------------------------------------------------- */
typedef vp_status (*vp_precond_fn)(void* ctx, const void* r, void* z, void* stream);
typedef struct {
  double tol;
  int maxit;
  int restart;            /* 1..64 */
  int use_initial_guess;  /* 0: start from u = 0 */
  vp_precond_fn precond;
  void* precond_ctx;
} vp_ls_opts;
typedef struct {
  int iterations;
  int matvecs;
  int restarts;
  int used_fallback;
  double estimated_residual;
  double true_residual;
  double seconds;
} vp_ls_stats;
vp_status vp_ls_operator(vp_plan plan, const float* q, const void* u, void* out);
vp_status vp_ls_rhs(vp_plan plan, const float* q, const void* u_inc, void* b);
vp_status vp_ls_solve(vp_plan plan, const float* q, const void* b, const void* u_inc, void* u, const vp_ls_opts* opts,
                      vp_ls_stats* stats);
/* One training pair for the learned preconditioner from solver iterates:
 * r = b - A u_s (u_s may be NULL: r = b), e = u_star - u_s (A e = r); with
 * s = sqrt(N^3)/||r|| writes the network input x = (s Re r, s Im r, q) as
 * 3 x N^3 floats and the target t = s (e - r) as 2 x N^3 floats. */
vp_status vp_ls_training_pair(vp_plan plan, const float* q, const void* b, const void* u_s, const void* u_star,
                              float* x_out, float* t_out, double* rnorm);
/* Orthonormal Krylov basis of the plain operator started from b: the vectors
 * v_0 = b/||b||, v_1, ..., v_m that the first cycle of unpreconditioned GMRES
 * builds (classical Gram-Schmidt applied twice, as in vp_ls_solve), with
 * A [v_0..v_{m-1}] = [v_0..v_m] H, H upper Hessenberg with h_{j+1,j} > 0.
 * V: device buffer of (m+1) x N^3 complex64, vector j at offset j N^3;
 * *count: vectors written (m+1; fewer only at an exact breakdown).  m in
 * [1, 64].  Draws the (A v_j, v_j) training pairs of the learned preconditioner. */
vp_status vp_ls_krylov_basis(vp_plan plan, const float* q, const void* b, int m, void* V, int* count);
/* The preconditioned directions z_j = M(v_j), j < m, of the first cycle of
 * flexible GMRES from b with the right preconditioner `precond` (required):
 * the vectors whose images A z_j span that cycle's search space.  Z: device
 * buffer of m x N^3 complex64; *count: directions written (m; fewer only when
 * the recurrence residual is exactly zero).  Draws on-policy training pairs
 * (A z_j, z_j) for the learned preconditioner. */
vp_status vp_ls_flexible_basis(vp_plan plan, const float* q, const void* b, int m, vp_precond_fn precond,
                               void* precond_ctx, void* Z, int* count);
/* The paper's solver (Section 5.3): unpreconditioned Bi-CGStab (van der Vorst
 * 1992; two operator products per iteration, each one apply of V) on either
 * form of the scattering problem, u the scattered field:
 *   VP_LS_FIELD:    u - k^2 V[q u] = k^2 V[q u_inc]
 *   VP_LS_DENSITY:  s - k^2 q V[s] = k^2 q u_inc,  u = V[s]   (the paper's
 *                   dual equation of Section 5.3)
 * plan: 2D or 3D Helmholtz plan.  dtype VP_C64: complex64 u_inc/u and a float
 * contrast q, the plan in VP_FP32; VP_C128: complex128 and double q, the plan
 * in VP_FP64.  q, u_inc, u: N^d device arrays in the plan's layout (u is
 * overwritten; it may not alias u_inc).  Starts from zero; stops when the
 * recurrence residual ||r|| / ||b|| < tol, checked after each half step (as
 * the paper's counts imply) and each full step, or after maxit iterations
 * (VP_OK either way: compare stats->estimated_residual with tol).
 * history: NULL or a host array of maxit + 1 doubles receiving ||r_j|| / ||b||
 * for j = 0 .. stats->iterations (the last entry ||s|| / ||b|| when the solve
 * stops at a half step).  stats: iterations (begun), matvecs (operator
 * products of the iteration; the right-hand side's apply, and the final
 * u = V[s] of the density form, are not counted), estimated_residual,
 * true_residual = ||b - M x|| / ||b|| for the solved form with M and b
 * evaluated in FP64, seconds (right-hand side, iteration and final apply).
 * Returns VP_ERR_NUMERICAL on a breakdown (a zero inner product) or a
 * non-finite value, with u the last iterate. */
enum { VP_LS_FIELD = 0, VP_LS_DENSITY = 1 };
vp_status vp_ls_bicgstab(vp_plan plan, const void* q, const void* u_inc, void* u, vp_dtype dtype, int form,
                         double tol, int maxit, double* history, vp_ls_stats* stats);
/* The same solve with FP64 accuracy at mostly FP32 cost (a project addition:
 * GB300 runs FP64 arithmetic at a small fraction of its FP32 rate): Bi-CGStab
 * with reliable updates (Sleijpen & van der Vorst 1996).  The recurrence runs
 * on the FP32 apply and accumulates a correction; whenever its residual has
 * fallen below delta times the largest residual since the last update (or
 * below tol), the correction is added to the FP64 solution and the true
 * residual b - M x, formed with the FP64 apply, replaces the recurrence
 * residual.  The solve stops when the true residual is below tol ||b||.
 * FP32 products slow Bi-CGStab down on strongly indefinite problems (measured:
 * the filtered disk at 80 wavelengths); when the FP32 phase has not converged
 * after maxit iterations, or three consecutive updates each gain less than 2x,
 * or it breaks down, FP64 Bi-CGStab (vp_ls_bicgstab's iteration, at most
 * maxit iterations) solves the correction equation M e = b - M x from the
 * mixed iterate x to the same tol ||b||, u is x + e (field) or V[s + e]
 * (density), and stats->used_fallback is set.
 * q: N^d doubles, u_inc/u: complex128 device arrays; the plan's precision may
 * be VP_FP32 or VP_FP64 (it is switched internally and restored).  delta in
 * (0, 1), e.g. 0.01.  stats: matvecs = operator products (FP32, plus the
 * FP64 ones of a fallback), restarts = the number of updates (one FP64 product
 * each), estimated_residual = the last true residual; other fields as for
 * vp_ls_bicgstab.  history[j]: the FP32
 * recurrence residual ||r_j|| / ||b|| after iteration j. */
vp_status vp_ls_bicgstab_mixed(vp_plan plan, const double* q, const void* u_inc, void* u, int form, double tol,
                               double delta, int maxit, double* history, vp_ls_stats* stats);
/* Variable-coefficient Poisson (linearised Poisson-Boltzmann with lambda = 0,
 * Section 5.2): div(eps grad phi) = rho with phi = V[sigma], V the Laplace
 * volume potential, gives the second-kind equation (eq. pbeq)
 *     -eps sigma + grad(eps) . grad V[sigma] = rho,
 * whose operator products use the exact-gradient apply (Section 3).  Solved
 * with the Bi-CGStab iteration of vp_ls_bicgstab (the paper uses GMRES).
 *   plan: 2D or 3D Laplace plan (derivative multipliers built on first use)
 *   eps: N^d reals; grad_eps: d blocks of N^d reals (d eps / d x_j); rho,
 *   sigma: N^d complex (real data: zero imaginary parts); device pointers.
 *   vp_pb_solve: dtype VP_C64 (float eps, FP32 plan) or VP_C128 (double, FP64);
 *   vp_pb_solve_mixed: FP64 data, FP32 iterations with FP64 reliable updates
 *   (as vp_ls_bicgstab_mixed).  The potential is phi = V[sigma] (vp_apply).
 * tol, maxit, history, stats and errors as for vp_ls_bicgstab. */
vp_status vp_pb_solve(vp_plan plan, const void* eps, const void* grad_eps, const void* rho, void* sigma,
                      vp_dtype dtype, double tol, int maxit, double* history, vp_ls_stats* stats);
vp_status vp_pb_solve_mixed(vp_plan plan, const double* eps, const double* grad_eps, const void* rho, void* sigma,
                            double tol, double delta, int maxit, double* history, vp_ls_stats* stats);
/* The same equation solved with restarted GMRES(m), the paper's solver for it
 * (Section 5.2; Saad & Schultz 1986), in FP64 on an FP64 plan: eps, grad_eps
 * as above (doubles), rho and sigma complex128 device arrays.  Arnoldi with
 * classical Gram-Schmidt applied twice (inner products summed in FP64 in a
 * fixed order: repeated solves are bit-identical), Givens rotations on the
 * host; each cycle restarts from the explicit residual rho - P sigma.
 *   restart: m in [1, 512] (the basis holds m + 1 vectors of N^d complex128;
 *            m is capped at maxit); maxit: the budget of Arnoldi steps.
 *   history[0..iterations] (maxit + 1 doubles, or NULL): |g_{j+1}| / ||rho||
 *            after step j + 1 (the GMRES residual estimate), replaced at a
 *            restart by the explicit residual.
 *   stats: iterations = Arnoldi steps, matvecs = operator products (one per
 *          step, plus one per restart), restarts (cycles begun from an
 *          explicit residual), estimated_residual (the last
 *          estimate), true_residual = ||rho - P sigma|| / ||rho|| (FP64),
 *          seconds.
 * Stops when the estimate (or the explicit residual at a restart) is below
 * tol, or after maxit steps (VP_OK; see stats).  rho = 0 gives sigma = 0 and
 * no iterations.  VP_ERR_NUMERICAL on a non-finite value or a breakdown
 * without convergence (a zero column of H), sigma the last iterate. */
vp_status vp_pb_gmres(vp_plan plan, const double* eps, const double* grad_eps, const void* rho, void* sigma,
                      double tol, int restart, int maxit, double* history, vp_ls_stats* stats);
const char* vp_ls_last_error(void);

/* ---------------------------------------------------------------------------
 * Learned right preconditioner for vp_ls_solve (a project addition; the
 * paper's solver is unpreconditioned).  A 3-level 3D U-Net on one S^3 sample
 * (S divisible by 4, C = 16 channels), channel-major float tensors [C][S][S][S]:
 * E1a 3->C, E1b C->C -> s1; 2x2x2 mean pool; E2a, E2b -> s2; pool; B1, B2;
 * nearest x2 up, concat with s2, D2a 2C->C, D2b; up, concat with s1, D1a 2C->C,
 * D1b C->2.  Every conv is 3x3x3, zero padding 1, with bias and leaky ReLU
 * (slope 0.1) except D1b.  Weights are bfloat16-rounded copies of FP32 master
 * weights.  The convolutions run on the tensor cores: the BF16 weights times
 * the two BF16 parts (hi, lo) of each FP32 activation, accumulated in FP32, so
 * they agree with FP32 arithmetic to about 2^-16 relative; the weight
 * gradients likewise (both operands split, FP32 partial sums per CTA reduced in
 * FP64); pooling, upsampling and activations are FP32.  Parameter layout for set/get: for each layer in
 * that order, w[C_out][C_in][27] (k = (kz*3 + ky)*3 + kx) then b[C_out].
 * Input channels: (Re r, Im r, q) with r scaled to unit RMS (sqrt(n) r/||r||);
 * output: the deviation of the correction from r, in the same scale.
 * vp_unet_loss_grad runs forward and backward for the mean squared error and
 * keeps the gradients; vp_unet_adam_step applies Adam (beta 0.9/0.999, eps 1e-8).
 * vp_unet_precond is a vp_precond_fn (ctx = the network, bound to a contrast
 * with vp_unet_bind): z = r + (||r||/sqrt(n)) net(sqrt(n) r/||r||, q), so a
 * network with a zero last layer is the identity (plain GMRES).
 * Calls are asynchronous on the network's stream.  A convolution whose wait
 * for its MMAs runs past a bounded clock budget sets a device error word
 * instead of hanging: vp_unet_status synchronises the stream and returns
 * VP_ERR_TIMEOUT if it is set (vp_unet_precond checks it on every call, and
 * vp_unet_loss_grad when it returns the loss).
 * ------------------------------------------------------------------------- */
typedef struct vp_unet_s* vp_unet;
vp_status vp_unet_create(vp_unet* out, int S, int C);
vp_status vp_unet_param_count(vp_unet net, size_t* count);
vp_status vp_unet_set_stream(vp_unet net, void* stream);
vp_status vp_unet_set_weights(vp_unet net, const float* host, size_t count);
vp_status vp_unet_get_weights(vp_unet net, int which /* 0 FP32, 1 BF16-rounded, 2 gradients */, float* host,
                              size_t count);
vp_status vp_unet_forward(vp_unet net, const float* in, float* out);
vp_status vp_unet_loss_grad(vp_unet net, const float* in, const float* target, double* loss);
vp_status vp_unet_adam_step(vp_unet net, double lr);
/* Training checkpoints: Adam's first and second moments (vp_unet_param_count
 * floats each, host memory) and its step count.  vp_unet_set_weights resets
 * them, so a resume calls vp_unet_set_weights, then vp_unet_set_adam; the
 * next vp_unet_adam_step then continues exactly as the saved run would have.
 * VP_ERR_INVALID_ARG for a NULL argument, a count other than the parameter
 * count or a negative step.  Both synchronise the network's stream. */
vp_status vp_unet_get_adam(vp_unet net, float* m, float* v, size_t count, long long* step);
vp_status vp_unet_set_adam(vp_unet net, const float* m, const float* v, size_t count, long long step);
/* Leaky-ReLU slope in [0, 1] (default 0.1); 1 makes the network linear in its input. */
vp_status vp_unet_set_slope(vp_unet net, double slope);
vp_status vp_unet_bind(vp_unet net, const float* q);
vp_status vp_unet_precond(void* ctx, const void* r, void* z, void* stream);
vp_status vp_unet_status(vp_unet net);
/* Budget of each bounded wait of the tensor-core kernels (default about 2 s,
 * or VP_TIMEOUT_MS milliseconds from the environment at vp_unet_create;
 * seconds > 0).  vp_unet_withhold is a test hook: on != 0 makes the kernels
 * issue no MMAs, so their waits run out and the next status check reports
 * VP_ERR_TIMEOUT.  Every report clears the error word. */
vp_status vp_unet_set_timeout(vp_unet net, double seconds);
vp_status vp_unet_withhold(vp_unet net, int on);
const char* vp_unet_last_error(vp_unet net);
vp_status vp_unet_destroy(vp_unet net);

/* ---------------------------------------------------------------------------
 * Potential apply without device allocation (the paper has no counterpart;
 * this is a deployment aid).
 *
 * For callers that cannot call cudaMalloc where they apply the operator: code
 * living inside another framework whose allocator owns all device memory,
 * latency-bound loops that cannot afford an allocation's implicit
 * synchronisation, or plug-ins that may allocate only while initialising.
 * Create the plan during set-up (plan creation allocates the multiplier), then
 * call this instead of vp_apply: it computes the same phi = T * f with the same
 * kernels, taking its scratch from one array of VP_NOALLOC_SCRATCH_BYTES
 * compiled into the library, and calls no allocation routine.
 *   - f, phi: device pointers (host pointers return VP_ERR_INVALID_ARG); no
 *     gradients.  dtype as for vp_apply.
 *   - Grids whose scratch exceeds the array return VP_ERR_UNSUPPORTED with a
 *     message: scratch = 6 N^3 (3D) or 2 N^2 (2D) complex elements of the plan's
 *     precision, e.g. up to N = 128 (3D) and N = 2048 (2D) in FP32.
 *   - The array is shared by every call on a device and keeps the last call's
 *     contents (nothing needs to start at zero).  Calls whose kernels overlap
 *     on the GPU race on it: serialise them (one stream, or events).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with the plan's device current; make that first
 *     call before any stream capture.  Under CUDA's default lazy module loading
 *     that lookup is also what loads the array onto the device, so the first
 *     call allocates it (and can fail with VP_ERR_CUDA when the device memory
 *     is exhausted then); with eager loading (CUDA_MODULE_LOADING=EAGER) it is
 *     allocated when the library's context is set up.  Either way the device
 *     holds it until the process exits.
 *   - The address is cached per process and per device: do not reset a device
 *     (cudaDeviceReset) between calls, which would leave it stale.
 * ------------------------------------------------------------------------- */
#define VP_NOALLOC_SCRATCH_BYTES (128u * 1024u * 1024u)
vp_status vp_apply_noalloc(vp_plan plan, const void* f, void* phi, vp_dtype dtype);

#ifdef __cplusplus
}
#endif

#endif /* VP_H */
