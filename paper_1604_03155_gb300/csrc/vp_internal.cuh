// vp_internal.cuh -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/vp.h"
#include "pencil_fft.cuh"

namespace vp {

// The default budget of the bounded device waits of batches and networks from
// the environment: VP_TIMEOUT_MS (milliseconds, > 0) in seconds, else 0 (keep
// the built-in default).  Read at vp_batch_create and vp_unet_create.
inline double env_timeout_seconds() {
  const char* s = getenv("VP_TIMEOUT_MS");
  if (!s || !*s) return 0.0;
  char* end = nullptr;
  const double ms = strtod(s, &end);
  return (end && *end == '\0' && ms > 0.0 && ms < 1e12) ? ms * 1e-3 : 0.0;
}

// VP_LOG from the environment (read once): 0 silent (default), 1 every error
// message the library records, 2 also the autotuners' choices.  Messages go
// to stderr, one line each, prefixed "vp: ".
int log_level();
void log_line(int level, const char* what, const std::string& msg);

// An NVTX range (domain-less push/pop) for the scope: the library's entry
// points and pass launches appear by name in profilers (ncu --nvtx
// --nvtx-include "fused_axis0/"); without a tool attached it costs a function
// pointer test.
class NvtxRange {
 public:
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Gauss-Legendre nodes of the 2D Helmholtz spectrum near s = k.
constexpr int GL_NODES = 24;
// |s - k| below which the 2D Helmholtz numerator is a divided difference.
constexpr double HELM2D_NEAR_K = 1.0;
// x = Ls below which the biharmonic spectra are summed from their power series
constexpr double BIHARM_SERIES_X = 2.0;

// precompute.cu
cudaError_t set_gauss_legendre(const double* x, const double* w);
cudaError_t launch_spectrum(double2* G, int d, const int* M1s, int kernel, double k, double L, cudaStream_t s);
cudaError_t launch_matrix(double* M, int N, int type, cudaStream_t s);
cudaError_t launch_axis_transform(const double2* in, double2* out, const double* M, long long O, int P, int Q,
                                  long long I, cudaStream_t s);
cudaError_t launch_narrow(const double2* in, float2* out, long long count, cudaStream_t s);
cudaError_t launch_finalize(const double2* in, double2* out_u, double2* out64, float2* out32, long long count,
                            double scale, int times_minus_i, cudaStream_t s);
cudaError_t launch_twiddles(double2* tw64, float2* tw32, int n, cudaStream_t s);

// Makes `dev` current for the guard's scope and restores the caller's current
// device when it ends, so that no entry point leaves another device current.
class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
    if (prev_ != dev) {
      err_ = cudaSetDevice(dev);
      switched_ = (err_ == cudaSuccess && prev_ >= 0);
    }
  }
  ~DeviceGuard() {
    if (switched_) cudaSetDevice(prev_);
  }
  cudaError_t error() const { return err_; }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;

 private:
  int prev_ = -1;
  bool switched_ = false;
  cudaError_t err_ = cudaSuccess;
};
#define VP_CAT2(a, b) a##b
#define VP_CAT(a, b) VP_CAT2(a, b)

// Pass kinds of the apply.
enum PassKind { FWD_CONTIG = 0, FWD_STRIDED = 1, INV_CONTIG = 2, INV_STRIDED = 3, FUSED_STRIDED = 4 };

struct PassShape {
  int threads;
  int W;
  size_t smem;
};

// apply_*.cu: launch one pass for FFT length n.  Returns cudaErrorInvalidValue
// when n is not built.
cudaError_t launch_pass_f32(PassKind kind, int n, const PassArgs<float>& a, cudaStream_t s);
cudaError_t launch_pass_f64(PassKind kind, int n, const PassArgs<double>& a, cudaStream_t s);
bool pass_shape_f32(PassKind kind, int n, PassShape* out);
// fourstep.cu: launches an FP32 pass on the four-step kernels when they serve
// its length and arguments (returns false otherwise, *err untouched).
bool launch_fourstep(PassKind kind, int n, const PassArgs<float>& a, cudaStream_t s, cudaError_t* err);
// The candidate tile shapes of a four-step pass (names, and whether each fits
// a CTA's shared memory); returns their count, 0 for other lengths.
int fourstep_shapes(PassKind kind, int n, char (*names)[32], bool* fits);
// On-disk autotuner cache (batch.cu): value for key (0 when absent), append.
int autotune_cache_lookup(const std::string& key);
void autotune_cache_store(const std::string& key, int value);
// Whether the four-step engine runs this pass (length, data type, alignment).
bool fourstep_serves(PassKind kind, int n, const PassArgs<float>& a);
bool pass_shape_f64(PassKind kind, int n, PassShape* out);

// FFT lengths with compiled passes (2N).
bool fft_length_built(int n);

// tc_fused.cu: the fused axis-0 pass of the 3D apply on the tensor cores
// (2N = 256 or 512).  split: 0 BF16 x 2, 1 FP16 x 2 (scaled), 2 BF16 x 3.
struct TcFusedArgs {
  const float2* in;    // spectrum after the two forward passes (in place allowed)
  float2* out;
  long long pitch_pos; // element stride between positions along axis 0 (= (2N)^2)
  long long npencils;  // pencils (= (2N)^2), a multiple of 8
  const float2* mult;  // FP32 multiplier octant (N+1)^3, pre-scaled by 1/(2N)^3
  const float2* tw;    // twiddles exp(-2 pi i q/2N), q in [0, 2N)
  const uint16_t* bmat;  // DFT matrices from tc_build_bmat
  int* err;            // device error word: bit 0 = a bounded wait timed out
};
bool tc_length_supported(int n);
size_t tc_bmat_bytes(int n, int split);
cudaError_t tc_build_bmat(int n, int split, uint16_t* out, cudaStream_t s);
cudaError_t launch_tc_fused(int n, int split, const TcFusedArgs& a, cudaStream_t s);

// vp_capi.cu: the device a plan was created on; the scratch bytes of one
// potential-only apply; that apply on a caller-supplied workspace (device
// pointers only, allocates nothing).
int plan_device(vp_plan p);
cudaStream_t plan_stream(vp_plan p);
int plan_is_fp32(vp_plan p);
int plan_is_fp64(vp_plan p);
// Nystrom entries (entries.cu): the plan's FP64 kernel octant T (which =
// VP_ARRAY_T) or T_axis (VP_ARRAY_TJ, built on first use), a device flag word
// owned by the plan, and the plan's error message.
vp_status plan_kernel_octant(vp_plan p, int which, int axis, const double2** oct);
vp_status plan_kernel_octant32(vp_plan p, int which, int axis, const float2** oct);
int* plan_flag_word(vp_plan p);
vp_status entries_fail(vp_plan p, vp_status st, const char* msg);
// ls.cu: the message vp_ls_last_error returns on this thread
void ls_set_error(const char* msg);
// The FP32 potential-only passes of a plan on workspace `ws` (input and output
// pointers left NULL): fills args/kinds and each pass's transform length,
// returns the number of passes.
int plan_pass_args_f32(vp_plan p, float2* ws, PassArgs<float>* args, int* kinds, int* lens);
size_t plan_apply_workspace_bytes(vp_plan p);
vp_status apply_with_workspace(vp_plan p, const void* f, void* phi, vp_dtype dtype, void* ws, size_t ws_bytes);
// The exact gradient (d fields, d blocks of N^d) on a caller workspace of
// plan_grad_workspace_bytes; the derivative multipliers must have been built
// (plan_prepare_grad) before, e.g. outside a stream capture.
int plan_kernel(vp_plan p);
// per-axis grids: not all N_j equal; N_0 N_1 (N_2) points; N_j per axis (1 beyond d)
int plan_is_aniso(vp_plan p);
long long plan_points(vp_plan p);
void plan_dims(vp_plan p, int* N);
vp_status plan_prepare_grad(vp_plan p);
size_t plan_grad_workspace_bytes(vp_plan p);
vp_status apply_grad_with_workspace(vp_plan p, const void* f, void* grad, vp_dtype dtype, void* ws, size_t ws_bytes);

// 3x3x3 convolution of the U-Net on the tensor cores (unet_tc.cu): channel-major
// FP32 activations [C][S][S][S], the input the concatenation of x1 (c1
// channels) and x2 (c2, may be 0), weights w[co][ci][27] holding BF16 values,
// optional bias, leaky ReLU (slope) when act; a timed-out wait sets *err.
namespace unet_tc {
struct ConvArgs {
  const float* x1;
  int c1;
  const float* x2;
  int c2;
  const float* w;
  const float* bias;
  float* y;
  int co, S, act;
  float slope;
  int* err;
  long long wait_cycles;  // budget of each bounded wait (clock cycles)
  int withhold;           // test hook: issue no MMAs, so the waits run out
};
cudaError_t conv3d(const ConvArgs& a, cudaStream_t s);
// Weight and bias gradients of a convolution (input x1, x2 as in ConvArgs,
// dy: co <= 16 channels at the output) as nblk per-CTA partials
// part[blk][(ci * 27 + tap) * co + o] and part[blk][(c1 + c2) * 27 * co + o].
struct WgradArgs {
  const float* x1;
  int c1;
  const float* x2;
  int c2;
  const float* dy;
  int co;
  float* part;
  int nblk, S;
  int* err;
  long long wait_cycles;
  int withhold;
};
cudaError_t wgrad3d(const WgradArgs& a, cudaStream_t s);
// output row segments of an S^3 grid (at most this many CTAs do work)
long long wgrad_rows(int S);
}  // namespace unet_tc

}  // namespace vp
