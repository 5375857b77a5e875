// pencil_fft.cuh -- batched pencil FFT passes of the apply (Section 4 of
// Vico, Greengard & Ferrando: zero-pad to (2N)^d, FFT, multiply, inverse FFT,
// crop).  One pass transforms one axis of a batch of pencils of length n = 2N.
//
// Engine: Stockham auto-sort FFT.  A pencil is held by T_p = n/E threads, E
// complex values each, in registers.  Each stage of radix R performs E/R
// radix-R butterflies per thread; between stages the values go through shared
// memory once (write, barrier, read).  Stage s with Ns = product of the radices
// before it reads butterfly j's inputs at j + r n/R, twiddles them by
// w^(k r n/(Ns R)) with k = j mod Ns, and writes output r to
// (j/Ns) Ns R + k + r Ns.  The first stage reads global memory directly and the
// last writes global memory directly.
//
// Memory pipeline: CTAs are persistent (the grid is the SM count times the
// resident CTAs per SM) and walk the tiles with a grid stride.  The input of
// the next tiles is staged into shared memory with 16-byte cp.async copies
// (NSTG-deep ring) while the current tile's butterflies run, so the SM keeps
// HBM requests in flight through the compute phases.
//
// Pruning: the forward input is f zero-padded from N to 2N, so the first
// stage (Ns = 1) loads only r < R/2 (positions < N) and never reads the zero
// half.  The inverse output is cropped to N, so the last inverse stage stores
// only r < R/2.  The inverse runs the radices in reverse order; then its first
// stage reads exactly the positions the forward's last stage wrote, in the same
// registers, so a fused forward -> multiply -> inverse pencil needs no
// exchange at the turn.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vp {

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename Real> struct CxT;
template <> struct CxT<float> { using T = float2; };
template <> struct CxT<double> { using T = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cconjmul(C a, C b) {  // a * conj(b)
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C mul_mi(C a) {
  return INV ? C{-a.y, a.x} : C{a.y, -a.x};
}
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return {a.x * s, a.y * s}; }

// ---------------------------------------------------------------------------
// small DFT codelets, in place on v[0..R-1], forward sign -1 (INV: +1)
// ---------------------------------------------------------------------------
template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<2, INV> {
  template <typename C> __device__ __forceinline__ static void run(C* v) {
    C a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  }
};

template <bool INV> struct Dft<3, INV> {
  template <typename C> __device__ __forceinline__ static void run(C* v) {
    using R = decltype(v[0].x);
    const R s3 = (R)0.86602540378443864676;  // sin(2 pi/3)
    C t1 = cadd(v[1], v[2]);
    C t2 = {v[0].x - (R)0.5 * t1.x, v[0].y - (R)0.5 * t1.y};
    C d = csub(v[1], v[2]);
    C t3 = mul_mi<INV>(cscale(d, s3));  // -i sin(2pi/3) (b - c) forward
    v[0] = cadd(v[0], t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
  }
};

template <bool INV> struct Dft<4, INV> {
  template <typename C> __device__ __forceinline__ static void run(C* v) {
    C t0 = cadd(v[0], v[2]);
    C t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]);
    C t3 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

// R = 8: two radix-4 transforms on the even/odd samples, then radix-2 with w8^k.
template <bool INV> struct Dft<8, INV> {
  template <typename C> __device__ __forceinline__ static void run(C* v) {
    using R = decltype(v[0].x);
    const R h = (R)0.70710678118654752440;
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, INV>::run(e);
    Dft<4, INV>::run(o);
    // w8^1 = (1 -+ i) h, w8^2 = -+ i, w8^3 = (-1 -+ i) h  (upper sign forward)
    C o1 = INV ? C{(o[1].x - o[1].y) * h, (o[1].x + o[1].y) * h} : C{(o[1].x + o[1].y) * h, (o[1].y - o[1].x) * h};
    C o2 = mul_mi<INV>(o[2]);
    C o3 = INV ? C{(-o[3].x - o[3].y) * h, (o[3].x - o[3].y) * h} : C{(o[3].y - o[3].x) * h, (-o[3].x - o[3].y) * h};
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

// R = 16 = 4 x 4: sample n = j2 + 4 j1; Y[j2][k1] = DFT4_j1; X[k1 + 4 k2] =
// DFT4_j2(w16^(j2 k1) Y[j2][k1]).
template <bool INV> struct Dft<16, INV> {
  template <typename C> __device__ __forceinline__ static void run(C* v) {
    using R = decltype(v[0].x);
    const R c1 = (R)0.92387953251128675613;  // cos(pi/8)
    const R s1 = (R)0.38268343236508977173;  // sin(pi/8)
    const R h = (R)0.70710678118654752440;
    C y[4][4];
#pragma unroll
    for (int j2 = 0; j2 < 4; ++j2) {
      y[j2][0] = v[j2];
      y[j2][1] = v[j2 + 4];
      y[j2][2] = v[j2 + 8];
      y[j2][3] = v[j2 + 12];
      Dft<4, INV>::run(y[j2]);
    }
    // twiddles w16^(j2 k1), w16 = exp(-+ 2 pi i/16); tw(m) = (cos(m pi/8), -+ sin(m pi/8))
    const R cs[10] = {(R)1, c1, h, s1, (R)0, -s1, -h, -c1, (R)-1, -c1};
    const R sn[10] = {(R)0, s1, h, c1, (R)1, c1, h, s1, (R)0, -s1};
#pragma unroll
    for (int j2 = 1; j2 < 4; ++j2) {
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) {
        const int m = j2 * k1;  // <= 9
        C w = {cs[m], INV ? sn[m] : -sn[m]};
        y[j2][k1] = cmul(y[j2][k1], w);
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C z[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      Dft<4, INV>::run(z);
      v[k1] = z[0];
      v[k1 + 4] = z[1];
      v[k1 + 8] = z[2];
      v[k1 + 12] = z[3];
    }
  }
};

// R = 32: radix-16 transforms of the even and odd samples, then radix 2 with
// w32^k = cos(pi k/16) -+ i sin(pi k/16).
template <bool INV> struct Dft<32, INV> {
  template <typename C> __device__ __forceinline__ static void run(C* v) {
    using R = decltype(v[0].x);
    // cos(pi k/16), k = 0..8
    const R c[9] = {(R)1,
                    (R)0.98078528040323044913,
                    (R)0.92387953251128675613,
                    (R)0.83146961230254523708,
                    (R)0.70710678118654752440,
                    (R)0.55557023301960222474,
                    (R)0.38268343236508977173,
                    (R)0.19509032201612826785,
                    (R)0};
    C e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    Dft<16, INV>::run(e);
    Dft<16, INV>::run(o);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      // cos(pi k/16) and sin(pi k/16) = cos(pi (8-k)/16)
      const R ck = k <= 8 ? c[k] : -c[16 - k];
      const R sk = k <= 8 ? c[8 - k] : c[k - 8];
      const C w = {ck, INV ? sk : -sk};
      const C t = cmul(o[k], w);
      v[k] = cadd(e[k], t);
      v[k + 16] = csub(e[k], t);
    }
  }
};

// ---------------------------------------------------------------------------
// compile-time plan: radices chosen greedily (16, 8, 4, 3, 2) dividing both the
// remaining length and the per-thread count E.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pick_radix(int rem, int E) {
  return (rem % 32 == 0 && E % 32 == 0)  ? 32
         : (rem % 16 == 0 && E % 16 == 0)  ? 16
         : (rem % 8 == 0 && E % 8 == 0)  ? 8
         : (rem % 4 == 0 && E % 4 == 0)  ? 4
         : (rem % 3 == 0 && E % 3 == 0)  ? 3
         : (rem % 2 == 0 && E % 2 == 0)  ? 2
                                         : 0;
}
__host__ __device__ constexpr int plan_nstages(int n, int E) {
  int rem = n, c = 0;
  while (rem > 1) {
    int r = pick_radix(rem, E);
    if (r == 0) return -1;
    rem /= r;
    ++c;
  }
  return c;
}
__host__ __device__ constexpr int plan_radix(int n, int E, int s) {
  int rem = n;
  for (int i = 0; i < s; ++i) rem /= pick_radix(rem, E);
  return pick_radix(rem, E);
}
__host__ __device__ constexpr int stage_radix(int n, int E, bool inv, int s) {
  return plan_radix(n, E, inv ? plan_nstages(n, E) - 1 - s : s);
}
__host__ __device__ constexpr int stage_ns(int n, int E, bool inv, int s) {
  int p = 1;
  for (int i = 0; i < s; ++i) p *= stage_radix(n, E, inv, i);
  return p;
}

// Per-thread element count: 16 (24 with a factor 3) in FP32, 8 (12) in FP64.
template <typename Real> __host__ __device__ constexpr int elems_per_thread(int n) {
  return (n % 3 == 0) ? (sizeof(Real) == 4 ? (n >= 24 ? 24 : 12) : 12)
                      : (sizeof(Real) == 4 ? (n >= 16 ? 16 : 8) : 8);
}

// ---------------------------------------------------------------------------
// shared-memory exchange layouts
//  contiguous pencils: element (w, pos) at w*P + pos + (pos >> SH), P odd:
//    radix-strided positions of one pencil and equal positions of different
//    pencils both fall in distinct banks;
//  strided pencils: e = pos*W + w at e + (e >> SH): the W pencils of a row are
//    adjacent (as in global memory) and one pad per 2^SH elements spreads
//    radix-strided rows over the banks.
// SH = 4 for 8-byte elements (16 per 128-byte row), 3 for 16-byte elements.
// ---------------------------------------------------------------------------
template <typename Real> struct SmemLayout {
  static constexpr int SH = sizeof(Real) == 4 ? 4 : 3;
};
template <typename Real> __host__ __device__ constexpr int smem_pitch(int n) {
  return n + (n >> SmemLayout<Real>::SH) + 1;
}
template <typename Real> __host__ __device__ constexpr int xchg_elems(int n, int W, bool contig) {
  return contig ? W * smem_pitch<Real>(n) : (n * W + ((n * W) >> SmemLayout<Real>::SH) + 1);
}

enum PassMode { MODE_FWD = 0, MODE_INV = 1, MODE_FUSED1 = 2, MODE_FUSEDN = 3 };

// Pencils per CTA: 256 threads' worth; strided passes take at least 8 pencils
// (64-byte row segments) and at most 64; bounded by an exchange buffer of
// `budget` bytes (40 KB; 72 KB for the fused passes, which measured faster
// with wider tiles and fewer, larger CTAs).
template <typename Real>
__host__ __device__ constexpr int pencils_per_cta(int n, bool contig, int E, int budget = 40 * 1024) {
  int Tp = n / E;
  int w = 256 / Tp;
  if (w < 1) w = 1;
  if (!contig) {
    if (w < 8) w = 8;
    if (w > 64) w = 64;
  } else if (w > 32) {
    w = 32;
  }
  while (w > 1 && (long)xchg_elems<Real>(n, w, contig) * 2 * (long)sizeof(Real) > budget) w >>= 1;
  while (w > 1 && w * Tp > 1024) w >>= 1;
  return w;
}

// Input elements of one tile's first stage per pencil (pruned forward: N).
__host__ __device__ constexpr int stage_in_len(int n, int mode) { return mode == MODE_INV ? n : n / 2; }

// ---------------------------------------------------------------------------
// multiplier fields of the fused pass
// ---------------------------------------------------------------------------
struct FieldDesc {
  const void* mult;   // octant (N+1)^d of complex Real, pre-scaled by 1/(2N)^d
  int odd_axis;       // -1, or the axis along which the octant is extended oddly
  int spectral_axis;  // -1, or axis j for the 2N-mode factor i pi m_j (Nyquist 0)
};

template <typename Real> struct PassArgs {
  using C = typename CxT<Real>::T;
  const void* in;
  void* out;
  long long in_pitch_o, in_pitch_pos;    // element strides of the input
  long long out_pitch_o, out_pitch_pos;  // element strides of the output
  long long out_field_stride;            // between fused output fields
  int O;       // outer count: rows (contiguous pencils) or slabs (strided)
  int I;       // inner count of strided pencils (1 for contiguous)
  int nblk_i;  // ceil(I / W)
  int in_real, out_real;
  int async_ok;  // input rows 16-byte aligned: stage them with cp.async
  int* err;      // device error word (bounded waits), or null
  int cfg;       // four-step passes: candidate tile shape (0: the measured default)
  // contiguous passes over several fields in one launch: rows [f*rows_per_field,
  // (f+1)*rows_per_field) are written to outs[f] (nout > 1), else to out
  int nout;
  long long rows_per_field;
  void* outs[4];
  const C* tw;   // twiddles exp(-2 pi i q/n), q in [0, n)
  // fused pass only
  int nfields;
  int d;
  int Nh;      // N = n/2 of the fused axis (axis 0)
  int nn[3];   // transform length 2 N_j of every axis (the grid may differ per axis)
  int Nhs[3];  // N_j
  FieldDesc fields[4];
};

template <typename Real, typename C, bool COHERENT>
__device__ __forceinline__ C ld_in(const PassArgs<Real>& a, long long idx) {
  if (COHERENT) {
    if (a.in_real) return C{__ldcg(reinterpret_cast<const Real*>(a.in) + idx), (Real)0};
    return __ldcg(reinterpret_cast<const C*>(a.in) + idx);
  }
  if (a.in_real) return C{__ldg(reinterpret_cast<const Real*>(a.in) + idx), (Real)0};
  return __ldg(reinterpret_cast<const C*>(a.in) + idx);
}
template <typename Real, typename C>
__device__ __forceinline__ void st_out(const PassArgs<Real>& a, void* out, long long idx, C v) {
  if (a.out_real)
    reinterpret_cast<Real*>(out)[idx] = v.x;
  else
    reinterpret_cast<C*>(out)[idx] = v;
}

// ---------------------------------------------------------------------------
// cp.async (16-byte global -> shared copies, L2 only)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// one stage's butterflies on the registers of one thread
// ---------------------------------------------------------------------------
template <typename C, int n, int E, bool INV, int S>
__device__ __forceinline__ void stage_compute(C (&v)[E], int t, const C* __restrict__ tw) {
  constexpr int R = stage_radix(n, E, INV, S);
  constexpr int Ns = stage_ns(n, E, INV, S);
  constexpr int Tp = n / E;
#pragma unroll
  for (int q = 0; q < E / R; ++q) {
    const int j = t + q * Tp;
    if (Ns > 1) {
      const int k = j % Ns;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = __ldg(tw + k * r * (n / (Ns * R)));
        v[q * R + r] = INV ? cconjmul(v[q * R + r], w) : cmul(v[q * R + r], w);
      }
    }
    Dft<R, INV>::run(&v[q * R]);
  }
}

template <int n, int E, bool INV, int S> __device__ __forceinline__ int stage_out_pos(int j, int r) {
  constexpr int R = stage_radix(n, E, INV, S);
  constexpr int Ns = stage_ns(n, E, INV, S);
  return (j / Ns) * Ns * R + (j % Ns) + r * Ns;
}
template <int n, int E, bool INV, int S> __device__ __forceinline__ int stage_in_pos(int j, int r) {
  constexpr int R = stage_radix(n, E, INV, S);
  return j + r * (n / R);
}

template <typename Real, int n, int W, bool CONTIG> __device__ __forceinline__ int saddr(int w, int pos) {
  if (CONTIG) return w * smem_pitch<Real>(n) + pos + (pos >> SmemLayout<Real>::SH);
  const int e = pos * W + w;
  return e + (e >> SmemLayout<Real>::SH);
}

// Exchange after stage S (compute done) into stage S+1 (loads done).
template <typename Real, typename C, int n, int E, int W, bool CONTIG, bool INV, int S>
__device__ __forceinline__ void exchange(C (&v)[E], C* sm, int w, int t) {
  constexpr int R0 = stage_radix(n, E, INV, S);
  constexpr int R1 = stage_radix(n, E, INV, S + 1);
  constexpr int Tp = n / E;
  __syncthreads();  // previous readers of sm are done
#pragma unroll
  for (int q = 0; q < E / R0; ++q)
#pragma unroll
    for (int r = 0; r < R0; ++r)
      sm[saddr<Real, n, W, CONTIG>(w, stage_out_pos<n, E, INV, S>(t + q * Tp, r))] = v[q * R0 + r];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < E / R1; ++q)
#pragma unroll
    for (int r = 0; r < R1; ++r)
      v[q * R1 + r] = sm[saddr<Real, n, W, CONTIG>(w, stage_in_pos<n, E, INV, S + 1>(t + q * Tp, r))];
}

// Runs stages [S, NS) of a transform whose stage S inputs are already loaded.
template <typename Real, typename C, int n, int E, int W, bool CONTIG, bool INV, int S, int NS> struct StageRun {
  __device__ __forceinline__ static void run(C (&v)[E], C* sm, int w, int t, const C* tw) {
    stage_compute<C, n, E, INV, S>(v, t, tw);
    if constexpr (S + 1 < NS) {
      exchange<Real, C, n, E, W, CONTIG, INV, S>(v, sm, w, t);
      StageRun<Real, C, n, E, W, CONTIG, INV, S + 1, NS>::run(v, sm, w, t, tw);
    }
  }
};

__device__ __forceinline__ int fold_freq(int m, int n) { return m <= n - m ? m : n - m; }

// Launch configuration of a pass.  E (values per thread), W (pencils per CTA),
// NSTG (staging ring depth) and MINB (CTAs per SM the registers must allow)
// default to the tuned choices; 0 selects the default.
template <typename Real, int n, bool CONTIG, int MODE, int E_ = 0, int W_ = 0, int NSTG_ = 0, int MINB_ = 0>
struct PassCfg {
  static constexpr int E = E_ > 0 ? E_ : elems_per_thread<Real>(n);
  static constexpr int Tp = n / E;
  static constexpr int W = W_ > 0 ? W_ : pencils_per_cta<Real>(n, CONTIG, E, MODE >= MODE_FUSED1 ? 72 * 1024 : 40 * 1024);
  static constexpr int threads = W * Tp;
  static constexpr int nstages = plan_nstages(n, E);
  static constexpr int NIN = stage_in_len(n, MODE);
  // rounded up to 128 bytes: the staging ring that follows takes 16-byte copies
  static constexpr size_t xchg_bytes = ((size_t)xchg_elems<Real>(n, W, CONTIG) * 2 * sizeof(Real) + 127) / 128 * 128;
  static constexpr size_t slot_bytes = (size_t)W * NIN * 2 * sizeof(Real);
  // staging ring depth: 3 slots when they fit a 96 KB budget, else 2 (fused: 2)
  static constexpr int NSTG =
      NSTG_ > 0 ? NSTG_ : ((MODE < MODE_FUSED1 && xchg_bytes + 3 * slot_bytes <= 96 * 1024) ? 3 : 2);
  static constexpr size_t smem = xchg_bytes + NSTG * slot_bytes;
  // by default at most 128 registers per thread: at least two 256-thread CTAs per SM
  static constexpr int min_blocks =
      MINB_ > 0 ? MINB_ : ((65536 / (threads * 128)) < 1 ? 1 : (65536 / (threads * 128)));
};

// Stages the input of one tile into a staging slot with 16-byte copies.
// Strided slot layout [pos][w] (rows of W pencils, as in global memory);
// contiguous slot layout [w][pos].  Real input is staged as reals.
template <typename Real, int n, bool CONTIG, int MODE, typename Cfg>
__device__ __forceinline__ void stage_tile(const PassArgs<Real>& a, long long tile, unsigned char* slot) {
  using C = typename CxT<Real>::T;
  constexpr int W = Cfg::W, NIN = Cfg::NIN, THREADS = Cfg::threads;
  const int esize = a.in_real ? (int)sizeof(Real) : (int)sizeof(C);
  const int per16 = 16 / esize;  // elements per 16-byte chunk
  const char* gin = reinterpret_cast<const char*>(a.in);
  if (CONTIG) {
    const long long row0 = tile * W;
    const int cpr = NIN / per16;  // chunks per row
    for (int c = threadIdx.x; c < W * cpr; c += THREADS) {
      const int w = c / cpr, k = c % cpr;
      if (row0 + w < a.O)
        cp_async16(slot + ((size_t)w * NIN + (size_t)k * per16) * esize,
                   gin + ((row0 + w) * a.in_pitch_o + (long long)k * per16) * esize);
    }
  } else {
    const long long o = tile / a.nblk_i;
    const int inner0 = (int)(tile % a.nblk_i) * W;
    const int cpr = W / per16;
    for (int c = threadIdx.x; c < NIN * cpr; c += THREADS) {
      const int pos = c / cpr, k = c % cpr;
      if (inner0 + k * per16 < a.I)
        cp_async16(slot + ((size_t)pos * W + (size_t)k * per16) * esize,
                   gin + (o * a.in_pitch_o + pos * a.in_pitch_pos + inner0 + (long long)k * per16) * esize);
    }
  }
}

// ---------------------------------------------------------------------------
// the pass kernel
//   MODE_FWD:    N valid inputs -> n outputs       (forward, pruned input)
//   MODE_INV:    n inputs -> N outputs             (inverse, cropped output)
//   MODE_FUSED1: N inputs -> fwd -> x multiplier -> inv -> N outputs
//   MODE_FUSEDN: the same for nfields fields sharing one forward transform
// CONTIG: pencils are contiguous rows; otherwise pencils are strided and the
// W pencils of a tile are W consecutive inner indices (coalesced).
// ---------------------------------------------------------------------------
// One tile of a pass: first-stage loads (from the staging slot when `staged`,
// else from global memory), the stages, the multiply of a fused pass and the
// stores.  COHERENT reads global input with ld.global.cg (L2) instead of the
// read-only path, for data written earlier by the same kernel.
template <typename Real, int n, bool CONTIG, int MODE, typename Cfg, bool COHERENT>
__device__ __forceinline__ void process_tile(const PassArgs<Real>& a, long long tile, typename CxT<Real>::T* sm,
                                             const unsigned char* slot, bool staged) {
  using C = typename CxT<Real>::T;
  constexpr int E = Cfg::E;
  constexpr int Tp = Cfg::Tp;
  constexpr int W = Cfg::W;
  constexpr int NS = Cfg::nstages;
  constexpr int NIN = Cfg::NIN;
  static_assert(NS > 0, "unsupported FFT length");
  constexpr bool FWD_FIRST = (MODE != MODE_INV);
  constexpr int R_first = stage_radix(n, E, !FWD_FIRST, 0);
  constexpr int R_lastinv = stage_radix(n, E, true, NS - 1);
  static_assert(!FWD_FIRST || R_first % 2 == 0, "pruned first stage needs an even radix");
  static_assert(MODE == MODE_FWD || R_lastinv % 2 == 0, "cropped last stage needs an even radix");
  const int tid = threadIdx.x;
  const int w = CONTIG ? tid / Tp : tid % W;
  const int t = CONTIG ? tid % Tp : tid / W;
  const C* tw = a.tw;

  // tile -> pencil coordinates
  long long in_base, out_base;
  bool valid;
  int inner = 0;
  void* outp = a.out;
  if (CONTIG) {
    const long long row = tile * W + w;
    valid = row < a.O;
    in_base = row * a.in_pitch_o;
    out_base = row * a.out_pitch_o;
    if (a.nout > 1) {
      const int f = valid ? (int)(row / a.rows_per_field) : 0;
      outp = a.outs[f];
      out_base = (row - f * a.rows_per_field) * a.out_pitch_o;
    }
  } else {
    const long long o = tile / a.nblk_i;
    inner = (int)(tile % a.nblk_i) * W + w;
    valid = inner < a.I;
    in_base = o * a.in_pitch_o + inner;
    out_base = o * a.out_pitch_o + inner;
  }

  C v[E];
  // ---- first stage loads: staged shared memory (or global memory) ----
  {
    constexpr int R = R_first;
#pragma unroll
    for (int q = 0; q < E / R; ++q) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int pos = stage_in_pos<n, E, !FWD_FIRST, 0>(t + q * Tp, r);
        C x = {(Real)0, (Real)0};
        if (valid && (!FWD_FIRST || r < R / 2)) {
          if (staged) {
            const int e = CONTIG ? w * NIN + pos : pos * W + w;
            if (a.in_real)
              x = C{reinterpret_cast<const Real*>(slot)[e], (Real)0};
            else
              x = reinterpret_cast<const C*>(slot)[e];
          } else {
            x = ld_in<Real, C, COHERENT>(a, in_base + (long long)pos * a.in_pitch_pos);
          }
        }
        v[q * R + r] = x;
      }
    }
  }

  if constexpr (MODE == MODE_FWD) {
    StageRun<Real, C, n, E, W, CONTIG, false, 0, NS>::run(v, sm, w, t, tw);
    constexpr int R = stage_radix(n, E, false, NS - 1);
    if (valid) {
#pragma unroll
      for (int q = 0; q < E / R; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int pos = stage_out_pos<n, E, false, NS - 1>(t + q * Tp, r);
          st_out<Real, C>(a, outp, out_base + (long long)pos * a.out_pitch_pos, v[q * R + r]);
        }
    }
  } else if constexpr (MODE == MODE_INV) {
    StageRun<Real, C, n, E, W, CONTIG, true, 0, NS>::run(v, sm, w, t, tw);
    constexpr int R = R_lastinv;
    if (valid) {
#pragma unroll
      for (int q = 0; q < E / R; ++q)
#pragma unroll
        for (int r = 0; r < R / 2; ++r) {
          const int pos = stage_out_pos<n, E, true, NS - 1>(t + q * Tp, r);
          st_out<Real, C>(a, outp, out_base + (long long)pos * a.out_pitch_pos, v[q * R + r]);
        }
    }
  } else {
    // frequencies of the other axes (fused axis = axis 0, the slowest); the
    // multiplier octant is [N_0 + 1][N_1 + 1]([N_2 + 1])
    const int n1 = a.nn[1], n2 = a.nn[2];
    int m1 = 0, m2 = 0;
    if (a.d == 3) {
      m1 = inner / n2;
      m2 = inner % n2;
    } else {
      m1 = inner;
    }
    const long long np1_1 = a.Nhs[1] + 1, np1_2 = a.Nhs[2] + 1;
    const long long oct_rest =
        (a.d == 3) ? (long long)fold_freq(m1, n1) * np1_2 + fold_freq(m2, n2) : fold_freq(m1, n1);
    const long long oct_pitch0 = (a.d == 3) ? np1_1 * np1_2 : np1_1;
    constexpr int RL = stage_radix(n, E, false, NS - 1);  // == first inverse radix
    // multiplier of field 0, issued before the forward transform to hide its latency
    C g[E];
    {
      const C* mult = reinterpret_cast<const C*>(a.fields[0].mult);
#pragma unroll
      for (int q = 0; q < E / RL; ++q)
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int m0 = stage_out_pos<n, E, false, NS - 1>(t + q * Tp, r);
          g[q * RL + r] = valid ? __ldg(mult + fold_freq(m0, n) * oct_pitch0 + oct_rest) : C{(Real)0, (Real)0};
        }
    }
    StageRun<Real, C, n, E, W, CONTIG, false, 0, NS>::run(v, sm, w, t, tw);
    const int nf = (MODE == MODE_FUSED1) ? 1 : a.nfields;
    for (int fi = 0; fi < nf; ++fi) {
      const FieldDesc fd = a.fields[fi];
      if (fi > 0) {
        const C* mult = reinterpret_cast<const C*>(fd.mult);
#pragma unroll
        for (int q = 0; q < E / RL; ++q)
#pragma unroll
          for (int r = 0; r < RL; ++r) {
            const int m0 = stage_out_pos<n, E, false, NS - 1>(t + q * Tp, r);
            g[q * RL + r] = valid ? __ldg(mult + fold_freq(m0, n) * oct_pitch0 + oct_rest) : C{(Real)0, (Real)0};
          }
      }
      C y[(MODE == MODE_FUSED1) ? 1 : E];
      C* yy = (MODE == MODE_FUSED1) ? v : y;
#pragma unroll
      for (int q = 0; q < E / RL; ++q)
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int m0 = stage_out_pos<n, E, false, NS - 1>(t + q * Tp, r);
          C gg = g[q * RL + r];
          if (fd.odd_axis >= 0) {
            const int mj = fd.odd_axis == 0 ? m0 : (fd.odd_axis == 1 ? m1 : m2);
            const int Nj = fd.odd_axis == 0 ? a.Nhs[0] : (fd.odd_axis == 1 ? a.Nhs[1] : a.Nhs[2]);
            if (mj > Nj) gg = C{-gg.x, -gg.y};
          }
          if (fd.spectral_axis >= 0) {
            const int j = fd.spectral_axis;
            const int mj = j == 0 ? m0 : (j == 1 ? m1 : m2);
            const int Nj = j == 0 ? a.Nhs[0] : (j == 1 ? a.Nhs[1] : a.Nhs[2]);
            const int nj = j == 0 ? a.nn[0] : (j == 1 ? a.nn[1] : a.nn[2]);
            const int ms = mj < Nj ? mj : (mj == Nj ? 0 : mj - nj);
            const Real f = (Real)3.14159265358979323846 * (Real)ms;
            gg = C{-gg.y * f, gg.x * f};  // i pi m_j * g
          }
          yy[q * RL + r] = cmul(v[q * RL + r], gg);
        }
      if constexpr (MODE == MODE_FUSED1) {
        StageRun<Real, C, n, E, W, CONTIG, true, 0, NS>::run(v, sm, w, t, tw);
      } else {
        StageRun<Real, C, n, E, W, CONTIG, true, 0, NS>::run(y, sm, w, t, tw);
      }
      constexpr int R = R_lastinv;
      if (valid) {
        const long long ob = out_base + (long long)fi * a.out_field_stride;
#pragma unroll
        for (int q = 0; q < E / R; ++q)
#pragma unroll
          for (int r = 0; r < R / 2; ++r) {
            const int pos = stage_out_pos<n, E, true, NS - 1>(t + q * Tp, r);
            st_out<Real, C>(a, outp, ob + (long long)pos * a.out_pitch_pos, yy[q * R + r]);
          }
      }
    }
  }
}

template <typename Real, int n, bool CONTIG, int MODE, typename Cfg = PassCfg<Real, n, CONTIG, MODE>>
__global__ void __launch_bounds__(Cfg::threads, Cfg::min_blocks) pencil_pass(const PassArgs<Real> a) {
  using C = typename CxT<Real>::T;
  constexpr int W = Cfg::W;
  constexpr int NSTG = Cfg::NSTG;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  unsigned char* stg = smem_raw + Cfg::xchg_bytes;

  const long long ntiles = CONTIG ? (a.O + W - 1) / W : (long long)a.O * a.nblk_i;
  // strided rows narrower than one 16-byte chunk are read directly
  constexpr bool STAGEABLE = CONTIG || ((W * 2 * sizeof(Real)) % 16 == 0);
  const bool staged = STAGEABLE && a.async_ok != 0;

  // prologue: stage the first NSTG-1 tiles of this CTA
#pragma unroll
  for (int s = 0; s < NSTG - 1; ++s) {
    const long long tl = blockIdx.x + (long long)s * gridDim.x;
    if (staged && tl < ntiles) stage_tile<Real, n, CONTIG, MODE, Cfg>(a, tl, stg + s * Cfg::slot_bytes);
    cp_async_commit();
  }

  int it = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    {
      const long long tl = tile + (long long)(NSTG - 1) * gridDim.x;
      if (staged && tl < ntiles)
        stage_tile<Real, n, CONTIG, MODE, Cfg>(a, tl, stg + ((it + NSTG - 1) % NSTG) * Cfg::slot_bytes);
      cp_async_commit();
    }
    cp_async_wait<NSTG - 1>();
    __syncthreads();
    const unsigned char* slot = stg + (it % NSTG) * Cfg::slot_bytes;

    process_tile<Real, n, CONTIG, MODE, Cfg, false>(a, tile, sm, slot, staged);
    __syncthreads();  // this tile's slot and the exchange buffer are free again
  }
  cp_async_wait<0>();
}

}  // namespace vp
