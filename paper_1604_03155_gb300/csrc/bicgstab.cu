// bicgstab.cu -- the scattering solver of Section 5.3 (Vico, Greengard &
// Ferrando): unpreconditioned Bi-CGStab (van der Vorst 1992) on the
// Lippmann-Schwinger equation, two operator products per iteration, each one
// apply of the plan's volume potential V (the Green's function of
// -(Delta + k^2)).
//
// Two forms of one problem (u the scattered field, q the real contrast):
//   field:    A u = u - k^2 V[q u]   = k^2 V[q u_inc]
//   density:  B s = s - k^2 q V[s]   = k^2 q u_inc,      u = V[s]
// The density form is the paper's dual equation of Section 5.3 (s is the
// source density whose potential is the scattered field); the field form is
// the one the GMRES solver of ls.cu uses.  Both give the same u.
//
// The recurrence (Saad, Iterative Methods for Sparse Linear Systems, Alg. 7.7,
// with the early exit at the half step): x_0 = 0, r_0 = r^ = b, p_0 = r_0;
//   v = M p, alpha = <r^, r_j> / <r^, v>, s = r_j - alpha v
//   (stop with x_j + alpha p when ||s|| < tol ||b||)
//   t = M s, omega = <t, s> / <t, t>, x_{j+1} = x_j + alpha p + omega s,
//   r_{j+1} = s - omega t (stop when ||r_{j+1}|| < tol ||b||),
//   beta = (<r^, r_{j+1}> / <r^, r_j>) (alpha / omega), p = r_{j+1} + beta (p - omega v).
//
// GPU layout: every scalar of the recurrence (rho, alpha, omega, beta, the
// residual norms, the stop flag and the counters) lives in one device struct
// written by one-block scalar kernels from the per-block partial sums of the
// vector kernels, so an iteration is a fixed launch sequence (captured once as
// a CUDA graph) with no host round trip.  The host reads iteration j's state
// (copied into pinned memory at the end of the iteration) while iteration j+1
// runs; the kernels of an iteration that starts after the stop return at once
// (its two applies still run, on data that is discarded).  Inner products:
// per-thread partial sums in the vector precision, FP64 across threads and
// blocks, in a fixed order (the result does not depend on scheduling).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <chrono>
#include <string>

#include "../../include/vp.h"
#include "vp_internal.cuh"

namespace {

constexpr int kBlocks = 304;  // 2 x 152 SMs
constexpr int kThreads = 512;
constexpr int kScalThreads = 256;

enum { BCG_RUNNING = 0, BCG_CONVERGED = 1, BCG_CONVERGED_HALF = 2, BCG_BREAKDOWN = 3, BCG_NONFINITE = 4 };

struct BcgState {
  double2 rho, alpha, omega, beta;
  double bnorm2, rnorm2, snorm2, tol, tol2;
  int done, first, breakdown, iterations, matvecs, pad;
};

template <typename R>
struct Cx;
template <>
struct Cx<float> {
  using T = float2;
};
template <>
struct Cx<double> {
  using T = double2;
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Sums K complex per-thread accumulators over the block (FP64 across threads)
// and writes them to part[blockIdx.x * K + k].
template <int K>
__device__ __forceinline__ void block_partials(const double (&re)[K], const double (&im)[K], double2* __restrict__ part) {
  __shared__ double2 red[K][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double a = re[k], b = im[k];
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) red[k][warp] = make_double2(a, b);
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double2 s = make_double2(0.0, 0.0);
    for (int w = 0; w < kThreads / 32; ++w) {
      s.x += red[threadIdx.x][w].x;
      s.y += red[threadIdx.x][w].y;
    }
    part[blockIdx.x * K + threadIdx.x] = s;
  }
}

// out[k] = sum over the kBlocks partials (one block of kScalThreads threads;
// every thread returns the same sums)
template <int K>
__device__ __forceinline__ void sum_partials(const double2* __restrict__ part, double2 (&out)[K]) {
  __shared__ double2 red[K][kScalThreads];
  for (int k = 0; k < K; ++k) {
    double2 s = make_double2(0.0, 0.0);
    for (int b = threadIdx.x; b < kBlocks; b += kScalThreads) {
      s.x += part[b * K + k].x;
      s.y += part[b * K + k].y;
    }
    red[k][threadIdx.x] = s;
  }
  __syncthreads();
  for (int o = kScalThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < K; ++k) {
        red[k][threadIdx.x].x += red[k][threadIdx.x + o].x;
        red[k][threadIdx.x].y += red[k][threadIdx.x + o].y;
      }
    __syncthreads();
  }
  for (int k = 0; k < K; ++k) out[k] = red[k][0];
}

#define GRID_LOOP(i, n) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// ---------------------------------------------------------------------------
// vector kernels (kBlocks x kThreads); all return at once after the stop
// ---------------------------------------------------------------------------

// t0 = q u (the field form's operand of V)
template <typename R>
__global__ void __launch_bounds__(kThreads) k_qmul(typename Cx<R>::T* __restrict__ out, const R* __restrict__ q,
                                                   const typename Cx<R>::T* __restrict__ in, long long n) {
  GRID_LOOP(i, n) {
    const R qi = q[i];
    out[i] = {qi * in[i].x, qi * in[i].y};
  }
}

// b = k^2 src (field: src = V[q u_inc]) or k^2 q src (density: src = u_inc);
// r = r^ = b; x = p = v = 0; partials (<r^, r>, ||r||^2) = (||b||^2, ||b||^2)
template <typename R, bool DENSITY>
__global__ void __launch_bounds__(kThreads) k_start(const typename Cx<R>::T* __restrict__ src, const R* __restrict__ q,
                                                    R k2, typename Cx<R>::T* __restrict__ b,
                                                    typename Cx<R>::T* __restrict__ r, typename Cx<R>::T* __restrict__ rh,
                                                    typename Cx<R>::T* __restrict__ x, typename Cx<R>::T* __restrict__ p,
                                                    typename Cx<R>::T* __restrict__ v, long long n,
                                                    double2* __restrict__ part) {
  using C = typename Cx<R>::T;
  R acc = 0;
  GRID_LOOP(i, n) {
    const R f = DENSITY ? k2 * q[i] : k2;
    const C bi = {f * src[i].x, f * src[i].y};
    b[i] = bi;
    r[i] = bi;
    rh[i] = bi;
    x[i] = {0, 0};
    p[i] = {0, 0};
    v[i] = {0, 0};
    acc += bi.x * bi.x + bi.y * bi.y;
  }
  const double re[2] = {(double)acc, (double)acc}, im[2] = {0.0, 0.0};
  block_partials<2>(re, im, part);
}

// b = k^2 src (field) or k^2 q src (density)
template <typename R, bool DENSITY>
__global__ void __launch_bounds__(kThreads) k_rhs(const typename Cx<R>::T* __restrict__ src, const R* __restrict__ q,
                                                  R k2, typename Cx<R>::T* __restrict__ b, long long n) {
  GRID_LOOP(i, n) {
    const R f = DENSITY ? k2 * q[i] : k2;
    b[i] = {f * src[i].x, f * src[i].y};
  }
}

// p = r + beta (p - omega v); t0 = q p (field form)
template <typename R, bool DENSITY>
__global__ void __launch_bounds__(kThreads) k_p(const BcgState* __restrict__ st, typename Cx<R>::T* __restrict__ p,
                                                const typename Cx<R>::T* __restrict__ r,
                                                const typename Cx<R>::T* __restrict__ v, const R* __restrict__ q,
                                                typename Cx<R>::T* __restrict__ t0, long long n) {
  using C = typename Cx<R>::T;
  if (st->done) return;
  const R br = (R)st->beta.x, bi = (R)st->beta.y, wr = (R)st->omega.x, wi = (R)st->omega.y;
  GRID_LOOP(i, n) {
    const C pv = p[i], vv = v[i], rv = r[i];
    const R dx = pv.x - (wr * vv.x - wi * vv.y), dy = pv.y - (wr * vv.y + wi * vv.x);
    const C np = {rv.x + br * dx - bi * dy, rv.y + br * dy + bi * dx};
    p[i] = np;
    if (!DENSITY) {
      const R qi = q[i];
      t0[i] = {qi * np.x, qi * np.y};
    }
  }
}

// v = p - k^2 t1 (field) or p - k^2 q t1 (density); partial <r^, v>
template <typename R, bool DENSITY>
__global__ void __launch_bounds__(kThreads) k_v(const BcgState* __restrict__ st, typename Cx<R>::T* __restrict__ v,
                                                const typename Cx<R>::T* __restrict__ p,
                                                const typename Cx<R>::T* __restrict__ t1, const R* __restrict__ q,
                                                const typename Cx<R>::T* __restrict__ rh, R k2, long long n,
                                                double2* __restrict__ part) {
  using C = typename Cx<R>::T;
  if (st->done) return;
  R ar = 0, ai = 0;
  GRID_LOOP(i, n) {
    const R f = DENSITY ? k2 * q[i] : k2;
    const C tv = t1[i], pv = p[i], h = rh[i];
    const C vv = {pv.x - f * tv.x, pv.y - f * tv.y};
    v[i] = vv;
    ar += h.x * vv.x + h.y * vv.y;
    ai += h.x * vv.y - h.y * vv.x;
  }
  const double re[1] = {(double)ar}, im[1] = {(double)ai};
  block_partials<1>(re, im, part);
}

// s = r - alpha v (written over r); x += alpha p; t0 = q s (field form); partial ||s||^2
template <typename R, bool DENSITY>
__global__ void __launch_bounds__(kThreads) k_s(const BcgState* __restrict__ st, typename Cx<R>::T* __restrict__ r,
                                                const typename Cx<R>::T* __restrict__ v,
                                                typename Cx<R>::T* __restrict__ x,
                                                const typename Cx<R>::T* __restrict__ p, const R* __restrict__ q,
                                                typename Cx<R>::T* __restrict__ t0, long long n,
                                                double2* __restrict__ part) {
  using C = typename Cx<R>::T;
  if (st->done) return;
  const R ar = (R)st->alpha.x, ai = (R)st->alpha.y;
  R acc = 0;
  GRID_LOOP(i, n) {
    const C rv = r[i], vv = v[i], pv = p[i], xv = x[i];
    const C s = {rv.x - (ar * vv.x - ai * vv.y), rv.y - (ar * vv.y + ai * vv.x)};
    r[i] = s;
    x[i] = {xv.x + ar * pv.x - ai * pv.y, xv.y + ar * pv.y + ai * pv.x};
    if (!DENSITY) {
      const R qi = q[i];
      t0[i] = {qi * s.x, qi * s.y};
    }
    acc += s.x * s.x + s.y * s.y;
  }
  const double re[1] = {(double)acc}, im[1] = {0.0};
  block_partials<1>(re, im, part);
}

// t = s - k^2 t1 (field) or s - k^2 q t1 (density), written over t1;
// partials <t, s>, <t, t>
template <typename R, bool DENSITY>
__global__ void __launch_bounds__(kThreads) k_t(const BcgState* __restrict__ st, typename Cx<R>::T* __restrict__ t1,
                                                const typename Cx<R>::T* __restrict__ s, const R* __restrict__ q, R k2,
                                                long long n, double2* __restrict__ part) {
  using C = typename Cx<R>::T;
  if (st->done) return;
  R tsr = 0, tsi = 0, tt = 0;
  GRID_LOOP(i, n) {
    const R f = DENSITY ? k2 * q[i] : k2;
    const C tv = t1[i], sv = s[i];
    const C t = {sv.x - f * tv.x, sv.y - f * tv.y};
    t1[i] = t;
    tsr += t.x * sv.x + t.y * sv.y;
    tsi += t.x * sv.y - t.y * sv.x;
    tt += t.x * t.x + t.y * t.y;
  }
  const double re[2] = {(double)tsr, (double)tt}, im[2] = {(double)tsi, 0.0};
  block_partials<2>(re, im, part);
}

// x += omega s; r = s - omega t (s held in r); partials <r^, r>, ||r||^2
template <typename R>
__global__ void __launch_bounds__(kThreads) k_xr(const BcgState* __restrict__ st, typename Cx<R>::T* __restrict__ x,
                                                 typename Cx<R>::T* __restrict__ r,
                                                 const typename Cx<R>::T* __restrict__ t,
                                                 const typename Cx<R>::T* __restrict__ rh, long long n,
                                                 double2* __restrict__ part) {
  using C = typename Cx<R>::T;
  if (st->done) return;
  const R wr = (R)st->omega.x, wi = (R)st->omega.y;
  R hr = 0, hi = 0, nn = 0;
  GRID_LOOP(i, n) {
    const C sv = r[i], tv = t[i], xv = x[i], h = rh[i];
    x[i] = {xv.x + wr * sv.x - wi * sv.y, xv.y + wr * sv.y + wi * sv.x};
    const C rn = {sv.x - (wr * tv.x - wi * tv.y), sv.y - (wr * tv.y + wi * tv.x)};
    r[i] = rn;
    hr += h.x * rn.x + h.y * rn.y;
    hi += h.x * rn.y - h.y * rn.x;
    nn += rn.x * rn.x + rn.y * rn.y;
  }
  const double re[2] = {(double)hr, (double)nn}, im[2] = {(double)hi, 0.0};
  block_partials<2>(re, im, part);
}

// partials of ||b - M x||^2 and ||b||^2 from t1 = V[q x] (field) or V[x] (density)
template <typename R, bool DENSITY>
__global__ void __launch_bounds__(kThreads) k_resid(const typename Cx<R>::T* __restrict__ b,
                                                    const typename Cx<R>::T* __restrict__ x,
                                                    const typename Cx<R>::T* __restrict__ t1, const R* __restrict__ q,
                                                    R k2, long long n, double2* __restrict__ part) {
  using C = typename Cx<R>::T;
  double rr = 0.0, bb = 0.0;
  GRID_LOOP(i, n) {
    const R f = DENSITY ? k2 * q[i] : k2;
    const C bv = b[i], xv = x[i], tv = t1[i];
    const double ex = (double)bv.x - ((double)xv.x - (double)f * tv.x);
    const double ey = (double)bv.y - ((double)xv.y - (double)f * tv.y);
    rr += ex * ex + ey * ey;
    bb += (double)bv.x * bv.x + (double)bv.y * bv.y;
  }
  const double re[2] = {rr, bb}, im[2] = {0.0, 0.0};
  block_partials<2>(re, im, part);
}

// float -> double conversions for the FP64 true residual of an FP32 solve
__global__ void k_widen_c(double2* __restrict__ out, const float2* __restrict__ in, long long n) {
  GRID_LOOP(i, n) out[i] = make_double2(in[i].x, in[i].y);
}
__global__ void k_widen_r(double* __restrict__ out, const float* __restrict__ in, long long n) {
  GRID_LOOP(i, n) out[i] = in[i];
}

// ---------------------------------------------------------------------------
// scalar kernels (one block of kScalThreads)
// ---------------------------------------------------------------------------

// after k_start / k_xr: rho_{j+1} = <r^, r>, ||r||^2; stop test; beta
__global__ void __launch_bounds__(kScalThreads) k_scal_rho(BcgState* __restrict__ st, const double2* __restrict__ part) {
  if (st->done) return;
  double2 s[2];
  sum_partials<2>(part, s);
  if (threadIdx.x != 0) return;
  const double2 rho_new = s[0];
  const double rn2 = s[1].x;
  st->rnorm2 = rn2;
  if (st->first) {
    st->first = 0;
    st->bnorm2 = rn2;
    st->tol2 = st->tol * st->tol * rn2;
    if (!(rn2 > 0.0)) {  // b = 0: u = 0
      st->done = isfinite(rn2) ? BCG_CONVERGED : BCG_NONFINITE;
      return;
    }
  } else if (!isfinite(rn2) || !finite2(rho_new)) {
    st->done = BCG_NONFINITE;
    return;
  } else if (rn2 < st->tol2) {
    st->done = BCG_CONVERGED;
    return;
  } else if (st->breakdown) {
    st->done = BCG_BREAKDOWN;
    return;
  }
  if (rho_new.x == 0.0 && rho_new.y == 0.0) {
    st->done = BCG_BREAKDOWN;
    return;
  }
  st->beta = cmul(cdiv(rho_new, st->rho), cdiv(st->alpha, st->omega));
  st->rho = rho_new;
}

// after k_v: alpha = rho / <r^, v>
__global__ void __launch_bounds__(kScalThreads) k_scal_alpha(BcgState* __restrict__ st, const double2* __restrict__ part) {
  if (st->done) return;
  double2 s[1];
  sum_partials<1>(part, s);
  if (threadIdx.x != 0) return;
  ++st->iterations;
  ++st->matvecs;
  if (!finite2(s[0])) {
    st->done = BCG_NONFINITE;
  } else if (s[0].x == 0.0 && s[0].y == 0.0) {
    st->done = BCG_BREAKDOWN;
  } else {
    st->alpha = cdiv(st->rho, s[0]);
  }
}

// after k_s: ||s||^2 and the half-step stop test
__global__ void __launch_bounds__(kScalThreads) k_scal_s(BcgState* __restrict__ st, const double2* __restrict__ part) {
  if (st->done) return;
  double2 s[1];
  sum_partials<1>(part, s);
  if (threadIdx.x != 0) return;
  st->snorm2 = s[0].x;
  if (!isfinite(s[0].x))
    st->done = BCG_NONFINITE;
  else if (s[0].x < st->tol2)
    st->done = BCG_CONVERGED_HALF;
}

// after k_t: omega = <t, s> / <t, t> (0 with a breakdown flag when t = 0)
__global__ void __launch_bounds__(kScalThreads) k_scal_omega(BcgState* __restrict__ st, const double2* __restrict__ part) {
  if (st->done) return;
  double2 s[2];
  sum_partials<2>(part, s);
  if (threadIdx.x != 0) return;
  ++st->matvecs;
  if (!finite2(s[0]) || !isfinite(s[1].x)) {
    st->done = BCG_NONFINITE;
  } else if (s[1].x == 0.0 || (s[0].x == 0.0 && s[0].y == 0.0)) {
    st->omega = make_double2(0.0, 0.0);
    st->breakdown = 1;
  } else {
    st->omega = make_double2(s[0].x / s[1].x, s[0].y / s[1].x);
  }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------

struct Err {
  vp_status st = VP_OK;
  std::string msg;
};

#define BCG_CUDA(E, call)                                          \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      (E).st = e_ == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA; \
      (E).msg = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return (E).st;                                               \
    }                                                              \
  } while (0)

template <typename R>
struct Work {
  using C = typename Cx<R>::T;
  long long n = 0;
  C *b = nullptr, *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *t0 = nullptr, *t1 = nullptr;
  C* x = nullptr;        // the iterate: x_own (density form) or the caller's u (field form)
  C* x_own = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  double2* part = nullptr;
  BcgState* st = nullptr;
  BcgState* host = nullptr;  // pinned: slots 0 and 1 (per-iteration copies), 2 (start and final)
  cudaStream_t s = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaGraph_t g[2] = {nullptr, nullptr};
  cudaGraphExec_t gx[2] = {nullptr, nullptr};
  ~Work() {
    if (s) cudaStreamSynchronize(s);
    for (int i = 0; i < 2; ++i) {
      if (gx[i]) cudaGraphExecDestroy(gx[i]);
      if (g[i]) cudaGraphDestroy(g[i]);
      if (ev[i]) cudaEventDestroy(ev[i]);
    }
    cudaFree(b);
    cudaFree(r);
    cudaFree(rh);
    cudaFree(p);
    cudaFree(v);
    cudaFree(t0);
    cudaFree(t1);
    cudaFree(x_own);
    cudaFree(ws);
    cudaFree(part);
    cudaFree(st);
    cudaFreeHost(host);
    if (s) cudaStreamDestroy(s);
  }
};

// restores the plan's stream and precision on every exit path
struct PlanGuard {
  vp_plan plan;
  cudaStream_t stream;
  vp_precision prec;
  bool restore_prec = false;
  ~PlanGuard() {
    vp_plan_set_stream(plan, stream);
    if (restore_prec) vp_plan_set_precision(plan, prec);
  }
};

template <typename R>
vp_dtype cdtype() {
  return sizeof(R) == 8 ? VP_C128 : VP_C64;
}

// one operator product's apply of V: field form V[t0], density form V[in]
template <typename R, bool DENSITY>
vp_status apply_v(vp_plan plan, Work<R>& w, const typename Cx<R>::T* in) {
  return vp::apply_with_workspace(plan, DENSITY ? (const void*)in : (const void*)w.t0, w.t1, cdtype<R>(), w.ws,
                                  w.ws_bytes);
}

// one iteration on w.s, its state copied to host slot `slot`
template <typename R, bool DENSITY>
vp_status enqueue_iteration(vp_plan plan, Work<R>& w, const R* q, R k2, int slot) {
  const long long n = w.n;
  k_p<R, DENSITY><<<kBlocks, kThreads, 0, w.s>>>(w.st, w.p, w.r, w.v, q, w.t0, n);
  vp_status st = apply_v<R, DENSITY>(plan, w, w.p);
  if (st != VP_OK) return st;
  k_v<R, DENSITY><<<kBlocks, kThreads, 0, w.s>>>(w.st, w.v, w.p, w.t1, q, w.rh, k2, n, w.part);
  k_scal_alpha<<<1, kScalThreads, 0, w.s>>>(w.st, w.part);
  k_s<R, DENSITY><<<kBlocks, kThreads, 0, w.s>>>(w.st, w.r, w.v, w.x, w.p, q, w.t0, n, w.part);
  k_scal_s<<<1, kScalThreads, 0, w.s>>>(w.st, w.part);
  if ((st = apply_v<R, DENSITY>(plan, w, w.r)) != VP_OK) return st;
  k_t<R, DENSITY><<<kBlocks, kThreads, 0, w.s>>>(w.st, w.t1, w.r, q, k2, n, w.part);
  k_scal_omega<<<1, kScalThreads, 0, w.s>>>(w.st, w.part);
  k_xr<R><<<kBlocks, kThreads, 0, w.s>>>(w.st, w.x, w.r, w.t1, w.rh, n, w.part);
  k_scal_rho<<<1, kScalThreads, 0, w.s>>>(w.st, w.part);
  if (cudaMemcpyAsync(w.host + slot, w.st, sizeof(BcgState), cudaMemcpyDeviceToHost, w.s) != cudaSuccess)
    return VP_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ERR_CUDA;
}

// ||b - M x|| / ||b|| with the operator of this precision (w.t0/w.t1 as scratch)
template <typename R, bool DENSITY>
vp_status residual(vp_plan plan, Work<R>& w, const typename Cx<R>::T* b, const typename Cx<R>::T* x, const R* q,
                   R k2, double* out, Err& E) {
  const long long n = w.n;
  if (!DENSITY) k_qmul<R><<<kBlocks, kThreads, 0, w.s>>>(w.t0, q, x, n);
  vp_status st = apply_v<R, DENSITY>(plan, w, x);
  if (st != VP_OK) return st;
  k_resid<R, DENSITY><<<kBlocks, kThreads, 0, w.s>>>(b, x, w.t1, q, k2, n, w.part);
  double2 h[2 * kBlocks];
  BCG_CUDA(E, cudaMemcpyAsync(h, w.part, sizeof(h), cudaMemcpyDeviceToHost, w.s));
  BCG_CUDA(E, cudaStreamSynchronize(w.s));
  double rr = 0.0, bb = 0.0;
  for (int i = 0; i < kBlocks; ++i) {
    rr += h[2 * i].x;
    bb += h[2 * i + 1].x;
  }
  *out = bb > 0 ? sqrt(rr / bb) : sqrt(rr);
  return VP_OK;
}

template <typename R>
vp_status alloc_work(Work<R>& w, vp_plan plan, long long n, bool density, Err& E) {
  using C = typename Cx<R>::T;
  w.n = n;
  BCG_CUDA(E, cudaStreamCreateWithFlags(&w.s, cudaStreamNonBlocking));
  for (int i = 0; i < 2; ++i) BCG_CUDA(E, cudaEventCreateWithFlags(&w.ev[i], cudaEventDisableTiming));
  C** vecs[] = {&w.b, &w.r, &w.rh, &w.p, &w.v, &w.t1};
  for (C** pp : vecs) BCG_CUDA(E, cudaMalloc(pp, n * sizeof(C)));
  if (!density) BCG_CUDA(E, cudaMalloc(&w.t0, n * sizeof(C)));
  if (density) {
    BCG_CUDA(E, cudaMalloc(&w.x_own, n * sizeof(C)));
    w.x = w.x_own;
  }
  w.ws_bytes = vp::plan_apply_workspace_bytes(plan);
  BCG_CUDA(E, cudaMalloc(&w.ws, w.ws_bytes));
  BCG_CUDA(E, cudaMalloc(&w.part, 2 * kBlocks * sizeof(double2)));
  BCG_CUDA(E, cudaMalloc(&w.st, sizeof(BcgState)));
  BCG_CUDA(E, cudaMallocHost(&w.host, 3 * sizeof(BcgState)));
  return VP_OK;
}

template <typename R, bool DENSITY>
vp_status solve(vp_plan plan, const R* q, const typename Cx<R>::T* uinc, typename Cx<R>::T* u, double k2d,
                long long n, double tol, int maxit, double* history, vp_ls_stats* stats, Err& E) {
  using C = typename Cx<R>::T;
  const auto t_start = std::chrono::steady_clock::now();
  Work<R> w;
  vp_status st = alloc_work<R>(w, plan, n, DENSITY, E);
  if (st != VP_OK) return st;
  if (!DENSITY) w.x = u;  // the field form iterates on u itself
  const R k2 = (R)k2d;
  PlanGuard guard{plan, vp::plan_stream(plan), VP_FP32};
  BCG_CUDA(E, cudaStreamSynchronize(guard.stream));  // inputs produced on the plan's stream
  if ((st = vp_plan_set_stream(plan, w.s)) != VP_OK) return st;

  // right-hand side (an uncaptured apply also sets up every pass kernel before capture)
  if (!DENSITY) {
    k_qmul<R><<<kBlocks, kThreads, 0, w.s>>>(w.t0, q, uinc, n);
    if ((st = apply_v<R, false>(plan, w, uinc)) != VP_OK) return st;
    k_start<R, false><<<kBlocks, kThreads, 0, w.s>>>(w.t1, q, k2, w.b, w.r, w.rh, w.x, w.p, w.v, n, w.part);
  } else {
    if ((st = apply_v<R, true>(plan, w, uinc)) != VP_OK) return st;
    k_start<R, true><<<kBlocks, kThreads, 0, w.s>>>(uinc, q, k2, w.b, w.r, w.rh, w.x, w.p, w.v, n, w.part);
  }
  BcgState init;
  memset(&init, 0, sizeof(init));
  init.rho = init.alpha = init.omega = make_double2(1.0, 0.0);
  init.tol = tol;
  init.first = 1;
  w.host[2] = init;
  BCG_CUDA(E, cudaMemcpyAsync(w.st, w.host + 2, sizeof(BcgState), cudaMemcpyHostToDevice, w.s));
  k_scal_rho<<<1, kScalThreads, 0, w.s>>>(w.st, w.part);
  BCG_CUDA(E, cudaGetLastError());
  BCG_CUDA(E, cudaMemcpyAsync(w.host + 2, w.st, sizeof(BcgState), cudaMemcpyDeviceToHost, w.s));
  BCG_CUDA(E, cudaStreamSynchronize(w.s));
  if (history) history[0] = 1.0;
  BcgState last = w.host[2];

  if (!last.done) {
    // the iteration as two graphs (state copied to host slot 0 or 1)
    for (int k = 0; k < 2; ++k) {
      BCG_CUDA(E, cudaStreamBeginCapture(w.s, cudaStreamCaptureModeThreadLocal));
      vp_status cs = enqueue_iteration<R, DENSITY>(plan, w, q, k2, k);
      cudaError_t ce = cudaStreamEndCapture(w.s, &w.g[k]);
      if (cs != VP_OK) return cs;
      BCG_CUDA(E, ce);
      BCG_CUDA(E, cudaGraphInstantiate(&w.gx[k], w.g[k], 0));
    }
    // iteration j runs while the host reads iteration j-1's state
    for (int j = 1; j <= maxit + 1; ++j) {
      if (j <= maxit) {
        BCG_CUDA(E, cudaGraphLaunch(w.gx[j & 1], w.s));
        BCG_CUDA(E, cudaEventRecord(w.ev[j & 1], w.s));
      }
      if (j >= 2) {
        BCG_CUDA(E, cudaEventSynchronize(w.ev[(j - 1) & 1]));
        last = w.host[(j - 1) & 1];
        if (history && last.bnorm2 > 0)
          history[j - 1] = sqrt((last.done == BCG_CONVERGED_HALF ? last.snorm2 : last.rnorm2) / last.bnorm2);
        if (last.done) break;
      }
    }
    BCG_CUDA(E, cudaStreamSynchronize(w.s));
  }
  if (DENSITY) {  // u = V[s]
    BCG_CUDA(E, cudaGetLastError());
    st = vp::apply_with_workspace(plan, w.x, u, cdtype<R>(), w.ws, w.ws_bytes);
    if (st != VP_OK) return st;
  }
  BCG_CUDA(E, cudaStreamSynchronize(w.s));
  const auto t_end = std::chrono::steady_clock::now();

  // true residual ||b - M x|| / ||b||, the operator and b evaluated in FP64
  double tr = 0.0;
  if constexpr (sizeof(R) == 8) {
    st = residual<R, DENSITY>(plan, w, w.b, w.x, q, k2, &tr, E);
    if (st != VP_OK) return st;
  } else {
    Work<double> w64;
    if ((st = alloc_work<double>(w64, plan, n, DENSITY, E)) != VP_OK) return st;
    guard.restore_prec = true;
    if ((st = vp_plan_set_precision(plan, VP_FP64)) != VP_OK) return st;
    cudaFree(w64.ws);  // resize for the FP64 passes
    w64.ws = nullptr;
    w64.ws_bytes = vp::plan_apply_workspace_bytes(plan);
    BCG_CUDA(E, cudaMalloc(&w64.ws, w64.ws_bytes));
    BCG_CUDA(E, cudaStreamSynchronize(w.s));
    if ((st = vp_plan_set_stream(plan, w64.s)) != VP_OK) return st;
    double* q64 = reinterpret_cast<double*>(w64.rh);  // n doubles fit in n complex
    k_widen_r<<<kBlocks, kThreads, 0, w64.s>>>(q64, reinterpret_cast<const float*>(q), n);
    k_widen_c<<<kBlocks, kThreads, 0, w64.s>>>(w64.p, reinterpret_cast<const float2*>(uinc), n);
    if (!DENSITY) {  // b = k^2 V[q u_inc] in FP64
      k_qmul<double><<<kBlocks, kThreads, 0, w64.s>>>(w64.t0, q64, w64.p, n);
      if ((st = apply_v<double, false>(plan, w64, w64.p)) != VP_OK) return st;
      k_rhs<double, false><<<kBlocks, kThreads, 0, w64.s>>>(w64.t1, q64, k2d, w64.b, n);
    } else {  // b = k^2 q u_inc
      k_rhs<double, true><<<kBlocks, kThreads, 0, w64.s>>>(w64.p, q64, k2d, w64.b, n);
    }
    double2* x64 = w64.r;
    k_widen_c<<<kBlocks, kThreads, 0, w64.s>>>(x64, reinterpret_cast<const float2*>(w.x), n);
    st = residual<double, DENSITY>(plan, w64, w64.b, x64, q64, k2d, &tr, E);
    if (st != VP_OK) return st;
  }
  if (stats) {
    stats->iterations = last.iterations;
    stats->matvecs = last.matvecs;
    stats->restarts = 0;
    stats->used_fallback = 0;
    stats->estimated_residual =
        last.bnorm2 > 0 ? sqrt((last.done == BCG_CONVERGED_HALF ? last.snorm2 : last.rnorm2) / last.bnorm2) : 0.0;
    stats->true_residual = tr;
    stats->seconds = std::chrono::duration<double>(t_end - t_start).count();
  }
  if (last.done == BCG_NONFINITE) {
    E.msg = "Bi-CGStab produced a non-finite value";
    return E.st = VP_ERR_NUMERICAL;
  }
  if (last.done == BCG_BREAKDOWN) {
    E.msg = "Bi-CGStab breakdown (a zero inner product) before convergence";
    return E.st = VP_ERR_NUMERICAL;
  }
  return VP_OK;
}

}  // namespace

extern "C" {

vp_status vp_ls_bicgstab(vp_plan plan, const void* q, const void* u_inc, void* u, vp_dtype dtype, int form,
                         double tol, int maxit, double* history, vp_ls_stats* stats) {
  int d = 0, N = 0;
  double k = 0.0;
  if (!plan) {
    vp::ls_set_error("plan is NULL");
    return VP_ERR_INVALID_ARG;
  }
  vp_status st = vp_plan_info(plan, &d, &N, &k, nullptr, nullptr);
  if (st != VP_OK) return st;
  auto bad = [](const char* m) {
    vp::ls_set_error(m);
    return VP_ERR_INVALID_ARG;
  };
  if (!(k > 0)) return bad("the scattering solve needs a Helmholtz plan");
  if (!q || !u_inc || !u) return bad("q, u_inc and u are required");
  if (u == u_inc) return bad("u may not alias u_inc");
  if (form != VP_LS_FIELD && form != VP_LS_DENSITY) return bad("form must be VP_LS_FIELD or VP_LS_DENSITY");
  if (!(tol > 0) || maxit < 1) return bad("tol > 0 and maxit >= 1 required");
  if (dtype == VP_C64) {
    if (!vp::plan_is_fp32(plan)) return bad("VP_C64 iterates with the FP32 apply: set the plan's precision to VP_FP32");
  } else if (dtype == VP_C128) {
    if (!vp::plan_is_fp64(plan)) return bad("VP_C128 iterates with the FP64 apply: set the plan's precision to VP_FP64");
  } else {
    return bad("dtype must be VP_C64 or VP_C128");
  }
  const long long n = (long long)N * N * (d == 3 ? N : 1);
  Err E;
  cudaSetDevice(vp::plan_device(plan));
  const bool dens = form == VP_LS_DENSITY;
  if (dtype == VP_C64) {
    auto qq = reinterpret_cast<const float*>(q);
    auto ui = reinterpret_cast<const float2*>(u_inc);
    auto uo = reinterpret_cast<float2*>(u);
    st = dens ? solve<float, true>(plan, qq, ui, uo, k * k, n, tol, maxit, history, stats, E)
              : solve<float, false>(plan, qq, ui, uo, k * k, n, tol, maxit, history, stats, E);
  } else {
    auto qq = reinterpret_cast<const double*>(q);
    auto ui = reinterpret_cast<const double2*>(u_inc);
    auto uo = reinterpret_cast<double2*>(u);
    st = dens ? solve<double, true>(plan, qq, ui, uo, k * k, n, tol, maxit, history, stats, E)
              : solve<double, false>(plan, qq, ui, uo, k * k, n, tol, maxit, history, stats, E);
  }
  if (st != VP_OK) vp::ls_set_error(E.msg.empty() ? vp_status_string(st) : E.msg.c_str());
  return st;
}

}  // extern "C"
