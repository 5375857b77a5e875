// krylov.cu -- the integral-equation solvers of Sections 5.2 and 5.3 (Vico,
// Greengard & Ferrando): unpreconditioned Bi-CGStab (van der Vorst 1992), two
// operator products per iteration, each one apply of the plan's volume
// potential V (or of its exact gradient); and restarted GMRES, the paper's
// solver for the Section 5.2 equation (at the end of the file).
//
// Lippmann-Schwinger scattering (Section 5.3; V the Green's function of
// -(Delta + k^2)), two forms of one problem (u the scattered field, q the real
// contrast):
//   field:    A u = u - k^2 V[q u]   = k^2 V[q u_inc]
//   density:  B s = s - k^2 q V[s]   = k^2 q u_inc,      u = V[s]
// The density form is the paper's dual equation of Section 5.3 (s is the
// source density whose potential is the scattered field); the field form is
// the one the GMRES solver of ls.cu uses.  Both give the same u.
// Variable-coefficient Poisson (Section 5.2, eq. pbeq; V the Laplace potential):
//   P s = -eps s + grad(eps) . grad V[s] = rho,            phi = V[s]
// Mixed precision (FP32 products, FP64 reliable updates) is described further
// down, before solve_mixed.
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

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>
#include <string>

#include "../../include/vp.h"
#include "vp_internal.cuh"

namespace {

constexpr int kBlocks = 304;  // 2 x 152 SMs
constexpr int kThreads = 512;
constexpr int kScalThreads = 256;
// mixed precision: consecutive reliable updates that each reduce the true
// residual by less than 2x before the solve falls back to FP64
constexpr int kMaxStall = 3;

enum { BCG_RUNNING = 0, BCG_CONVERGED = 1, BCG_CONVERGED_HALF = 2, BCG_BREAKDOWN = 3, BCG_NONFINITE = 4 };

struct BcgState {
  double2 rho, alpha, omega, beta;
  double bnorm2, rnorm2, snorm2, tol, tol2;
  // reliable updates (mixed precision): the update threshold delta^2 and the
  // largest ||r||^2 since the last update
  double delta2, maxrr2;
  double best2;  // smallest true ||r||^2 at an update
  int done, first, breakdown, iterations, matvecs;
  int mixed, update, epoch, updates, stall;  // stall: consecutive updates gaining less than 2x
};

// the vector and scalar kernels of an iteration do nothing after the stop or
// while a reliable update is pending
__device__ __forceinline__ bool idle(const BcgState* st) { return st->done || st->update; }

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

// The operator M of each form, applied at node i given t1 = the apply's
// output (V[q x] for the field form, V[x] for the density form, the d
// components of grad V[x] for the Poisson-Boltzmann form, d blocks of n):
//   field:    M x = x - k^2 V[q x]
//   density:  M x = x - k^2 q V[x]
//   pb:       M x = -eps x + grad(eps) . grad V[x]        (Section 5.2, eq. pbeq)
enum { F_FIELD = 0, F_DENSITY = 1, F_PB = 2 };

template <typename R>
struct OpArgs {
  const R* q;   // contrast q, or eps for the Poisson-Boltzmann form
  const R* ge;  // grad eps (d blocks of n), Poisson-Boltzmann form only
  R k2;
  int d;
  long long n;
};

template <typename R, int FORM>
__device__ __forceinline__ typename Cx<R>::T op_at(const typename Cx<R>::T xv, const typename Cx<R>::T* __restrict__ t1,
                                                   const OpArgs<R>& a, long long i) {
  using C = typename Cx<R>::T;
  if (FORM == F_PB) {
    const R e = a.q[i];
    C acc = {-e * xv.x, -e * xv.y};
    for (int j = 0; j < a.d; ++j) {
      const R g = a.ge[j * a.n + i];
      const C tj = t1[j * a.n + i];
      acc.x += g * tj.x;
      acc.y += g * tj.y;
    }
    return acc;
  }
  const R f = FORM == F_DENSITY ? a.k2 * a.q[i] : a.k2;
  const C tv = t1[i];
  return {xv.x - f * tv.x, xv.y - f * tv.y};
}

// the right-hand side: k^2 src (field, src = V[q u_inc]), k^2 q src (density,
// src = u_inc), src (Poisson-Boltzmann, src = rho)
template <typename R, int FORM>
__device__ __forceinline__ typename Cx<R>::T rhs_at(const typename Cx<R>::T sv, const OpArgs<R>& a, long long i) {
  if (FORM == F_PB) return sv;
  const R f = FORM == F_DENSITY ? a.k2 * a.q[i] : a.k2;
  return {f * sv.x, f * sv.y};
}

// b from src; r = r^ = b; x = p = v = 0; partials (<r^, r>, ||r||^2) = (||b||^2, ||b||^2)
template <typename R, int FORM>
__global__ void __launch_bounds__(kThreads) k_start(const typename Cx<R>::T* __restrict__ src, OpArgs<R> a,
                                                    typename Cx<R>::T* __restrict__ b,
                                                    typename Cx<R>::T* __restrict__ r, typename Cx<R>::T* __restrict__ rh,
                                                    typename Cx<R>::T* __restrict__ x, typename Cx<R>::T* __restrict__ p,
                                                    typename Cx<R>::T* __restrict__ v, double2* __restrict__ part) {
  using C = typename Cx<R>::T;
  R acc = 0;
  GRID_LOOP(i, a.n) {
    const C bi = rhs_at<R, FORM>(src[i], a, i);
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

// b from src only
template <typename R, int FORM>
__global__ void __launch_bounds__(kThreads) k_rhs(const typename Cx<R>::T* __restrict__ src, OpArgs<R> a,
                                                  typename Cx<R>::T* __restrict__ b) {
  GRID_LOOP(i, a.n) b[i] = rhs_at<R, FORM>(src[i], a, i);
}

// p = r + beta (p - omega v); t0 = q p (field form)
template <typename R, int FORM>
__global__ void __launch_bounds__(kThreads) k_p(const BcgState* __restrict__ st, typename Cx<R>::T* __restrict__ p,
                                                const typename Cx<R>::T* __restrict__ r,
                                                const typename Cx<R>::T* __restrict__ v, OpArgs<R> a,
                                                typename Cx<R>::T* __restrict__ t0) {
  using C = typename Cx<R>::T;
  if (idle(st)) return;
  const R br = (R)st->beta.x, bi = (R)st->beta.y, wr = (R)st->omega.x, wi = (R)st->omega.y;
  GRID_LOOP(i, a.n) {
    const C pv = p[i], vv = v[i], rv = r[i];
    const R dx = pv.x - (wr * vv.x - wi * vv.y), dy = pv.y - (wr * vv.y + wi * vv.x);
    const C np = {rv.x + br * dx - bi * dy, rv.y + br * dy + bi * dx};
    p[i] = np;
    if (FORM == F_FIELD) {
      const R qi = a.q[i];
      t0[i] = {qi * np.x, qi * np.y};
    }
  }
}

// v = M p; partial <r^, v>
template <typename R, int FORM>
__global__ void __launch_bounds__(kThreads) k_v(const BcgState* __restrict__ st, typename Cx<R>::T* __restrict__ v,
                                                const typename Cx<R>::T* __restrict__ p,
                                                const typename Cx<R>::T* __restrict__ t1, OpArgs<R> a,
                                                const typename Cx<R>::T* __restrict__ rh, double2* __restrict__ part) {
  using C = typename Cx<R>::T;
  if (idle(st)) return;
  R ar = 0, ai = 0;
  GRID_LOOP(i, a.n) {
    const C vv = op_at<R, FORM>(p[i], t1, a, i);
    const C h = rh[i];
    v[i] = vv;
    ar += h.x * vv.x + h.y * vv.y;
    ai += h.x * vv.y - h.y * vv.x;
  }
  const double re[1] = {(double)ar}, im[1] = {(double)ai};
  block_partials<1>(re, im, part);
}

// s = r - alpha v (written over r); x += alpha p; t0 = q s (field form); partial ||s||^2
template <typename R, int FORM>
__global__ void __launch_bounds__(kThreads) k_s(const BcgState* __restrict__ st, typename Cx<R>::T* __restrict__ r,
                                                const typename Cx<R>::T* __restrict__ v,
                                                typename Cx<R>::T* __restrict__ x,
                                                const typename Cx<R>::T* __restrict__ p, OpArgs<R> a,
                                                typename Cx<R>::T* __restrict__ t0, double2* __restrict__ part) {
  using C = typename Cx<R>::T;
  if (idle(st)) return;
  const R ar = (R)st->alpha.x, ai = (R)st->alpha.y;
  R acc = 0;
  GRID_LOOP(i, a.n) {
    const C rv = r[i], vv = v[i], pv = p[i], xv = x[i];
    const C s = {rv.x - (ar * vv.x - ai * vv.y), rv.y - (ar * vv.y + ai * vv.x)};
    r[i] = s;
    x[i] = {xv.x + ar * pv.x - ai * pv.y, xv.y + ar * pv.y + ai * pv.x};
    if (FORM == F_FIELD) {
      const R qi = a.q[i];
      t0[i] = {qi * s.x, qi * s.y};
    }
    acc += s.x * s.x + s.y * s.y;
  }
  const double re[1] = {(double)acc}, im[1] = {0.0};
  block_partials<1>(re, im, part);
}

// t = M s, written over the first n entries of t1; partials <t, s>, <t, t>
template <typename R, int FORM>
__global__ void __launch_bounds__(kThreads) k_t(const BcgState* __restrict__ st, typename Cx<R>::T* __restrict__ t1,
                                                const typename Cx<R>::T* __restrict__ s, OpArgs<R> a,
                                                double2* __restrict__ part) {
  using C = typename Cx<R>::T;
  if (idle(st)) return;
  R tsr = 0, tsi = 0, tt = 0;
  GRID_LOOP(i, a.n) {
    const C sv = s[i];
    const C t = op_at<R, FORM>(sv, t1, a, i);  // reads every component of t1 at i before the write
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
  if (idle(st)) return;
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

// partials of ||b - M x||^2 and ||b||^2 (t1: the apply of x's operand)
template <typename R, int FORM>
__global__ void __launch_bounds__(kThreads) k_resid(const typename Cx<R>::T* __restrict__ b,
                                                    const typename Cx<R>::T* __restrict__ x,
                                                    const typename Cx<R>::T* __restrict__ t1, OpArgs<R> a,
                                                    double2* __restrict__ part) {
  using C = typename Cx<R>::T;
  double rr = 0.0, bb = 0.0;
  GRID_LOOP(i, a.n) {
    const C bv = b[i];
    const C mx = op_at<R, FORM>(x[i], t1, a, i);
    const double ex = (double)bv.x - (double)mx.x, ey = (double)bv.y - (double)mx.y;
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
  if (idle(st)) return;
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
  } else if (st->breakdown) {
    st->done = BCG_BREAKDOWN;
    return;
  } else if (st->mixed) {
    // reliable update when the recurrence residual claims convergence or has
    // fallen by delta since the last update (rho is kept for the update's beta)
    if (rn2 < st->tol2 || rn2 < st->delta2 * st->maxrr2) {
      st->update = 1;
      return;
    }
    st->maxrr2 = fmax(st->maxrr2, rn2);
  } else if (rn2 < st->tol2) {
    st->done = BCG_CONVERGED;
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
  if (idle(st)) return;
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
  if (idle(st)) return;
  double2 s[1];
  sum_partials<1>(part, s);
  if (threadIdx.x != 0) return;
  st->snorm2 = s[0].x;
  if (!isfinite(s[0].x))
    st->done = BCG_NONFINITE;
  else if (s[0].x < st->tol2 && !st->mixed)  // mixed precision: the true residual decides
    st->done = BCG_CONVERGED_HALF;
}

// after k_t: omega = <t, s> / <t, t> (0 with a breakdown flag when t = 0)
__global__ void __launch_bounds__(kScalThreads) k_scal_omega(BcgState* __restrict__ st, const double2* __restrict__ part) {
  if (idle(st)) return;
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
// mixed precision with reliable updates (Sleijpen & van der Vorst 1996): the
// recurrence runs in FP32 on the correction x_lo; at an update the FP64 solution
// takes x_lo, the true residual b - M x is formed with the FP64 apply and
// replaces the recurrence residual, and the recurrence continues from it.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kThreads) k_narrow_r(float* __restrict__ out, const double* __restrict__ in,
                                                       long long n) {
  GRID_LOOP(i, n) out[i] = (float)in[i];
}

// r = r^ = (float) b; p = v = x_lo = 0; x = 0; partials (<r^, r>, ||b||^2 in FP64)
__global__ void __launch_bounds__(kThreads) k_mixed_init(const double2* __restrict__ b, float2* __restrict__ r,
                                                         float2* __restrict__ rh, float2* __restrict__ p,
                                                         float2* __restrict__ v, float2* __restrict__ xlo,
                                                         double2* __restrict__ x, long long n,
                                                         double2* __restrict__ part) {
  float acc = 0.f;
  double bb = 0.0;
  GRID_LOOP(i, n) {
    const double2 bv = b[i];
    const float2 rv = make_float2((float)bv.x, (float)bv.y);
    r[i] = rv;
    rh[i] = rv;
    p[i] = make_float2(0.f, 0.f);
    v[i] = make_float2(0.f, 0.f);
    xlo[i] = make_float2(0.f, 0.f);
    x[i] = make_double2(0.0, 0.0);
    acc += rv.x * rv.x + rv.y * rv.y;
    bb += bv.x * bv.x + bv.y * bv.y;
  }
  const double re[2] = {(double)acc, bb}, im[2] = {0.0, 0.0};
  block_partials<2>(re, im, part);
}

// x += x_lo, x_lo = 0; t0 = q x for the field form's FP64 product
template <int FORM>
__global__ void __launch_bounds__(kThreads) k_accumulate(double2* __restrict__ x, float2* __restrict__ xlo,
                                                         const double* __restrict__ q, double2* __restrict__ t0,
                                                         long long n) {
  GRID_LOOP(i, n) {
    const float2 d = xlo[i];
    const double2 xv = make_double2(x[i].x + d.x, x[i].y + d.y);
    x[i] = xv;
    xlo[i] = make_float2(0.f, 0.f);
    if (FORM == F_FIELD) {
      const double qi = q[i];
      t0[i] = make_double2(qi * xv.x, qi * xv.y);
    }
  }
}

// true residual r = b - M x in FP64 (t1: the FP64 apply of x's operand), its
// FP32 copy for the recurrence; partials (<r^, r>, ||r||^2 in FP64)
template <int FORM>
__global__ void __launch_bounds__(kThreads) k_true_residual(const double2* __restrict__ b,
                                                            const double2* __restrict__ x,
                                                            const double2* __restrict__ t1, OpArgs<double> a,
                                                            const float2* __restrict__ rh, float2* __restrict__ r,
                                                            double2* __restrict__ part) {
  float hr = 0.f, hi = 0.f;
  double nn = 0.0;
  GRID_LOOP(i, a.n) {
    const double2 bv = b[i];
    const double2 mx = op_at<double, FORM>(x[i], t1, a, i);
    const double ex = bv.x - mx.x, ey = bv.y - mx.y;
    const float2 rv = make_float2((float)ex, (float)ey);
    r[i] = rv;
    const float2 h = rh[i];
    hr += h.x * rv.x + h.y * rv.y;
    hi += h.x * rv.y - h.y * rv.x;
    nn += ex * ex + ey * ey;
  }
  const double re[2] = {(double)hr, nn}, im[2] = {(double)hi, 0.0};
  block_partials<2>(re, im, part);
}

// out = b - M x in FP64 (t1: the FP64 apply of x's operand); partials (||out||^2, ||b||^2)
template <int FORM>
__global__ void __launch_bounds__(kThreads) k_residual_vec(const double2* __restrict__ b,
                                                           const double2* __restrict__ x,
                                                           const double2* __restrict__ t1, OpArgs<double> a,
                                                           double2* __restrict__ out, double2* __restrict__ part) {
  double rr = 0.0, bb = 0.0;
  GRID_LOOP(i, a.n) {
    const double2 bv = b[i];
    const double2 mx = op_at<double, FORM>(x[i], t1, a, i);
    const double2 r = make_double2(bv.x - mx.x, bv.y - mx.y);
    out[i] = r;
    rr += r.x * r.x + r.y * r.y;
    bb += bv.x * bv.x + bv.y * bv.y;
  }
  const double re[2] = {rr, bb}, im[2] = {0.0, 0.0};
  block_partials<2>(re, im, part);
}

// u += e
__global__ void __launch_bounds__(kThreads) k_add(double2* __restrict__ u, const double2* __restrict__ e, long long n) {
  GRID_LOOP(i, n) u[i] = make_double2(u[i].x + e[i].x, u[i].y + e[i].y);
}

// after k_mixed_init (first) or k_true_residual: the stop test on the true
// residual, beta from the new residual, the update flag cleared
__global__ void __launch_bounds__(kScalThreads) k_scal_update(BcgState* __restrict__ st,
                                                              const double2* __restrict__ part) {
  if (st->done) return;
  double2 s[2];
  sum_partials<2>(part, s);
  if (threadIdx.x != 0) return;
  const double2 rho_new = s[0];
  const double rn2 = s[1].x;
  st->rnorm2 = rn2;
  st->update = 0;
  st->maxrr2 = rn2;
  if (st->first) {
    st->first = 0;
    st->bnorm2 = rn2;
    st->best2 = rn2;
    st->tol2 = st->tol * st->tol * rn2;
    st->rho = rho_new;
    st->beta = make_double2(0.0, 0.0);
    if (!(rn2 > 0.0)) st->done = isfinite(rn2) ? BCG_CONVERGED : BCG_NONFINITE;
    return;
  }
  ++st->epoch;
  ++st->updates;
  if (rn2 < 0.25 * st->best2) {
    st->stall = 0;
  } else {
    ++st->stall;
  }
  st->best2 = fmin(st->best2, rn2);
  if (!isfinite(rn2) || !finite2(rho_new)) {
    st->done = BCG_NONFINITE;
  } else if (rn2 < st->tol2) {
    st->done = BCG_CONVERGED;
  } else if (rho_new.x == 0.0 && rho_new.y == 0.0) {
    st->done = BCG_BREAKDOWN;
  } else {
    st->beta = cmul(cdiv(rho_new, st->rho), cdiv(st->alpha, st->omega));
    st->rho = rho_new;
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

// one operator product's apply: V[t0] (field), V[in] (density), grad V[in]
// (Poisson-Boltzmann: d fields into t1)
template <typename R, int FORM>
vp_status apply_v(vp_plan plan, Work<R>& w, const typename Cx<R>::T* in) {
  if (FORM == F_PB) return vp::apply_grad_with_workspace(plan, in, w.t1, cdtype<R>(), w.ws, w.ws_bytes);
  return vp::apply_with_workspace(plan, FORM == F_DENSITY ? (const void*)in : (const void*)w.t0, w.t1, cdtype<R>(),
                                  w.ws, w.ws_bytes);
}

// one iteration on w.s, its state copied to host slot `slot`
template <typename R, int FORM>
vp_status enqueue_iteration(vp_plan plan, Work<R>& w, const OpArgs<R>& a, int slot) {
  k_p<R, FORM><<<kBlocks, kThreads, 0, w.s>>>(w.st, w.p, w.r, w.v, a, w.t0);
  vp_status st = apply_v<R, FORM>(plan, w, w.p);
  if (st != VP_OK) return st;
  k_v<R, FORM><<<kBlocks, kThreads, 0, w.s>>>(w.st, w.v, w.p, w.t1, a, w.rh, w.part);
  k_scal_alpha<<<1, kScalThreads, 0, w.s>>>(w.st, w.part);
  k_s<R, FORM><<<kBlocks, kThreads, 0, w.s>>>(w.st, w.r, w.v, w.x, w.p, a, w.t0, w.part);
  k_scal_s<<<1, kScalThreads, 0, w.s>>>(w.st, w.part);
  if ((st = apply_v<R, FORM>(plan, w, w.r)) != VP_OK) return st;
  k_t<R, FORM><<<kBlocks, kThreads, 0, w.s>>>(w.st, w.t1, w.r, a, w.part);
  k_scal_omega<<<1, kScalThreads, 0, w.s>>>(w.st, w.part);
  k_xr<R><<<kBlocks, kThreads, 0, w.s>>>(w.st, w.x, w.r, w.t1, w.rh, a.n, w.part);
  k_scal_rho<<<1, kScalThreads, 0, w.s>>>(w.st, w.part);
  if (cudaMemcpyAsync(w.host + slot, w.st, sizeof(BcgState), cudaMemcpyDeviceToHost, w.s) != cudaSuccess)
    return VP_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ERR_CUDA;
}

// ||b - M x|| / ||b|| with the operator of this precision (w.t0/w.t1 as scratch,
// the plan's stream s, partials in part)
template <typename R, int FORM>
vp_status residual(vp_plan plan, Work<R>& w, cudaStream_t s, double2* part, const typename Cx<R>::T* b,
                   const typename Cx<R>::T* x, const OpArgs<R>& a, double* out, Err& E) {
  if (FORM == F_FIELD) k_qmul<R><<<kBlocks, kThreads, 0, s>>>(w.t0, a.q, x, a.n);
  vp_status st = apply_v<R, FORM>(plan, w, x);
  if (st != VP_OK) return st;
  k_resid<R, FORM><<<kBlocks, kThreads, 0, s>>>(b, x, w.t1, a, part);
  double2 h[2 * kBlocks];
  BCG_CUDA(E, cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, s));
  BCG_CUDA(E, cudaStreamSynchronize(s));
  double rr = 0.0, bb = 0.0;
  for (int i = 0; i < kBlocks; ++i) {
    rr += h[2 * i].x;
    bb += h[2 * i + 1].x;
  }
  *out = bb > 0 ? sqrt(rr / bb) : sqrt(rr);
  return VP_OK;
}

// the apply workspace of the form (the Poisson-Boltzmann form takes d gradient fields)
size_t form_workspace_bytes(vp_plan plan, int form) {
  return form == F_PB ? vp::plan_grad_workspace_bytes(plan) : vp::plan_apply_workspace_bytes(plan);
}

// vectors of one recurrence; x_own only when the iterate is not the caller's u
template <typename R>
vp_status alloc_work(Work<R>& w, vp_plan plan, long long n, int form, int d, bool own_x, Err& E) {
  using C = typename Cx<R>::T;
  w.n = n;
  BCG_CUDA(E, cudaStreamCreateWithFlags(&w.s, cudaStreamNonBlocking));
  for (int i = 0; i < 2; ++i) BCG_CUDA(E, cudaEventCreateWithFlags(&w.ev[i], cudaEventDisableTiming));
  C** vecs[] = {&w.b, &w.r, &w.rh, &w.p, &w.v};
  for (C** pp : vecs) BCG_CUDA(E, cudaMalloc(pp, n * sizeof(C)));
  BCG_CUDA(E, cudaMalloc(&w.t1, (form == F_PB ? d : 1) * n * sizeof(C)));
  if (form == F_FIELD) BCG_CUDA(E, cudaMalloc(&w.t0, n * sizeof(C)));
  if (own_x) {
    BCG_CUDA(E, cudaMalloc(&w.x_own, n * sizeof(C)));
    w.x = w.x_own;
  }
  w.ws_bytes = form_workspace_bytes(plan, form);
  BCG_CUDA(E, cudaMalloc(&w.ws, w.ws_bytes));
  BCG_CUDA(E, cudaMalloc(&w.part, 2 * kBlocks * sizeof(double2)));
  BCG_CUDA(E, cudaMalloc(&w.st, sizeof(BcgState)));
  BCG_CUDA(E, cudaMallocHost(&w.host, 3 * sizeof(BcgState)));
  return VP_OK;
}

// The solve in one precision R.  src: u_inc (field, density) or rho (PB);
// q: contrast or eps; ge: grad eps (PB).  u: the scattered field or sigma.
// rhs_given: src is the right-hand side b itself (a correction equation), not
// the incident field or rho it is formed from.
template <typename R, int FORM>
vp_status solve(vp_plan plan, const R* q, const R* ge, const typename Cx<R>::T* src, typename Cx<R>::T* u,
                double k2d, int d, long long n, double tol, int maxit, double* history, vp_ls_stats* stats, Err& E,
                bool rhs_given = false) {
  const auto t_start = std::chrono::steady_clock::now();
  Work<R> w;
  vp_status st = alloc_work<R>(w, plan, n, FORM, d, FORM == F_DENSITY, E);
  if (st != VP_OK) return st;
  if (FORM != F_DENSITY) w.x = u;  // the field and PB forms iterate on u itself
  const OpArgs<R> a{q, ge, (R)k2d, d, n};
  PlanGuard guard{plan, vp::plan_stream(plan), VP_FP32};
  BCG_CUDA(E, cudaStreamSynchronize(guard.stream));  // inputs produced on the plan's stream
  if ((st = vp_plan_set_stream(plan, w.s)) != VP_OK) return st;

  // right-hand side (an uncaptured apply also sets up every pass kernel before capture)
  if (FORM == F_FIELD) {
    k_qmul<R><<<kBlocks, kThreads, 0, w.s>>>(w.t0, q, src, n);
    if ((st = apply_v<R, FORM>(plan, w, src)) != VP_OK) return st;
  } else {
    if ((st = apply_v<R, FORM>(plan, w, src)) != VP_OK) return st;
  }
  if (rhs_given)  // b = src (the Poisson-Boltzmann form's right-hand side is src itself)
    k_start<R, F_PB><<<kBlocks, kThreads, 0, w.s>>>(src, a, w.b, w.r, w.rh, w.x, w.p, w.v, w.part);
  else if (FORM == F_FIELD)
    k_start<R, FORM><<<kBlocks, kThreads, 0, w.s>>>(w.t1, a, w.b, w.r, w.rh, w.x, w.p, w.v, w.part);
  else
    k_start<R, FORM><<<kBlocks, kThreads, 0, w.s>>>(src, a, w.b, w.r, w.rh, w.x, w.p, w.v, w.part);
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
      vp_status cs = enqueue_iteration<R, FORM>(plan, w, a, k);
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
  if (FORM == F_DENSITY) {  // u = V[s]
    BCG_CUDA(E, cudaGetLastError());
    st = vp::apply_with_workspace(plan, w.x, u, cdtype<R>(), w.ws, w.ws_bytes);
    if (st != VP_OK) return st;
  }
  BCG_CUDA(E, cudaStreamSynchronize(w.s));
  const auto t_end = std::chrono::steady_clock::now();

  // true residual ||b - M x|| / ||b||, the operator and b evaluated in FP64
  double tr = 0.0;
  if constexpr (sizeof(R) == 8) {
    st = residual<R, FORM>(plan, w, w.s, w.part, w.b, w.x, a, &tr, E);
    if (st != VP_OK) return st;
  } else {
    Work<double> w64;
    if ((st = alloc_work<double>(w64, plan, n, FORM, d, false, E)) != VP_OK) return st;
    guard.restore_prec = true;
    if ((st = vp_plan_set_precision(plan, VP_FP64)) != VP_OK) return st;
    cudaFree(w64.ws);  // resize for the FP64 passes
    w64.ws = nullptr;
    w64.ws_bytes = form_workspace_bytes(plan, FORM);
    BCG_CUDA(E, cudaMalloc(&w64.ws, w64.ws_bytes));
    BCG_CUDA(E, cudaStreamSynchronize(w.s));
    if ((st = vp_plan_set_stream(plan, w64.s)) != VP_OK) return st;
    double* q64 = reinterpret_cast<double*>(w64.rh);  // n doubles fit in n complex
    k_widen_r<<<kBlocks, kThreads, 0, w64.s>>>(q64, reinterpret_cast<const float*>(q), n);
    struct FreeGe {
      double* p = nullptr;
      ~FreeGe() { cudaFree(p); }
    } ge64;
    if (FORM == F_PB) {
      BCG_CUDA(E, cudaMalloc(&ge64.p, (size_t)d * n * sizeof(double)));
      k_widen_r<<<kBlocks, kThreads, 0, w64.s>>>(ge64.p, reinterpret_cast<const float*>(ge), (long long)d * n);
    }
    double2* src64 = w64.p;
    k_widen_c<<<kBlocks, kThreads, 0, w64.s>>>(src64, reinterpret_cast<const float2*>(src), n);
    const OpArgs<double> a64{q64, ge64.p, k2d, d, n};
    if (rhs_given) {
      k_rhs<double, F_PB><<<kBlocks, kThreads, 0, w64.s>>>(src64, a64, w64.b);
    } else if (FORM == F_FIELD) {  // b = k^2 V[q u_inc] in FP64
      k_qmul<double><<<kBlocks, kThreads, 0, w64.s>>>(w64.t0, q64, src64, n);
      if ((st = apply_v<double, FORM>(plan, w64, src64)) != VP_OK) return st;
      k_rhs<double, FORM><<<kBlocks, kThreads, 0, w64.s>>>(w64.t1, a64, w64.b);
    } else {
      k_rhs<double, FORM><<<kBlocks, kThreads, 0, w64.s>>>(src64, a64, w64.b);
    }
    double2* x64 = w64.r;
    k_widen_c<<<kBlocks, kThreads, 0, w64.s>>>(x64, reinterpret_cast<const float2*>(w.x), n);
    st = residual<double, FORM>(plan, w64, w64.s, w64.part, w64.b, x64, a64, &tr, E);
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

struct GraphHolder {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  cudaStream_t s = nullptr;  // synchronised before destruction
  ~GraphHolder() {
    if (s) cudaStreamSynchronize(s);
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
  }
};

// Mixed precision: q, ge (PB), src, u in FP64; the recurrence in FP32.
template <int FORM>
vp_status solve_mixed(vp_plan plan, const double* q64, const double* ge64, const double2* src, double2* u, double k2d,
                      int d, long long n, double tol, double delta, int maxit, double* history, vp_ls_stats* stats,
                      Err& E) {
  const auto t_start = std::chrono::steady_clock::now();
  PlanGuard guard{plan, vp::plan_stream(plan), vp::plan_is_fp64(plan) ? VP_FP64 : VP_FP32};
  guard.restore_prec = true;
  vp_status st = vp_plan_set_precision(plan, VP_FP32);
  if (st != VP_OK) return st;
  // FP32 recurrence: r, r^, p, v, t1 (and t0), x_lo, the FP32 workspace, state
  Work<float> w;
  if ((st = alloc_work<float>(w, plan, n, FORM, d, true, E)) != VP_OK) return st;
  struct Free {
    void* p = nullptr;
    ~Free() { cudaFree(p); }
  } q32, ge32;
  BCG_CUDA(E, cudaMalloc(&q32.p, n * sizeof(float)));
  if (FORM == F_PB) BCG_CUDA(E, cudaMalloc(&ge32.p, (size_t)d * n * sizeof(float)));
  // FP64 side: b, the solution x (the caller's u unless the density form),
  // t1 (and t0), the FP64 workspace
  Work<double> w64;
  w64.n = n;
  if ((st = vp_plan_set_precision(plan, VP_FP64)) != VP_OK) return st;
  BCG_CUDA(E, cudaMalloc(&w64.b, n * sizeof(double2)));
  BCG_CUDA(E, cudaMalloc(&w64.t1, (FORM == F_PB ? d : 1) * n * sizeof(double2)));
  if (FORM == F_FIELD) BCG_CUDA(E, cudaMalloc(&w64.t0, n * sizeof(double2)));
  if (FORM == F_DENSITY) {
    BCG_CUDA(E, cudaMalloc(&w64.x_own, n * sizeof(double2)));
    w64.x = w64.x_own;
  } else {
    w64.x = u;
  }
  w64.ws_bytes = form_workspace_bytes(plan, FORM);
  BCG_CUDA(E, cudaMalloc(&w64.ws, w64.ws_bytes));
  BCG_CUDA(E, cudaStreamSynchronize(guard.stream));
  if ((st = vp_plan_set_stream(plan, w.s)) != VP_OK) return st;
  const OpArgs<double> a64{q64, ge64, k2d, d, n};
  const OpArgs<float> a32{reinterpret_cast<const float*>(q32.p), reinterpret_cast<const float*>(ge32.p), (float)k2d,
                          d, n};

  // FP64 right-hand side (its apply also sets up the FP64 passes before capture)
  k_narrow_r<<<kBlocks, kThreads, 0, w.s>>>(reinterpret_cast<float*>(q32.p), q64, n);
  if (FORM == F_PB)
    k_narrow_r<<<kBlocks, kThreads, 0, w.s>>>(reinterpret_cast<float*>(ge32.p), ge64, (long long)d * n);
  if (FORM == F_FIELD) {
    k_qmul<double><<<kBlocks, kThreads, 0, w.s>>>(w64.t0, q64, src, n);
    if ((st = apply_v<double, FORM>(plan, w64, src)) != VP_OK) return st;
    k_rhs<double, FORM><<<kBlocks, kThreads, 0, w.s>>>(w64.t1, a64, w64.b);
  } else {
    if ((st = apply_v<double, FORM>(plan, w64, src)) != VP_OK) return st;
    k_rhs<double, FORM><<<kBlocks, kThreads, 0, w.s>>>(src, a64, w64.b);
  }
  k_mixed_init<<<kBlocks, kThreads, 0, w.s>>>(w64.b, w.r, w.rh, w.p, w.v, w.x, w64.x, n, w.part);
  BcgState init;
  memset(&init, 0, sizeof(init));
  init.rho = init.alpha = init.omega = make_double2(1.0, 0.0);
  init.tol = tol;
  init.delta2 = delta * delta;
  init.first = 1;
  init.mixed = 1;
  w.host[2] = init;
  BCG_CUDA(E, cudaMemcpyAsync(w.st, w.host + 2, sizeof(BcgState), cudaMemcpyHostToDevice, w.s));
  k_scal_update<<<1, kScalThreads, 0, w.s>>>(w.st, w.part);
  BCG_CUDA(E, cudaGetLastError());

  // the reliable update as one graph (FP64 passes)
  GraphHolder upd;
  upd.s = w.s;
  BCG_CUDA(E, cudaStreamBeginCapture(w.s, cudaStreamCaptureModeThreadLocal));
  k_accumulate<FORM><<<kBlocks, kThreads, 0, w.s>>>(w64.x, w.x, q64, w64.t0, n);
  st = apply_v<double, FORM>(plan, w64, w64.x);
  k_true_residual<FORM><<<kBlocks, kThreads, 0, w.s>>>(w64.b, w64.x, w64.t1, a64, w.rh, w.r, w.part);
  k_scal_update<<<1, kScalThreads, 0, w.s>>>(w.st, w.part);
  cudaError_t ce = cudaStreamEndCapture(w.s, &upd.g);
  if (st != VP_OK) return st;
  BCG_CUDA(E, ce);
  BCG_CUDA(E, cudaGraphInstantiate(&upd.x, upd.g, 0));

  // the FP32 iteration as two graphs (an uncaptured apply first sets up the FP32 passes)
  if ((st = vp_plan_set_precision(plan, VP_FP32)) != VP_OK) return st;
  if ((st = apply_v<float, FORM>(plan, w, w.p)) != VP_OK) return st;
  for (int k = 0; k < 2; ++k) {
    BCG_CUDA(E, cudaStreamBeginCapture(w.s, cudaStreamCaptureModeThreadLocal));
    vp_status cs = enqueue_iteration<float, FORM>(plan, w, a32, k);
    ce = cudaStreamEndCapture(w.s, &w.g[k]);
    if (cs != VP_OK) return cs;
    BCG_CUDA(E, ce);
    BCG_CUDA(E, cudaGraphInstantiate(&w.gx[k], w.g[k], 0));
  }
  BCG_CUDA(E, cudaMemcpyAsync(w.host + 2, w.st, sizeof(BcgState), cudaMemcpyDeviceToHost, w.s));
  BCG_CUDA(E, cudaStreamSynchronize(w.s));
  if (history) history[0] = 1.0;
  BcgState last = w.host[2];
  if (!last.done) {
    // iteration j runs while the host reads iteration j-1's state; an update
    // requested by iteration j-1 runs after iteration j (which then does nothing)
    int epoch = last.epoch;
    for (int j = 1; j <= maxit + 1; ++j) {
      if (j <= maxit) {
        BCG_CUDA(E, cudaGraphLaunch(w.gx[j & 1], w.s));
        BCG_CUDA(E, cudaEventRecord(w.ev[j & 1], w.s));
      }
      if (j >= 2) {
        BCG_CUDA(E, cudaEventSynchronize(w.ev[(j - 1) & 1]));
        last = w.host[(j - 1) & 1];
        // indexed by completed iterations: the idle iteration after an update request rewrites its entry
        if (history && last.bnorm2 > 0) history[last.iterations] = sqrt(last.rnorm2 / last.bnorm2);
        if (last.done || last.stall >= kMaxStall) break;
        if (last.update && last.epoch == epoch) {
          BCG_CUDA(E, cudaGraphLaunch(upd.x, w.s));
          ++epoch;
        }
      }
    }
    BCG_CUDA(E, cudaStreamSynchronize(w.s));
    if (last.done != BCG_CONVERGED) {  // fold the last correction into x
      BCG_CUDA(E, cudaGraphLaunch(upd.x, w.s));
    }
    BCG_CUDA(E, cudaMemcpyAsync(w.host + 2, w.st, sizeof(BcgState), cudaMemcpyDeviceToHost, w.s));
    BCG_CUDA(E, cudaStreamSynchronize(w.s));
    last = w.host[2];
  }
  if ((st = vp_plan_set_precision(plan, VP_FP64)) != VP_OK) return st;
  if (last.done != BCG_CONVERGED) {
    // FP32 products did not reach tol within the budget (the iteration count,
    // a stall or a breakdown): FP64 Bi-CGStab on the correction equation
    // M e = r = b - M x from the mixed iterate x (M x + M e = b), to tol ||b||
    struct Buf {
      double2* p = nullptr;
      ~Buf() { cudaFree(p); }
    } r64, e64;
    BCG_CUDA(E, cudaMalloc(&r64.p, n * sizeof(double2)));
    BCG_CUDA(E, cudaMalloc(&e64.p, n * sizeof(double2)));
    if (FORM == F_FIELD) k_qmul<double><<<kBlocks, kThreads, 0, w.s>>>(w64.t0, q64, w64.x, n);
    if ((st = apply_v<double, FORM>(plan, w64, w64.x)) != VP_OK) return st;
    k_residual_vec<FORM><<<kBlocks, kThreads, 0, w.s>>>(w64.b, w64.x, w64.t1, a64, r64.p, w.part);
    double2 h[2 * kBlocks];
    BCG_CUDA(E, cudaMemcpyAsync(h, w.part, sizeof(h), cudaMemcpyDeviceToHost, w.s));
    BCG_CUDA(E, cudaStreamSynchronize(w.s));
    double rr = 0.0, bb = 0.0;
    for (int i = 0; i < kBlocks; ++i) {
      rr += h[2 * i].x;
      bb += h[2 * i + 1].x;
    }
    double rn = sqrt(rr);
    const double bn = sqrt(bb);
    if (last.done == BCG_NONFINITE || !isfinite(rn)) {
      // the FP32 phase left a non-finite iterate (an overflow in FP32): the
      // FP64 solve starts from zero, r = b
      BCG_CUDA(E, cudaMemsetAsync(w64.x, 0, n * sizeof(double2), w.s));
      if (FORM == F_FIELD) k_qmul<double><<<kBlocks, kThreads, 0, w.s>>>(w64.t0, q64, w64.x, n);
      if ((st = apply_v<double, FORM>(plan, w64, w64.x)) != VP_OK) return st;
      k_residual_vec<FORM><<<kBlocks, kThreads, 0, w.s>>>(w64.b, w64.x, w64.t1, a64, r64.p, w.part);
      BCG_CUDA(E, cudaMemcpyAsync(h, w.part, sizeof(h), cudaMemcpyDeviceToHost, w.s));
      BCG_CUDA(E, cudaStreamSynchronize(w.s));
      rr = 0.0;
      for (int i = 0; i < kBlocks; ++i) rr += h[2 * i].x;
      rn = sqrt(rr);
      if (!isfinite(rn)) {
        E.msg = "mixed-precision Bi-CGStab: the right-hand side is not finite in FP64";
        return E.st = VP_ERR_NUMERICAL;
      }
    }
    vp_ls_stats s64;
    memset(&s64, 0, sizeof(s64));
    if (rn > 0.0) {
      st = solve<double, FORM>(plan, q64, ge64, r64.p, e64.p, k2d, d, n, tol * bn / rn, maxit, nullptr, &s64, E,
                               true);
      if (st != VP_OK && st != VP_ERR_NUMERICAL) return st;
    } else {
      BCG_CUDA(E, cudaMemsetAsync(e64.p, 0, n * sizeof(double2), w.s));
    }
    // u = x + e (field, Poisson-Boltzmann); u = V[s] + V[e_s] (density: the
    // correction solve returns V[e_s])
    if (FORM == F_DENSITY) {
      vp_status sa = vp::apply_with_workspace(plan, w64.x, u, VP_C128, w64.ws, w64.ws_bytes);
      if (sa != VP_OK) return sa;
    }
    k_add<<<kBlocks, kThreads, 0, w.s>>>(u, e64.p, n);
    BCG_CUDA(E, cudaStreamSynchronize(w.s));
    const auto t_end = std::chrono::steady_clock::now();
    if (stats) {
      stats->iterations = last.iterations + s64.iterations;
      stats->matvecs = last.matvecs + s64.matvecs;
      stats->restarts = last.updates;
      stats->used_fallback = 1;
      // the correction solve's residuals are relative to ||r||
      stats->estimated_residual = s64.estimated_residual * rn / bn;
      stats->true_residual = s64.true_residual * rn / bn;
      stats->seconds = std::chrono::duration<double>(t_end - t_start).count();
    }
    return st;
  }
  if (FORM == F_DENSITY) {  // u = V[s] in FP64
    st = vp::apply_with_workspace(plan, w64.x, u, VP_C128, w64.ws, w64.ws_bytes);
    if (st != VP_OK) return st;
  }
  BCG_CUDA(E, cudaStreamSynchronize(w.s));
  const auto t_end = std::chrono::steady_clock::now();
  double tr = 0.0;
  if ((st = residual<double, FORM>(plan, w64, w.s, w.part, w64.b, w64.x, a64, &tr, E)) != VP_OK) return st;
  if (stats) {
    stats->iterations = last.iterations;
    stats->matvecs = last.matvecs;
    stats->restarts = last.updates;
    stats->used_fallback = 0;
    stats->estimated_residual = last.bnorm2 > 0 ? sqrt(last.rnorm2 / last.bnorm2) : 0.0;
    stats->true_residual = tr;
    stats->seconds = std::chrono::duration<double>(t_end - t_start).count();
  }
  return VP_OK;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Restarted GMRES(m) in FP64: the paper's solver for the Section 5.2 equation
// P s = -eps s + grad(eps) . grad V[s] = rho (Saad & Schultz 1986; Saad,
// Iterative Methods for Sparse Linear Systems, Alg. 6.9, with the Givens
// rotations of Section 6.5.3).  Each cycle starts from v_0 = r / ||r||,
// r = b - P x (r = b in the first cycle, x = 0).  Arnoldi step j:
//   w = P v_j (one exact-gradient apply), then classical Gram-Schmidt applied
//   twice ("twice is enough"): per pass one kernel of all the inner products
//   h_i = <v_i, w>, i <= j (FP64, per-block partials summed in a fixed order)
//   and one kernel w -= sum_i h_i v_i; h_{j+1,j} = ||w||, v_{j+1} = w / ||w||.
// The column of H (j + 2 values) goes to the host, which applies the earlier
// rotations, forms the new one and updates g; |g_{j+1}| / ||b|| is the
// residual estimate.  The cycle ends after m steps or when the estimate is
// below tol (or the step budget is spent); the host solves the triangular
// system R y = g and x += sum_i y_i v_i runs on the device.
// ---------------------------------------------------------------------------
constexpr int kGmDots = 4;            // inner products per block row of k_gm_dots
constexpr int kGmMaxRestart = 512;    // the largest restart length m accepted

// part[(blockIdx.y * kBlocks + blockIdx.x) * kGmDots + k] = this block's share
// of <v_i, w>, i = blockIdx.y * kGmDots + k < count (zero for i >= count)
__global__ void __launch_bounds__(kThreads) k_gm_dots(const double2* __restrict__ V, long long n, int count,
                                                      const double2* __restrict__ w, double2* __restrict__ part) {
  const int i0 = blockIdx.y * kGmDots;
  double re[kGmDots], im[kGmDots];
#pragma unroll
  for (int k = 0; k < kGmDots; ++k) re[k] = im[k] = 0.0;
  GRID_LOOP(e, n) {
    const double2 wv = w[e];
#pragma unroll
    for (int k = 0; k < kGmDots; ++k)
      if (i0 + k < count) {
        const double2 v = V[(long long)(i0 + k) * n + e];
        re[k] += v.x * wv.x + v.y * wv.y;
        im[k] += v.x * wv.y - v.y * wv.x;
      }
  }
  block_partials<kGmDots>(re, im, part + (size_t)blockIdx.y * kBlocks * kGmDots);
}

// h[i] = <v_i, w> from the partials (one block per row of kGmDots products);
// col[i] = h[i] (first pass) or col[i] + h[i] (second pass)
__global__ void __launch_bounds__(kScalThreads) k_gm_reduce(const double2* __restrict__ part, int count,
                                                            double2* __restrict__ h, double2* __restrict__ col,
                                                            int accumulate) {
  double2 s[kGmDots];
  sum_partials<kGmDots>(part + (size_t)blockIdx.x * kBlocks * kGmDots, s);
  if (threadIdx.x == 0)
    for (int k = 0; k < kGmDots; ++k) {
      const int i = blockIdx.x * kGmDots + k;
      if (i < count) {
        h[i] = s[k];
        col[i] = accumulate ? make_double2(col[i].x + s[k].x, col[i].y + s[k].y) : s[k];
      }
    }
}

// w += sign * sum_{i < count} c_i v_i   (sign -1: a Gram-Schmidt pass; +1: x += V y)
__global__ void __launch_bounds__(kThreads) k_gm_axpy(double2* __restrict__ w, const double2* __restrict__ V,
                                                      long long n, int count, const double2* __restrict__ c,
                                                      double sign) {
  __shared__ double2 cs[kGmMaxRestart + 1];
  for (int i = threadIdx.x; i < count; i += blockDim.x) cs[i] = make_double2(sign * c[i].x, sign * c[i].y);
  __syncthreads();
  GRID_LOOP(e, n) {
    double2 acc = w[e];
    for (int i = 0; i < count; ++i) {
      const double2 v = V[(long long)i * n + e];
      acc.x += cs[i].x * v.x - cs[i].y * v.y;
      acc.y += cs[i].x * v.y + cs[i].y * v.x;
    }
    w[e] = acc;
  }
}

// partials of ||w||^2
__global__ void __launch_bounds__(kThreads) k_gm_norm(const double2* __restrict__ w, long long n,
                                                      double2* __restrict__ part) {
  double s = 0.0;
  GRID_LOOP(e, n) s += w[e].x * w[e].x + w[e].y * w[e].y;
  const double re[1] = {s}, im[1] = {0.0};
  block_partials<1>(re, im, part);
}

// *entry = (||w||, 0); *inv = 1 / ||w|| (0 when w = 0)
__global__ void __launch_bounds__(kScalThreads) k_gm_norm_reduce(const double2* __restrict__ part,
                                                                 double2* __restrict__ entry, double* __restrict__ inv) {
  double2 s[1];
  sum_partials<1>(part, s);
  if (threadIdx.x == 0) {
    const double nr = sqrt(s[0].x);
    *entry = make_double2(nr, 0.0);
    *inv = nr > 0.0 ? 1.0 / nr : 0.0;
  }
}

// w *= *inv (device scalar) or w *= c (host scalar, inv == nullptr)
__global__ void __launch_bounds__(kThreads) k_gm_scale(double2* __restrict__ w, long long n,
                                                       const double* __restrict__ inv, double c) {
  const double f = inv ? *inv : c;
  GRID_LOOP(e, n) w[e] = make_double2(w[e].x * f, w[e].y * f);
}

// w = P v (t1: the d components of grad V[v])
__global__ void __launch_bounds__(kThreads) k_gm_op(const double2* __restrict__ v, const double2* __restrict__ t1,
                                                    OpArgs<double> a, double2* __restrict__ w) {
  GRID_LOOP(i, a.n) w[i] = op_at<double, F_PB>(v[i], t1, a, i);
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
};

// The GMRES(m) solve of the Poisson-Boltzmann form; the plan is FP64.
vp_status gmres_pb(vp_plan plan, const double* eps, const double* ge, const double2* rho, double2* x, int d,
                   long long n, double tol, int m, int maxit, double* history, vp_ls_stats* stats, Err& E) {
  using cd = std::complex<double>;
  const auto t_start = std::chrono::steady_clock::now();
  m = m < maxit ? m : maxit;
  const int rows = (m + 1 + kGmDots - 1) / kGmDots;
  Work<double> w;  // stream, t1 (d gradient fields), apply workspace, partials
  w.n = n;
  BCG_CUDA(E, cudaStreamCreateWithFlags(&w.s, cudaStreamNonBlocking));
  BCG_CUDA(E, cudaMalloc(&w.t1, (size_t)d * n * sizeof(double2)));
  w.ws_bytes = form_workspace_bytes(plan, F_PB);
  BCG_CUDA(E, cudaMalloc(&w.ws, w.ws_bytes));
  BCG_CUDA(E, cudaMalloc(&w.part, 2 * kBlocks * sizeof(double2)));
  DevBuf V, partg, h, col, inv;
  BCG_CUDA(E, cudaMalloc(&V.p, (size_t)(m + 1) * n * sizeof(double2)));
  BCG_CUDA(E, cudaMalloc(&partg.p, (size_t)rows * kBlocks * kGmDots * sizeof(double2)));
  BCG_CUDA(E, cudaMalloc(&h.p, (m + 1) * sizeof(double2)));
  BCG_CUDA(E, cudaMalloc(&col.p, (m + 2) * sizeof(double2)));
  BCG_CUDA(E, cudaMalloc(&inv.p, sizeof(double)));
  struct HostBuf {
    double2* p = nullptr;
    ~HostBuf() { cudaFreeHost(p); }
  } hc;
  BCG_CUDA(E, cudaMallocHost(&hc.p, (m + 2) * sizeof(double2)));
  double2* const Vb = static_cast<double2*>(V.p);
  double2* const hd = static_cast<double2*>(h.p);
  double2* const cold = static_cast<double2*>(col.p);
  double* const invd = static_cast<double*>(inv.p);
  double2* const pg = static_cast<double2*>(partg.p);
  PlanGuard guard{plan, vp::plan_stream(plan), VP_FP64};
  BCG_CUDA(E, cudaStreamSynchronize(guard.stream));  // inputs produced on the plan's stream
  vp_status st = vp_plan_set_stream(plan, w.s);
  if (st != VP_OK) return st;
  const OpArgs<double> a{eps, ge, 0.0, d, n};
  auto host_sum = [&](int K, double* out) -> vp_status {  // out[k] = sum of the kBlocks partials' .x
    std::vector<double2> hp((size_t)K * kBlocks);
    BCG_CUDA(E, cudaMemcpyAsync(hp.data(), w.part, hp.size() * sizeof(double2), cudaMemcpyDeviceToHost, w.s));
    BCG_CUDA(E, cudaStreamSynchronize(w.s));
    for (int k = 0; k < K; ++k) {
      out[k] = 0.0;
      for (int b = 0; b < kBlocks; ++b) out[k] += hp[(size_t)b * K + k].x;
    }
    return VP_OK;
  };

  BCG_CUDA(E, cudaMemsetAsync(x, 0, n * sizeof(double2), w.s));
  k_gm_norm<<<kBlocks, kThreads, 0, w.s>>>(rho, n, w.part);
  double bn2 = 0.0;
  if ((st = host_sum(1, &bn2)) != VP_OK) return st;
  const double bn = sqrt(bn2);
  if (history) history[0] = 1.0;
  int it = 0, cycles = 0, matvecs = 0, restarts = 0;
  double est = bn > 0 ? 1.0 : 0.0;
  bool breakdown = false;
  std::vector<cd> H((size_t)(m + 1) * m), g(m + 1), sn(m), y(m);
  std::vector<double> cs(m);
  auto Hc = [&](int i, int j) -> cd& { return H[(size_t)j * (m + 1) + i]; };
  while (bn > 0) {
    // v_0 = r / ||r||
    double beta = bn;
    if (cycles == 0) {
      BCG_CUDA(E, cudaMemcpyAsync(Vb, rho, n * sizeof(double2), cudaMemcpyDeviceToDevice, w.s));
    } else {
      if ((st = apply_v<double, F_PB>(plan, w, x)) != VP_OK) return st;
      k_residual_vec<F_PB><<<kBlocks, kThreads, 0, w.s>>>(rho, x, w.t1, a, Vb, w.part);
      double sums[2];
      if ((st = host_sum(2, sums)) != VP_OK) return st;
      ++matvecs;
      ++restarts;
      beta = sqrt(sums[0]);
      est = beta / bn;
      if (history) history[it] = est;  // the explicit residual replaces the estimate
      if (est < tol || !std::isfinite(est)) break;
    }
    if (it >= maxit) break;
    if (beta == 0.0) break;
    k_gm_scale<<<kBlocks, kThreads, 0, w.s>>>(Vb, n, nullptr, 1.0 / beta);
    std::fill(g.begin(), g.end(), cd(0.0));
    g[0] = beta;
    int jend = 0;
    for (int j = 0; j < m; ++j) {
      double2* const vj = Vb + (size_t)j * n;
      double2* const wv = Vb + (size_t)(j + 1) * n;
      if ((st = apply_v<double, F_PB>(plan, w, vj)) != VP_OK) return st;
      k_gm_op<<<kBlocks, kThreads, 0, w.s>>>(vj, w.t1, a, wv);
      ++matvecs;
      const int cnt = j + 1, rws = (cnt + kGmDots - 1) / kGmDots;
      for (int pass = 0; pass < 2; ++pass) {
        k_gm_dots<<<dim3(kBlocks, rws), kThreads, 0, w.s>>>(Vb, n, cnt, wv, pg);
        k_gm_reduce<<<rws, kScalThreads, 0, w.s>>>(pg, cnt, hd, cold, pass);
        k_gm_axpy<<<kBlocks, kThreads, 0, w.s>>>(wv, Vb, n, cnt, hd, -1.0);
      }
      k_gm_norm<<<kBlocks, kThreads, 0, w.s>>>(wv, n, w.part);
      k_gm_norm_reduce<<<1, kScalThreads, 0, w.s>>>(w.part, cold + j + 1, invd);
      k_gm_scale<<<kBlocks, kThreads, 0, w.s>>>(wv, n, invd, 0.0);
      BCG_CUDA(E, cudaMemcpyAsync(hc.p, cold, (j + 2) * sizeof(double2), cudaMemcpyDeviceToHost, w.s));
      BCG_CUDA(E, cudaStreamSynchronize(w.s));
      BCG_CUDA(E, cudaGetLastError());
      bool finite = true;
      for (int i = 0; i <= j + 1; ++i) {
        Hc(i, j) = cd(hc.p[i].x, hc.p[i].y);
        finite = finite && std::isfinite(hc.p[i].x) && std::isfinite(hc.p[i].y);
      }
      if (!finite) {
        E.msg = "GMRES produced a non-finite value";
        return E.st = VP_ERR_NUMERICAL;
      }
      for (int i = 0; i < j; ++i) {  // the earlier rotations
        const cd t = cs[i] * Hc(i, j) + sn[i] * Hc(i + 1, j);
        Hc(i + 1, j) = -std::conj(sn[i]) * Hc(i, j) + cs[i] * Hc(i + 1, j);
        Hc(i, j) = t;
      }
      const double a0 = std::abs(Hc(j, j)), a1 = std::abs(Hc(j + 1, j)), den = std::hypot(a0, a1);
      if (den == 0.0) {  // P v_j = 0 within the basis: no progress is possible
        breakdown = true;
        break;
      }
      if (a0 == 0.0) {
        cs[j] = 0.0;
        sn[j] = std::conj(Hc(j + 1, j)) / den;
      } else {
        cs[j] = a0 / den;
        sn[j] = (Hc(j, j) / a0) * std::conj(Hc(j + 1, j)) / den;
      }
      Hc(j, j) = cs[j] * Hc(j, j) + sn[j] * Hc(j + 1, j);
      Hc(j + 1, j) = 0.0;
      g[j + 1] = -std::conj(sn[j]) * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      jend = j + 1;
      est = std::abs(g[j + 1]) / bn;
      if (history) history[it] = est;
      if (est < tol || it >= maxit) break;
    }
    // x += V y with R y = g (back substitution on the rotated H)
    for (int i = jend - 1; i >= 0; --i) {
      cd acc = g[i];
      for (int k = i + 1; k < jend; ++k) acc -= Hc(i, k) * y[k];
      y[i] = acc / Hc(i, i);
    }
    if (jend > 0) {
      for (int i = 0; i < jend; ++i) hc.p[i] = make_double2(y[i].real(), y[i].imag());
      BCG_CUDA(E, cudaMemcpyAsync(hd, hc.p, jend * sizeof(double2), cudaMemcpyHostToDevice, w.s));
      k_gm_axpy<<<kBlocks, kThreads, 0, w.s>>>(x, Vb, n, jend, hd, 1.0);
      BCG_CUDA(E, cudaStreamSynchronize(w.s));  // hc.p is rewritten by the next step's copy
    }
    ++cycles;
    if (breakdown || est < tol || it >= maxit) break;
  }
  BCG_CUDA(E, cudaStreamSynchronize(w.s));
  BCG_CUDA(E, cudaGetLastError());
  const auto t_end = std::chrono::steady_clock::now();
  double tr = 0.0;
  if (bn > 0 && (st = residual<double, F_PB>(plan, w, w.s, w.part, rho, x, a, &tr, E)) != VP_OK) return st;
  if (stats) {
    stats->iterations = it;
    stats->matvecs = matvecs;
    stats->restarts = restarts;  // explicit residuals formed at the start of a cycle
    stats->used_fallback = 0;
    stats->estimated_residual = est;
    stats->true_residual = tr;
    stats->seconds = std::chrono::duration<double>(t_end - t_start).count();
  }
  if (breakdown) {
    E.msg = "GMRES breakdown (a zero Hessenberg column) before convergence";
    return E.st = VP_ERR_NUMERICAL;
  }
  return VP_OK;
}

}  // namespace

namespace {

// common argument checks of the entry points; *n and *d on success
vp_status check_args(vp_plan plan, bool pb, const void* q, const void* ge, const void* src, const void* u, int form,
                     double tol, int maxit, long long* n, int* d, double* k) {
  int N = 0;
  auto bad = [](const char* m) {
    vp::ls_set_error(m);
    return VP_ERR_INVALID_ARG;
  };
  if (!plan) return bad("plan is NULL");
  vp_status st = vp_plan_info(plan, d, &N, k, nullptr, nullptr);
  if (st != VP_OK) return st;
  if (pb) {
    if (vp::plan_kernel(plan) != VP_LAPLACE) return bad("the Poisson-Boltzmann solve needs a Laplace plan");
    if (!q || !ge || !src || !u) return bad("eps, grad_eps, rho and sigma are required");
    if (u == src) return bad("sigma may not alias rho");
  } else {
    if (!(*k > 0)) return bad("the scattering solve needs a Helmholtz plan");
    if (!q || !src || !u) return bad("q, u_inc and u are required");
    if (u == src) return bad("u may not alias u_inc");
    if (form != VP_LS_FIELD && form != VP_LS_DENSITY) return bad("form must be VP_LS_FIELD or VP_LS_DENSITY");
  }
  if (!(tol > 0) || maxit < 1) return bad("tol > 0 and maxit >= 1 required");
  *n = vp::plan_points(plan);  // prod_j N_j
  return VP_OK;
}

template <typename R>
vp_status run_one(vp_plan plan, int FORMv, const void* q, const void* ge, const void* src, void* u, double k2, int d,
                  long long n, double tol, int maxit, double* history, vp_ls_stats* stats, Err& E) {
  using C = typename Cx<R>::T;
  auto qq = reinterpret_cast<const R*>(q);
  auto gg = reinterpret_cast<const R*>(ge);
  auto ss = reinterpret_cast<const C*>(src);
  auto uo = reinterpret_cast<C*>(u);
  if (FORMv == F_FIELD) return solve<R, F_FIELD>(plan, qq, gg, ss, uo, k2, d, n, tol, maxit, history, stats, E);
  if (FORMv == F_DENSITY) return solve<R, F_DENSITY>(plan, qq, gg, ss, uo, k2, d, n, tol, maxit, history, stats, E);
  return solve<R, F_PB>(plan, qq, gg, ss, uo, k2, d, n, tol, maxit, history, stats, E);
}

vp_status run_mixed(vp_plan plan, int FORMv, const double* q, const double* ge, const void* src, void* u, double k2,
                    int d, long long n, double tol, double delta, int maxit, double* history, vp_ls_stats* stats,
                    Err& E) {
  auto ss = reinterpret_cast<const double2*>(src);
  auto uo = reinterpret_cast<double2*>(u);
  if (FORMv == F_FIELD)
    return solve_mixed<F_FIELD>(plan, q, ge, ss, uo, k2, d, n, tol, delta, maxit, history, stats, E);
  if (FORMv == F_DENSITY)
    return solve_mixed<F_DENSITY>(plan, q, ge, ss, uo, k2, d, n, tol, delta, maxit, history, stats, E);
  return solve_mixed<F_PB>(plan, q, ge, ss, uo, k2, d, n, tol, delta, maxit, history, stats, E);
}

vp_status finish(vp_status st, const Err& E) {
  if (st != VP_OK) vp::ls_set_error(E.msg.empty() ? vp_status_string(st) : E.msg.c_str());
  return st;
}

vp_status check_mixed(vp_plan plan, double delta) {
  if (!(delta > 0 && delta < 1)) {
    vp::ls_set_error("delta must be in (0, 1)");
    return VP_ERR_INVALID_ARG;
  }
  if (!vp::plan_is_fp32(plan) && !vp::plan_is_fp64(plan)) {
    vp::ls_set_error("the plan's precision must be VP_FP32 or VP_FP64");
    return VP_ERR_INVALID_ARG;
  }
  return VP_OK;
}

vp_status check_dtype_prec(vp_plan plan, vp_dtype dtype) {
  const char* m = nullptr;
  if (dtype == VP_C64) {
    if (!vp::plan_is_fp32(plan)) m = "VP_C64 iterates with the FP32 apply: set the plan's precision to VP_FP32";
  } else if (dtype == VP_C128) {
    if (!vp::plan_is_fp64(plan)) m = "VP_C128 iterates with the FP64 apply: set the plan's precision to VP_FP64";
  } else {
    m = "dtype must be VP_C64 or VP_C128";
  }
  if (m) {
    vp::ls_set_error(m);
    return VP_ERR_INVALID_ARG;
  }
  return VP_OK;
}

}  // namespace

extern "C" {

vp_status vp_ls_bicgstab(vp_plan plan, const void* q, const void* u_inc, void* u, vp_dtype dtype, int form,
                         double tol, int maxit, double* history, vp_ls_stats* stats) {
  vp::NvtxRange range("vp_ls_bicgstab");
  long long n = 0;
  int d = 0;
  double k = 0.0;
  vp_status st = check_args(plan, false, q, nullptr, u_inc, u, form, tol, maxit, &n, &d, &k);
  if (st == VP_OK) st = check_dtype_prec(plan, dtype);
  if (st != VP_OK) return st;
  Err E;
  vp::DeviceGuard dg_(vp::plan_device(plan));
  const int f = form == VP_LS_DENSITY ? F_DENSITY : F_FIELD;
  st = dtype == VP_C64 ? run_one<float>(plan, f, q, nullptr, u_inc, u, k * k, d, n, tol, maxit, history, stats, E)
                       : run_one<double>(plan, f, q, nullptr, u_inc, u, k * k, d, n, tol, maxit, history, stats, E);
  return finish(st, E);
}

vp_status vp_ls_bicgstab_mixed(vp_plan plan, const double* q, const void* u_inc, void* u, int form, double tol,
                               double delta, int maxit, double* history, vp_ls_stats* stats) {
  long long n = 0;
  int d = 0;
  double k = 0.0;
  vp_status st = check_args(plan, false, q, nullptr, u_inc, u, form, tol, maxit, &n, &d, &k);
  if (st == VP_OK) st = check_mixed(plan, delta);
  if (st != VP_OK) return st;
  Err E;
  vp::DeviceGuard dg_(vp::plan_device(plan));
  const int f = form == VP_LS_DENSITY ? F_DENSITY : F_FIELD;
  st = run_mixed(plan, f, q, nullptr, u_inc, u, k * k, d, n, tol, delta, maxit, history, stats, E);
  return finish(st, E);
}

vp_status vp_pb_solve(vp_plan plan, const void* eps, const void* grad_eps, const void* rho, void* sigma,
                      vp_dtype dtype, double tol, int maxit, double* history, vp_ls_stats* stats) {
  long long n = 0;
  int d = 0;
  double k = 0.0;
  vp_status st = check_args(plan, true, eps, grad_eps, rho, sigma, 0, tol, maxit, &n, &d, &k);
  if (st == VP_OK) st = check_dtype_prec(plan, dtype);
  if (st == VP_OK) st = vp::plan_prepare_grad(plan);
  if (st != VP_OK) return st;
  Err E;
  vp::DeviceGuard dg_(vp::plan_device(plan));
  st = dtype == VP_C64 ? run_one<float>(plan, F_PB, eps, grad_eps, rho, sigma, 0.0, d, n, tol, maxit, history, stats, E)
                       : run_one<double>(plan, F_PB, eps, grad_eps, rho, sigma, 0.0, d, n, tol, maxit, history, stats, E);
  return finish(st, E);
}

vp_status vp_pb_gmres(vp_plan plan, const double* eps, const double* grad_eps, const void* rho, void* sigma,
                      double tol, int restart, int maxit, double* history, vp_ls_stats* stats) {
  long long n = 0;
  int d = 0;
  double k = 0.0;
  vp_status st = check_args(plan, true, eps, grad_eps, rho, sigma, 0, tol, maxit, &n, &d, &k);
  if (st == VP_OK) st = check_dtype_prec(plan, VP_C128);
  if (st == VP_OK && (restart < 1 || restart > kGmMaxRestart)) {
    vp::ls_set_error("restart must be in [1, 512]");
    st = VP_ERR_INVALID_ARG;
  }
  if (st == VP_OK) st = vp::plan_prepare_grad(plan);
  if (st != VP_OK) return st;
  Err E;
  vp::DeviceGuard dg_(vp::plan_device(plan));
  st = gmres_pb(plan, eps, grad_eps, static_cast<const double2*>(rho), static_cast<double2*>(sigma), d, n, tol,
                restart, maxit, history, stats, E);
  return finish(st, E);
}

vp_status vp_pb_solve_mixed(vp_plan plan, const double* eps, const double* grad_eps, const void* rho, void* sigma,
                            double tol, double delta, int maxit, double* history, vp_ls_stats* stats) {
  long long n = 0;
  int d = 0;
  double k = 0.0;
  vp_status st = check_args(plan, true, eps, grad_eps, rho, sigma, 0, tol, maxit, &n, &d, &k);
  if (st == VP_OK) st = check_mixed(plan, delta);
  if (st == VP_OK) st = vp::plan_prepare_grad(plan);
  if (st != VP_OK) return st;
  Err E;
  vp::DeviceGuard dg_(vp::plan_device(plan));
  st = run_mixed(plan, F_PB, eps, grad_eps, rho, sigma, 0.0, d, n, tol, delta, maxit, history, stats, E);
  return finish(st, E);
}

}  // extern "C"
