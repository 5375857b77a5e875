// ls.cu -- Lippmann-Schwinger scattering on the volume potential (Section 5.3 of
// Vico, Greengard & Ferrando) and its Krylov solver.
//
// The scattered field u of Delta u + k^2 (1 + q) u = -k^2 q u_inc solves the
// second-kind equation  A u = u - k^2 V[q u] = k^2 V[q u_inc] = b,  V the
// plan's volume potential (Green's function of -(Delta + k^2)).  The paper
// solves the dual density form with Bi-CGStab; this solver is right-
// preconditioned flexible GMRES(m) (Saad 1993) with classical Gram-Schmidt and
// one re-orthogonalisation (two batched dot kernels per iteration: FP32
// products and per-thread partial sums, FP64 sums across threads), complex64
// vectors and the FP32 apply.  The preconditioner is a
// caller function (e.g. the learned network, vp_unet_precond); when a
// preconditioned cycle fails to reduce the residual the solver falls back to
// plain GMRES.  Convergence is measured by the true residual of the FP64
// operator: ||b - A u|| / ||b|| with A and b evaluated in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <chrono>
#include <complex>
#include <string>
#include <vector>

#include "../../include/vp.h"
#include "vp_internal.cuh"

namespace {

using cd = std::complex<double>;

constexpr int kRedBlocks = 304;  // 2 x 152 SMs
constexpr int kDotBlocks = 1216; // 8 x 152 SMs: the batched dots need many loads in flight
constexpr int kRedThreads = 256;
constexpr int kMaxBasis = 64;    // restart length limit
constexpr int kStepWords = 2 * (kMaxBasis + 1) + 1;

__global__ void k_qmul(float2* __restrict__ out, const float* __restrict__ q, const float2* __restrict__ in, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float qi = q[i];
    const float2 v = in[i];
    out[i] = make_float2(qi * v.x, qi * v.y);
  }
}

__global__ void k_qmul64(double2* __restrict__ out, const float* __restrict__ q, const double2* __restrict__ in,
                         long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double qi = q[i];
    const double2 v = in[i];
    out[i] = make_double2(qi * v.x, qi * v.y);
  }
}

// out = u - k2 * vq (FP32), or b = k2 * vq when u == NULL
__global__ void k_combine(float2* __restrict__ out, const float2* __restrict__ u, const float2* __restrict__ vq,
                          float k2, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 w = vq[i];
    float2 r = make_float2(k2 * w.x, k2 * w.y);
    if (u) r = make_float2(u[i].x - r.x, u[i].y - r.y);
    out[i] = r;
  }
}

__global__ void k_combine64(double2* __restrict__ out, const double2* __restrict__ u, const double2* __restrict__ vq,
                            double k2, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 w = vq[i];
    double2 r = make_double2(k2 * w.x, k2 * w.y);
    if (u) r = make_double2(u[i].x - r.x, u[i].y - r.y);
    out[i] = r;
  }
}

// out = b - (u - k2 vq), FP64
__global__ void k_resid64(double2* __restrict__ out, const double2* __restrict__ b, const double2* __restrict__ u,
                          const double2* __restrict__ vq, double k2, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = make_double2(b[i].x - u[i].x + k2 * vq[i].x, b[i].y - u[i].y + k2 * vq[i].y);
}

__global__ void k_to64(double2* __restrict__ out, const float2* __restrict__ in, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = make_double2(in[i].x, in[i].y);
}

// partial[blk][j] = sum_i conj(V_j[i]) w[i] for j < m, per block.  Each thread
// sums its strided share (n / (304 x 256) terms, about 27 at N = 128) in FP32;
// the sums across threads and blocks are FP64.  (FP64 multiply-adds for every
// term would cost more than the apply on a GPU whose FP64 rate is 1/64 of FP32.)
__global__ void __launch_bounds__(kRedThreads) k_mdot(const float2* __restrict__ V, long long ldv, int m,
                                                      const float2* __restrict__ w, long long n, double2* __restrict__ partial) {
  __shared__ double2 red[kRedThreads / 32][kMaxBasis + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j0 = 0; j0 < m; j0 += 8) {
    float2 acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int mq = m - j0 < 8 ? m - j0 : 8;
    const float2* Vb = V + (long long)j0 * ldv;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // four independent elements per trip (more loads in flight), no bounds checks
    for (; i + 3 * stride < n; i += 4 * stride) {
      float2 wi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) wi[u] = w[i + u * stride];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q < mq) {
          const float2* Vq = Vb + (long long)q * ldv + i;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 v = Vq[u * stride];
            acc[q].x = fmaf(v.x, wi[u].x, fmaf(v.y, wi[u].y, acc[q].x));
            acc[q].y = fmaf(v.x, wi[u].y, fmaf(-v.y, wi[u].x, acc[q].y));
          }
        }
      }
    }
    for (; i < n; i += stride) {
      const float2 wi = w[i];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q < mq) {
          const float2 v = Vb[(long long)q * ldv + i];
          acc[q].x = fmaf(v.x, wi.x, fmaf(v.y, wi.y, acc[q].x));
          acc[q].y = fmaf(v.x, wi.y, fmaf(-v.y, wi.x, acc[q].y));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      double ax = acc[q].x, ay = acc[q].y;
      for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_down_sync(0xffffffffu, ax, o);
        ay += __shfl_down_sync(0xffffffffu, ay, o);
      }
      if (lane == 0 && j0 + q < m) red[warp][j0 + q] = make_double2(ax, ay);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int wv = 0; wv < kRedThreads / 32; ++wv) {
      s.x += red[wv][j].x;
      s.y += red[wv][j].y;
    }
    partial[(long long)blockIdx.x * m + j] = s;
  }
}

// partial[blk] = sum |x|^2 (FP64), complex64 or complex128 input
template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_norm2(const C* __restrict__ x, long long n, double* __restrict__ partial) {
  __shared__ double red[kRedThreads / 32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double a = x[i].x, b = x[i].y;
    acc += a * a + b * b;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int wv = 0; wv < kRedThreads / 32; ++wv) s += red[wv];
    partial[blockIdx.x] = s;
  }
}

// w -= sum_j h[j] V_j   (h on the device), FP32 arithmetic: w and V are FP32, and
// the second Gram-Schmidt pass removes what the first pass's rounding leaves
__global__ void k_mupdate(float2* __restrict__ w, const float2* __restrict__ V, long long ldv, int m,
                          const double2* __restrict__ h, long long n) {
  __shared__ float2 hs[kMaxBasis];
  for (int j = threadIdx.x; j < m; j += blockDim.x) hs[j] = make_float2((float)h[j].x, (float)h[j].y);
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float ax = w[i].x, ay = w[i].y;
    for (int j = 0; j < m; ++j) {
      const float2 v = V[(long long)j * ldv + i];
      ax = fmaf(-hs[j].x, v.x, fmaf(hs[j].y, v.y, ax));
      ay = fmaf(-hs[j].x, v.y, fmaf(-hs[j].y, v.x, ay));
    }
    w[i] = make_float2(ax, ay);
  }
}

// x += sum_j y[j] Z_j   (y on the device)
__global__ void k_mcombine(float2* __restrict__ x, const float2* __restrict__ Z, long long ldz, int m,
                           const double2* __restrict__ y, long long n) {
  __shared__ double2 ys[kMaxBasis];
  for (int j = threadIdx.x; j < m; j += blockDim.x) ys[j] = y[j];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double ax = x[i].x, ay = x[i].y;
    for (int j = 0; j < m; ++j) {
      const float2 z = Z[(long long)j * ldz + i];
      ax += ys[j].x * z.x - ys[j].y * z.y;
      ay += ys[j].x * z.y + ys[j].y * z.x;
    }
    x[i] = make_float2((float)ax, (float)ay);
  }
}

// out[j] = sum over the blocks' partial dots (FP64): one thread block per j
__global__ void __launch_bounds__(kRedThreads) k_reduce_dots(const double2* __restrict__ partial, int m, int blocks,
                                                             double2* __restrict__ out) {
  __shared__ double2 red[kRedThreads];
  const int j = blockIdx.x;
  double2 s = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < blocks; b += blockDim.x) {
    s.x += partial[(long long)b * m + j].x;
    s.y += partial[(long long)b * m + j].y;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x].x += red[threadIdx.x + o].x;
      red[threadIdx.x].y += red[threadIdx.x + o].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

// out = (||x||, 1/||x|| or 0) from the blocks' partial sums of |x|^2
__global__ void k_reduce_norm(const double* __restrict__ partial, int blocks, double2* __restrict__ out) {
  __shared__ double red[kRedThreads];
  double s = 0.0;
  for (int b = threadIdx.x; b < blocks; b += blockDim.x) s += partial[b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nrm = sqrt(red[0]);
    *out = make_double2(nrm, nrm > 0.0 ? 1.0 / nrm : 0.0);
  }
}

// x *= 1/||x|| with the norm on the device (left unchanged when it is zero)
__global__ void k_scale_by_norm(float2* __restrict__ x, const double2* __restrict__ nrm, long long n) {
  const double s = nrm->y;
  if (s == 0.0) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = make_float2((float)(x[i].x * s), (float)(x[i].y * s));
}

__global__ void k_scale_copy(float2* __restrict__ out, const float2* __restrict__ in, double s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = make_float2((float)(in[i].x * s), (float)(in[i].y * s));
}

__global__ void k_sub(float2* __restrict__ out, const float2* __restrict__ a, const float2* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = make_float2(a[i].x - b[i].x, a[i].y - b[i].y);
}

__global__ void k_pack_pair(float* __restrict__ x, float* __restrict__ t, const float2* __restrict__ r,
                            const float* __restrict__ q, const float2* __restrict__ ustar, const float2* __restrict__ us,
                            double s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] = (float)(r[i].x * s);
    x[n + i] = (float)(r[i].y * s);
    x[2 * n + i] = q[i];
    // target: the correction minus the residual (the network learns A^-1 - I)
    const float ex = ustar[i].x - (us ? us[i].x : 0.f) - r[i].x, ey = ustar[i].y - (us ? us[i].y : 0.f) - r[i].y;
    t[i] = (float)(ex * s);
    t[n + i] = (float)(ey * s);
  }
}

dim3 grid_for(long long n) {
  long long b = (n + 255) / 256;
  return dim3((unsigned)(b > 152 * 16 ? 152 * 16 : b));
}

struct Work {
  long long n = 0;
  int m = 0;
  float2* V = nullptr;  // (m+1) x n
  float2* Z = nullptr;  // m x n
  float2* t0 = nullptr;
  float2* t1 = nullptr;
  double2* d0 = nullptr;  // FP64 scratch for the true residual (4 x n)
  void* red = nullptr;    // reduction partials
  double2* hdev = nullptr;
  // one Arnoldi step's coefficients on the device and their pinned host copy:
  // [0, 65) first Gram-Schmidt pass, [65, 130) second pass, [130] (norm, 1/norm)
  double2* hstep = nullptr;
  double2* hstep_host = nullptr;
  std::string err;
  ~Work() {
    cudaFree(hstep);
    cudaFreeHost(hstep_host);
    cudaFree(V);
    cudaFree(Z);
    cudaFree(t0);
    cudaFree(t1);
    cudaFree(d0);
    cudaFree(red);
    cudaFree(hdev);
  }
};

vp_status cuda_err(Work& w, cudaError_t e, const char* what) {
  w.err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA;
}

#define LS_CUDA(w, call)                                  \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_err(w, e_, #call); \
  } while (0)

struct Ctx {
  vp_plan plan;
  const float* q;
  long long n;
  double k2;
  cudaStream_t s;
};

cudaStream_t get_stream(vp_plan p) { return vp::plan_stream(p); }

// out = A in (FP32): q*in -> V -> in - k^2 V[q in]
vp_status op32(const Ctx& c, Work& w, const float2* in, float2* out) {
  k_qmul<<<grid_for(c.n), 256, 0, c.s>>>(w.t0, c.q, in, c.n);
  vp_status st = vp_apply(c.plan, w.t0, w.t1, VP_C64);
  if (st != VP_OK) return st;
  k_combine<<<grid_for(c.n), 256, 0, c.s>>>(out, in, w.t1, (float)c.k2, c.n);
  LS_CUDA(w, cudaGetLastError());
  return VP_OK;
}

vp_status norm2(const Ctx& c, Work& w, const float2* x, double* out) {
  double* part = reinterpret_cast<double*>(w.red);
  k_norm2<float2><<<kRedBlocks, kRedThreads, 0, c.s>>>(x, c.n, part);
  std::vector<double> h(kRedBlocks);
  LS_CUDA(w, cudaMemcpyAsync(h.data(), part, kRedBlocks * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  LS_CUDA(w, cudaStreamSynchronize(c.s));
  double s = 0.0;
  for (double v : h) s += v;
  *out = sqrt(s);
  return VP_OK;
}

vp_status upload(const Ctx& c, Work& w, const cd* h, int m) {
  std::vector<double2> hh(m);
  for (int j = 0; j < m; ++j) hh[j] = make_double2(h[j].real(), h[j].imag());
  LS_CUDA(w, cudaMemcpyAsync(w.hdev, hh.data(), m * sizeof(double2), cudaMemcpyHostToDevice, c.s));
  LS_CUDA(w, cudaStreamSynchronize(c.s));  // hh is a stack buffer
  return VP_OK;
}

vp_status norm2_64(const Ctx& c, Work& w, const double2* x, double* out) {
  double* part = reinterpret_cast<double*>(w.red);
  k_norm2<double2><<<kRedBlocks, kRedThreads, 0, c.s>>>(x, c.n, part);
  std::vector<double> h(kRedBlocks);
  LS_CUDA(w, cudaMemcpyAsync(h.data(), part, kRedBlocks * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  LS_CUDA(w, cudaStreamSynchronize(c.s));
  double s = 0.0;
  for (double v : h) s += v;
  *out = sqrt(s);
  return VP_OK;
}

// True residual ||b - A u|| / ||b|| with the operator applied in FP64.  b is
// k^2 V[q u_inc] evaluated in FP64 when u_inc is given, else the FP32 b.
vp_status true_residual(const Ctx& c, Work& w, const float2* u, const float2* b32, const float2* uinc, double* out) {
  double2* U = w.d0;
  double2* B = w.d0 + c.n;
  double2* T = w.d0 + 2 * c.n;
  double2* Y = w.d0 + 3 * c.n;
  vp_precision prec;
  vp_status st = vp_plan_set_precision(c.plan, VP_FP64);
  if (st != VP_OK) return st;
  (void)prec;
  if (uinc) {
    k_to64<<<grid_for(c.n), 256, 0, c.s>>>(U, uinc, c.n);
    k_qmul64<<<grid_for(c.n), 256, 0, c.s>>>(T, c.q, U, c.n);
    st = vp_apply(c.plan, T, Y, VP_C128);
    if (st == VP_OK) k_combine64<<<grid_for(c.n), 256, 0, c.s>>>(B, nullptr, Y, c.k2, c.n);
  } else {
    k_to64<<<grid_for(c.n), 256, 0, c.s>>>(B, b32, c.n);
  }
  if (st == VP_OK) {
    k_to64<<<grid_for(c.n), 256, 0, c.s>>>(U, u, c.n);
    k_qmul64<<<grid_for(c.n), 256, 0, c.s>>>(T, c.q, U, c.n);
    st = vp_apply(c.plan, T, Y, VP_C128);
  }
  vp_plan_set_precision(c.plan, VP_FP32);
  if (st != VP_OK) return st;
  k_resid64<<<grid_for(c.n), 256, 0, c.s>>>(T, B, U, Y, c.k2, c.n);
  double rn = 0.0, bn = 0.0;
  if ((st = norm2_64(c, w, T, &rn)) != VP_OK) return st;
  if ((st = norm2_64(c, w, B, &bn)) != VP_OK) return st;
  *out = bn > 0 ? rn / bn : rn;
  return VP_OK;
}

// One FGMRES(m) cycle from x: returns the estimated relative residual.
vp_status fgmres_cycle(const Ctx& c, Work& w, const float2* b, float2* x, double bnorm, double tol, int max_inner,
                       vp_precond_fn M, void* Mctx, int* iters, int* matvecs, double* est) {
  const int m = w.m;
  const long long n = c.n;
  // r = b - A x  -> V_0
  vp_status st = op32(c, w, x, w.V);  // V_0 = A x
  if (st != VP_OK) return st;
  ++*matvecs;
  k_sub<<<grid_for(n), 256, 0, c.s>>>(w.V, b, w.V, n);
  double beta = 0.0;
  if ((st = norm2(c, w, w.V, &beta)) != VP_OK) return st;
  *est = beta / bnorm;
  if (!(beta > 0) || *est < tol || !std::isfinite(beta)) return VP_OK;
  k_scale_copy<<<grid_for(n), 256, 0, c.s>>>(w.V, w.V, 1.0 / beta, n);
  std::vector<cd> H((size_t)(m + 1) * m, cd(0)), cs(m), sn(m), g(m + 1, cd(0));
  g[0] = beta;
  int j = 0;
  for (; j < m && j < max_inner; ++j) {
    float2* vj = w.V + (long long)j * n;
    float2* zj = w.Z + (long long)j * n;
    float2* wv = w.V + (long long)(j + 1) * n;
    if (M) {
      st = M(Mctx, vj, zj, c.s);
      if (st != VP_OK) return st;
    } else {
      LS_CUDA(w, cudaMemcpyAsync(zj, vj, n * sizeof(float2), cudaMemcpyDeviceToDevice, c.s));
    }
    if ((st = op32(c, w, zj, wv)) != VP_OK) return st;
    ++*matvecs;
    // classical Gram-Schmidt, twice; coefficients and the norm stay on the
    // device, and one copy per step brings them to the host for H and Givens
    double2* h1d = w.hstep;
    double2* h2d = w.hstep + (kMaxBasis + 1);
    double2* nd = w.hstep + 2 * (kMaxBasis + 1);
    double2* part = reinterpret_cast<double2*>(w.red);
    k_mdot<<<kDotBlocks, kRedThreads, 0, c.s>>>(w.V, n, j + 1, wv, n, part);
    k_reduce_dots<<<j + 1, kRedThreads, 0, c.s>>>(part, j + 1, kDotBlocks, h1d);
    k_mupdate<<<grid_for(n), 256, 0, c.s>>>(wv, w.V, n, j + 1, h1d, n);
    k_mdot<<<kDotBlocks, kRedThreads, 0, c.s>>>(w.V, n, j + 1, wv, n, part);
    k_reduce_dots<<<j + 1, kRedThreads, 0, c.s>>>(part, j + 1, kDotBlocks, h2d);
    k_mupdate<<<grid_for(n), 256, 0, c.s>>>(wv, w.V, n, j + 1, h2d, n);
    k_norm2<float2><<<kRedBlocks, kRedThreads, 0, c.s>>>(wv, n, reinterpret_cast<double*>(w.red));
    k_reduce_norm<<<1, kRedThreads, 0, c.s>>>(reinterpret_cast<const double*>(w.red), kRedBlocks, nd);
    k_scale_by_norm<<<grid_for(n), 256, 0, c.s>>>(wv, nd, n);
    LS_CUDA(w, cudaGetLastError());
    LS_CUDA(w, cudaMemcpyAsync(w.hstep_host, w.hstep, kStepWords * sizeof(double2), cudaMemcpyDeviceToHost, c.s));
    LS_CUDA(w, cudaStreamSynchronize(c.s));
    const double2* hh = w.hstep_host;
    for (int i = 0; i <= j; ++i)
      H[(size_t)i * m + j] = cd(hh[i].x + hh[kMaxBasis + 1 + i].x, hh[i].y + hh[kMaxBasis + 1 + i].y);
    const double hn = hh[2 * (kMaxBasis + 1)].x;
    H[(size_t)(j + 1) * m + j] = hn;
    // Givens rotations on the new column
    for (int i = 0; i < j; ++i) {
      const cd a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
      H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
      H[(size_t)(i + 1) * m + j] = -std::conj(sn[i]) * a + cs[i] * bb;
    }
    const cd a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
    const double den = std::sqrt(std::norm(a) + std::norm(bb));
    if (den == 0.0) {
      cs[j] = 1.0;
      sn[j] = 0.0;
    } else if (std::abs(a) == 0.0) {
      cs[j] = 0.0;
      sn[j] = std::conj(bb) / std::abs(bb);
    } else {
      cs[j] = std::abs(a) / den;
      sn[j] = (a / std::abs(a)) * std::conj(bb) / den;
    }
    H[(size_t)j * m + j] = cs[j] * a + sn[j] * bb;
    H[(size_t)(j + 1) * m + j] = 0.0;
    g[j + 1] = -std::conj(sn[j]) * g[j];
    g[j] = cs[j] * g[j];
    ++*iters;
    *est = std::abs(g[j + 1]) / bnorm;
    if (*est < tol || !std::isfinite(*est)) {
      ++j;
      break;
    }
  }
  // y = H^{-1} g (upper triangular), x += Z y
  const int k = j;
  std::vector<cd> y(k);
  for (int i = k - 1; i >= 0; --i) {
    cd acc = g[i];
    for (int l = i + 1; l < k; ++l) acc -= H[(size_t)i * m + l] * y[l];
    y[i] = acc / H[(size_t)i * m + i];
  }
  if ((st = upload(c, w, y.data(), k)) != VP_OK) return st;
  k_mcombine<<<grid_for(n), 256, 0, c.s>>>(x, w.Z, n, k, w.hdev, n);
  LS_CUDA(w, cudaGetLastError());
  return VP_OK;
}

thread_local std::string g_ls_error;

vp_status ls_fail(vp_status st, const std::string& m) {
  vp::log_line(1, "solver", m);
  g_ls_error = m;
  return st;
}

vp_status check_plan(vp_plan plan, long long* n, double* k2) {
  int d = 0, N = 0;
  double k = 0.0;
  if (!plan) return ls_fail(VP_ERR_INVALID_ARG, "plan is NULL");
  vp_status st = vp_plan_info(plan, &d, &N, &k, nullptr, nullptr);
  if (st != VP_OK) return st;
  if (d != 3 || !(k > 0) || vp::plan_is_aniso(plan))
    return ls_fail(VP_ERR_INVALID_ARG, "the scattering solve needs a cubic 3D Helmholtz plan");
  if (!vp::plan_is_fp32(plan)) return ls_fail(VP_ERR_INVALID_ARG, "the scattering solve iterates in FP32: set the plan's precision to VP_FP32");
  *n = (long long)N * N * N;
  *k2 = k * k;
  return VP_OK;
}

// basis: the Arnoldi and preconditioned-direction vectors; fp64: the FP64
// scratch of the true residual (also used as plain scratch by the callers
// that take it)
vp_status alloc_work(Work& w, long long n, int m, bool basis, bool fp64 = true) {
  w.n = n;
  w.m = m;
  if (basis) {
    LS_CUDA(w, cudaMalloc(&w.V, (size_t)(m + 1) * n * sizeof(float2)));
    LS_CUDA(w, cudaMalloc(&w.Z, (size_t)m * n * sizeof(float2)));
  }
  LS_CUDA(w, cudaMalloc(&w.t0, n * sizeof(float2)));
  LS_CUDA(w, cudaMalloc(&w.t1, n * sizeof(float2)));
  if (fp64) LS_CUDA(w, cudaMalloc(&w.d0, 4 * n * sizeof(double2)));
  LS_CUDA(w, cudaMalloc(&w.red, (size_t)kDotBlocks * (kMaxBasis + 1) * sizeof(double2)));
  LS_CUDA(w, cudaMalloc(&w.hdev, (kMaxBasis + 1) * sizeof(double2)));
  if (basis) {
    LS_CUDA(w, cudaMalloc(&w.hstep, kStepWords * sizeof(double2)));
    LS_CUDA(w, cudaMallocHost(&w.hstep_host, kStepWords * sizeof(double2)));
  }
  return VP_OK;
}

}  // namespace

namespace vp {
void ls_set_error(const char* msg) {
  g_ls_error = msg;
  vp::log_line(1, "solver", g_ls_error);
}
}  // namespace vp

extern "C" {

vp_status vp_ls_operator(vp_plan plan, const float* q, const void* u, void* out) {
  long long n;
  double k2;
  vp_status st = check_plan(plan, &n, &k2);
  if (st != VP_OK) return st;
  vp::DeviceGuard dg_(vp::plan_device(plan));
  if (dg_.error() != cudaSuccess) return ls_fail(VP_ERR_CUDA, "cannot make the plan's device current");
  if (!q || !u || !out || u == out) return ls_fail(VP_ERR_INVALID_ARG, "q, u, out must be distinct device pointers");
  Work w;
  if ((st = alloc_work(w, n, 0, false, false)) != VP_OK) return ls_fail(st, w.err);
  Ctx c{plan, q, n, k2, get_stream(plan)};
  st = op32(c, w, reinterpret_cast<const float2*>(u), reinterpret_cast<float2*>(out));
  cudaStreamSynchronize(c.s);
  return st;
}

vp_status vp_ls_rhs(vp_plan plan, const float* q, const void* u_inc, void* b) {
  long long n;
  double k2;
  vp_status st = check_plan(plan, &n, &k2);
  if (st != VP_OK) return st;
  vp::DeviceGuard dg_(vp::plan_device(plan));
  if (dg_.error() != cudaSuccess) return ls_fail(VP_ERR_CUDA, "cannot make the plan's device current");
  if (!q || !u_inc || !b || u_inc == b) return ls_fail(VP_ERR_INVALID_ARG, "q, u_inc, b must be distinct device pointers");
  Work w;
  if ((st = alloc_work(w, n, 0, false, false)) != VP_OK) return ls_fail(st, w.err);
  Ctx c{plan, q, n, k2, get_stream(plan)};
  k_qmul<<<grid_for(n), 256, 0, c.s>>>(w.t0, q, reinterpret_cast<const float2*>(u_inc), n);
  st = vp_apply(plan, w.t0, w.t1, VP_C64);
  if (st != VP_OK) return st;
  k_combine<<<grid_for(n), 256, 0, c.s>>>(reinterpret_cast<float2*>(b), nullptr, w.t1, (float)k2, n);
  cudaStreamSynchronize(c.s);
  return VP_OK;
}

vp_status vp_ls_solve(vp_plan plan, const float* q, const void* b, const void* u_inc, void* u, const vp_ls_opts* opts,
                      vp_ls_stats* stats) {
  vp::NvtxRange range("vp_ls_solve");
  long long n;
  double k2;
  vp_status st = check_plan(plan, &n, &k2);
  if (st != VP_OK) return st;
  vp::DeviceGuard dg_(vp::plan_device(plan));
  if (dg_.error() != cudaSuccess) return ls_fail(VP_ERR_CUDA, "cannot make the plan's device current");
  if (!q || !b || !u || !opts) return ls_fail(VP_ERR_INVALID_ARG, "q, b, u and opts are required");
  if (opts->restart < 1 || opts->restart > kMaxBasis) return ls_fail(VP_ERR_INVALID_ARG, "restart must be in [1, 64]");
  if (!(opts->tol > 0) || opts->maxit < 1) return ls_fail(VP_ERR_INVALID_ARG, "tol > 0 and maxit >= 1 required");
  Work w;
  if ((st = alloc_work(w, n, opts->restart, true)) != VP_OK) return ls_fail(st, w.err);
  Ctx c{plan, q, n, k2, get_stream(plan)};
  float2* x = reinterpret_cast<float2*>(u);
  const float2* bb = reinterpret_cast<const float2*>(b);
  if (!opts->use_initial_guess) cudaMemsetAsync(x, 0, n * sizeof(float2), c.s);
  const auto t0 = std::chrono::steady_clock::now();
  double bnorm = 0.0;
  if ((st = norm2(c, w, bb, &bnorm)) != VP_OK) return ls_fail(st, w.err);
  int iters = 0, matvecs = 0, restarts = 0, fallback = 0;
  double est = 1.0, prev = 1e300;
  vp_precond_fn M = opts->precond;
  while (iters < opts->maxit) {
    const double before = est;
    st = fgmres_cycle(c, w, bb, x, bnorm > 0 ? bnorm : 1.0, opts->tol, opts->maxit - iters, M, opts->precond_ctx,
                      &iters, &matvecs, &est);
    if (st != VP_OK) return ls_fail(st, w.err.empty() ? "fgmres cycle failed" : w.err);
    ++restarts;
    if (est < opts->tol) break;
    // fallback: a preconditioned cycle that did not reduce the residual (or produced
    // a non-finite value) switches the rest of the solve to plain GMRES
    if (M && (!std::isfinite(est) || est > 0.9 * before)) {
      M = nullptr;
      fallback = 1;
      if (!std::isfinite(est)) cudaMemsetAsync(x, 0, n * sizeof(float2), c.s);
    }
    if (!M && est >= prev * 0.999999 && restarts > 3) break;  // stagnation of plain GMRES
    prev = est;
  }
  // final recurrence check from the true FP32 residual
  double tr = 0.0;
  st = true_residual(c, w, x, bb, reinterpret_cast<const float2*>(u_inc), &tr);
  if (st != VP_OK) return ls_fail(st, w.err.empty() ? "true residual failed" : w.err);
  const auto t1 = std::chrono::steady_clock::now();
  if (stats) {
    stats->iterations = iters;
    stats->matvecs = matvecs;
    stats->restarts = restarts;
    stats->used_fallback = fallback;
    stats->estimated_residual = est;
    stats->true_residual = tr;
    stats->seconds = std::chrono::duration<double>(t1 - t0).count();
  }
  return VP_OK;
}

vp_status vp_ls_training_pair(vp_plan plan, const float* q, const void* b, const void* u_s, const void* u_star,
                              float* x_out, float* t_out, double* rnorm) {
  long long n;
  double k2;
  vp_status st = check_plan(plan, &n, &k2);
  if (st != VP_OK) return st;
  vp::DeviceGuard dg_(vp::plan_device(plan));
  if (dg_.error() != cudaSuccess) return ls_fail(VP_ERR_CUDA, "cannot make the plan's device current");
  if (!q || !b || !u_star || !x_out || !t_out) return ls_fail(VP_ERR_INVALID_ARG, "NULL argument");
  Work w;
  if ((st = alloc_work(w, n, 0, false)) != VP_OK) return ls_fail(st, w.err);
  Ctx c{plan, q, n, k2, get_stream(plan)};
  float2* r = reinterpret_cast<float2*>(w.d0);  // FP64 scratch reused as two complex64 vectors
  float2* Au = r + n;
  if (u_s) {
    if ((st = op32(c, w, reinterpret_cast<const float2*>(u_s), Au)) != VP_OK) return st;
    k_sub<<<grid_for(n), 256, 0, c.s>>>(r, reinterpret_cast<const float2*>(b), Au, n);
  } else {
    cudaMemcpyAsync(r, b, n * sizeof(float2), cudaMemcpyDeviceToDevice, c.s);
  }
  double nr = 0.0;
  if ((st = norm2(c, w, r, &nr)) != VP_OK) return ls_fail(st, w.err);
  if (!(nr > 0)) return ls_fail(VP_ERR_NUMERICAL, "zero residual");
  k_pack_pair<<<grid_for(n), 256, 0, c.s>>>(x_out, t_out, r, q, reinterpret_cast<const float2*>(u_star),
                                            reinterpret_cast<const float2*>(u_s), sqrt((double)n) / nr, n);
  if (rnorm) *rnorm = nr;
  cudaStreamSynchronize(c.s);
  return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ERR_CUDA;
}

vp_status vp_ls_krylov_basis(vp_plan plan, const float* q, const void* b, int m, void* V, int* count) {
  long long n;
  double k2;
  vp_status st = check_plan(plan, &n, &k2);
  if (st != VP_OK) return st;
  vp::DeviceGuard dg_(vp::plan_device(plan));
  if (dg_.error() != cudaSuccess) return ls_fail(VP_ERR_CUDA, "cannot make the plan's device current");
  if (!q || !b || !V || !count) return ls_fail(VP_ERR_INVALID_ARG, "NULL argument");
  if (m < 1 || m > kMaxBasis) return ls_fail(VP_ERR_INVALID_ARG, "m must be in [1, 64]");
  Work w;
  if ((st = alloc_work(w, n, m, true)) != VP_OK) return ls_fail(st, w.err);
  Ctx c{plan, q, n, k2, get_stream(plan)};
  const float2* bb = reinterpret_cast<const float2*>(b);
  double bnorm = 0.0;
  if ((st = norm2(c, w, bb, &bnorm)) != VP_OK) return ls_fail(st, w.err);
  if (!(bnorm > 0)) return ls_fail(VP_ERR_NUMERICAL, "b is zero");
  // one plain cycle of m steps from x = 0 (the FP64 scratch is free here); tol 0 never stops it early
  float2* x = reinterpret_cast<float2*>(w.d0);
  LS_CUDA(w, cudaMemsetAsync(x, 0, n * sizeof(float2), c.s));
  int iters = 0, matvecs = 0;
  double est = 1.0;
  st = fgmres_cycle(c, w, bb, x, bnorm, 0.0, m, nullptr, nullptr, &iters, &matvecs, &est);
  if (st != VP_OK) return ls_fail(st, w.err.empty() ? "Arnoldi cycle failed" : w.err);
  *count = iters + 1;
  LS_CUDA(w, cudaMemcpyAsync(V, w.V, (size_t)(iters + 1) * n * sizeof(float2), cudaMemcpyDeviceToDevice, c.s));
  LS_CUDA(w, cudaStreamSynchronize(c.s));
  return VP_OK;
}

vp_status vp_ls_flexible_basis(vp_plan plan, const float* q, const void* b, int m, vp_precond_fn precond,
                               void* precond_ctx, void* Z, int* count) {
  long long n;
  double k2;
  vp_status st = check_plan(plan, &n, &k2);
  if (st != VP_OK) return st;
  vp::DeviceGuard dg_(vp::plan_device(plan));
  if (dg_.error() != cudaSuccess) return ls_fail(VP_ERR_CUDA, "cannot make the plan's device current");
  if (!q || !b || !Z || !count || !precond) return ls_fail(VP_ERR_INVALID_ARG, "NULL argument");
  if (m < 1 || m > kMaxBasis) return ls_fail(VP_ERR_INVALID_ARG, "m must be in [1, 64]");
  Work w;
  if ((st = alloc_work(w, n, m, true)) != VP_OK) return ls_fail(st, w.err);
  Ctx c{plan, q, n, k2, get_stream(plan)};
  const float2* bb = reinterpret_cast<const float2*>(b);
  double bnorm = 0.0;
  if ((st = norm2(c, w, bb, &bnorm)) != VP_OK) return ls_fail(st, w.err);
  if (!(bnorm > 0)) return ls_fail(VP_ERR_NUMERICAL, "b is zero");
  float2* x = reinterpret_cast<float2*>(w.d0);
  LS_CUDA(w, cudaMemsetAsync(x, 0, n * sizeof(float2), c.s));
  int iters = 0, matvecs = 0;
  double est = 1.0;
  st = fgmres_cycle(c, w, bb, x, bnorm, 0.0, m, precond, precond_ctx, &iters, &matvecs, &est);
  if (st != VP_OK) return ls_fail(st, w.err.empty() ? "flexible Arnoldi cycle failed" : w.err);
  *count = iters;
  LS_CUDA(w, cudaMemcpyAsync(Z, w.Z, (size_t)iters * n * sizeof(float2), cudaMemcpyDeviceToDevice, c.s));
  LS_CUDA(w, cudaStreamSynchronize(c.s));
  return VP_OK;
}

const char* vp_ls_last_error(void) { return g_ls_error.c_str(); }

}  // extern "C"
