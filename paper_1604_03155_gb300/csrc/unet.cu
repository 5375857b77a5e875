// unet.cu -- the learned right preconditioner of the Lippmann-Schwinger solve
// (a project addition; the paper's solver is unpreconditioned Bi-CGStab).
//
// A 3-level 3D U-Net on one S^3 sample, channel-major [C][S][S][S]:
//   E1a conv 3->C, E1b conv C->C -> s1 (S); pool; E2a, E2b -> s2 (S/2); pool;
//   B1, B2 (S/4); up, concat [up, s2], D2a 2C->C, D2b (S/2); up, concat
//   [up, s1], D1a 2C->C, D1b C->2 (linear) (S).
// conv = 3x3x3 cross-correlation, zero padding 1, bias; leaky ReLU (slope 0.1
// by default, 1 = linear network) after every conv but the last; pool = 2x2x2 mean; up = nearest x2.
// Weights are kept in FP32 for the optimiser and rounded to bfloat16 for every
// forward and backward pass (BF16 weights; FP32 activations and gradients, split
// into two BF16 parts on the tensor cores).
//
// Kernels (all the network's own):
//  * convolutions: implicit GEMMs on the tensor cores (unet_tc.cu), BF16
//    weights times the two BF16 parts of the FP32 activations, FP32
//    accumulation.  Two input pointers model the skip concatenation without a
//    copy.
//  * input gradient: the same convolution with the layer's weights flipped in
//    k and transposed in (co, ci).
//  * weight gradients: implicit GEMMs on the tensor cores as well (unet_tc.cu),
//    both operands split into BF16 parts; each CTA writes one partial and
//    k_wreduce sums the partials in FP64 in a fixed order (deterministic).
//  * pool/up forward and backward, leaky-ReLU backward, MSE loss, Adam.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/vp.h"
#include "vp_internal.cuh"

namespace {

constexpr int kLayers = 10;

__device__ __forceinline__ float lrelu(float v, float slope) { return v > 0.f ? v : slope * v; }

// dw[co][ci][k] = sum_blocks part[blk][(ci*27+k)*CO + co]; db[co] likewise (FP64 sums)
__global__ void k_wreduce(const float* __restrict__ part, int nblk, int Ci, int CO, float* __restrict__ dw,
                          float* __restrict__ db) {
  const long long nw = (long long)Ci * 27 * CO;
  const long long stride = nw + CO;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < stride; i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(long long)b * stride + i];
    if (i < nw) {
      const long long co = i % CO, ck = i / CO;  // ck = ci*27 + k
      dw[co * (long long)Ci * 27 + ck] = (float)s;
    } else {
      db[i - nw] = (float)s;
    }
  }
}

// wf[ci][co][k'] = w[co][ci][26 - k']  (input-gradient weights)
__global__ void k_flip(const float* __restrict__ w, float* __restrict__ wf, int Co, int Ci) {
  const int n = Co * Ci * 27;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k = i % 27, co = (i / 27) % Co, ci = i / (27 * Co);
    wf[i] = w[((long long)co * Ci + ci) * 27 + (26 - k)];
  }
}

__global__ void k_pool(const float* __restrict__ x, float* __restrict__ y, int C, int S) {
  const int h = S / 2;
  const long long n = (long long)C * h * h * h;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / ((long long)h * h * h);
    const long long r = i % ((long long)h * h * h);
    const int z = (int)(r / (h * h)), yy = (int)((r / h) % h), xx = (int)(r % h);
    const float* src = x + c * (long long)S * S * S;
    float s = 0.f;
    for (int d = 0; d < 8; ++d)
      s += src[((long long)(2 * z + (d >> 2)) * S + 2 * yy + ((d >> 1) & 1)) * S + 2 * xx + (d & 1)];
    y[i] = 0.125f * s;
  }
}

// y (S^3 fine) = nearest-neighbour up of x (h^3 coarse), or its adjoint (sum into coarse) when back
__global__ void k_up(const float* __restrict__ x, float* __restrict__ y, int C, int S, int scale_back) {
  const int h = S / 2;
  if (!scale_back) {
    // S a multiple of 4: one float4 of an output row (x positions 4j .. 4j + 3)
    // from the float2 at 2j of the coarse row (both aligned); else one value.
    // Indices fit 32 bits (C S^3 < 2^31).
    const int q = S % 4 == 0 ? S / 4 : S, n = C * S * S * q;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const int r = i / q, j = i - r * q;  // r = (c S + z) S + yy
      const int yy = r % S, cz = r / S, z = cz % S, c = cz / S;
      const float* src = x + (((long long)c * h + z / 2) * h + yy / 2) * h;
      if (S % 4 == 0) {
        const float2 v = *reinterpret_cast<const float2*>(src + 2 * j);
        reinterpret_cast<float4*>(y)[i] = make_float4(v.x, v.x, v.y, v.y);
      } else {
        y[i] = src[j / 2];
      }
    }
  } else {
    // x fine (S^3) -> y coarse: y = sum of the 8 children (mean when scale_back == 2)
    const long long n = (long long)C * h * h * h;
    const float f = scale_back == 2 ? 0.125f : 1.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
      const long long c = i / ((long long)h * h * h), r = i % ((long long)h * h * h);
      const int z = (int)(r / (h * h)), yy = (int)((r / h) % h), xx = (int)(r % h);
      const float* src = x + c * (long long)S * S * S;
      float s = 0.f;
      for (int d = 0; d < 8; ++d)
        s += src[((long long)(2 * z + (d >> 2)) * S + 2 * yy + ((d >> 1) & 1)) * S + 2 * xx + (d & 1)];
      y[i] = f * s;
    }
  }
}

// pool adjoint: y_fine[...] (+)= x_coarse / 8
__global__ void k_pool_back(const float* __restrict__ dc, float* __restrict__ df, int C, int S, int accumulate) {
  const int h = S / 2;
  const long long n = (long long)C * S * S * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / ((long long)S * S * S), r = i % ((long long)S * S * S);
    const int z = (int)(r / (S * S)), yy = (int)((r / S) % S), xx = (int)(r % S);
    const float v = 0.125f * dc[c * (long long)h * h * h + ((long long)(z / 2) * h + yy / 2) * h + xx / 2];
    df[i] = accumulate ? df[i] + v : v;
  }
}

// dz = dy * lrelu'(y) (y is the activated output: the sign is preserved)
__global__ void k_lrelu_back(float* __restrict__ dz, const float* __restrict__ dy, const float* __restrict__ y, long long n,
                             float slope) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dz[i] = y[i] > 0.f ? dy[i] : slope * dy[i];
}


// MSE: dout = 2 (out - t)/n, partial sums of (out - t)^2 in FP64
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ t, float* __restrict__ dout, long long n,
                      double* __restrict__ part) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = out[i] - t[i];
    s += (double)d * d;
    dout[i] = 2.f * d / (float)n;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += red[i];
    part[blockIdx.x] = a;
  }
}

__device__ __forceinline__ float bf16_round(float v) {
  unsigned u = __float_as_uint(v);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  return __uint_as_float(u);
}

__global__ void k_round_bf16(const float* __restrict__ w, float* __restrict__ wq, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    wq[i] = bf16_round(w[i]);
}

__global__ void k_adam(float* __restrict__ w, float* __restrict__ wq, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wq[i] = bf16_round(wi);
  }
}

// network input [Re r, Im r, q] with r scaled by s
__global__ void k_pack_input(float* __restrict__ x, const float2* __restrict__ r, const float* __restrict__ q, double s,
                             long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] = (float)(r[i].x * s);
    x[n + i] = (float)(r[i].y * s);
    x[2 * n + i] = q[i];
  }
}

// z = r + s * o: the network output is the correction's deviation from r
__global__ void k_unpack_output(float2* __restrict__ z, const float2* __restrict__ r, const float* __restrict__ o,
                                double s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = make_float2((float)(r[i].x + o[i] * s), (float)(r[i].y + o[n + i] * s));
}

__global__ void __launch_bounds__(256) k_norm2c(const float2* __restrict__ x, long long n, double* __restrict__ part) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += (double)x[i].x * x[i].x + (double)x[i].y * x[i].y;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < 8; ++i) a += red[i];
    part[blockIdx.x] = a;
  }
}

dim3 g1(long long n) {
  long long b = (n + 255) / 256;
  return dim3((unsigned)(b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

struct vp_unet_s {
  int S = 0, C = 0;
  float slope = 0.1f;  // leaky-ReLU slope; 1 makes the network linear
  int device = 0;
  cudaStream_t stream = nullptr;
  int co[kLayers], ci[kLayers];
  long long woff[kLayers], boff[kLayers];
  long long nparams = 0;
  float *w = nullptr, *wq = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *wf = nullptr;
  long long step = 0;
  // activations (S: s1-level, S2 = S/2, S4 = S/4)
  float *x0 = nullptr, *a1 = nullptr, *s1 = nullptr, *p1 = nullptr, *a3 = nullptr, *s2 = nullptr, *p2 = nullptr,
        *a5 = nullptr, *a6 = nullptr, *u2 = nullptr, *a7 = nullptr, *a8 = nullptr, *u1 = nullptr, *a9 = nullptr,
        *out = nullptr;
  // gradient scratch
  float *gA = nullptr, *gB = nullptr, *gC = nullptr, *gS1 = nullptr, *gS2 = nullptr, *dout = nullptr;
  float* part = nullptr;
  int part_blocks = 0;
  double* red = nullptr;
  int* err = nullptr;        // device error word: a convolution's bounded wait timed out
  long long wait_cycles = 4000000000ll;  // budget of each bounded wait (about 2 s)
  int withhold = 0;                      // test hook: the convolutions issue no MMAs
  const float* q = nullptr;  // bound contrast for the preconditioner
  std::vector<void*> allocs;
  std::string last_error;
};

namespace {

vp_status ufail(vp_unet u, vp_status st, const std::string& m) {
  vp::log_line(1, "network", m);
  if (u) u->last_error = m;
  return st;
}

template <typename T> cudaError_t ualloc(vp_unet u, T** p, long long count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess) u->allocs.push_back(*p);
  return e;
}

cudaError_t conv(vp_unet u, const float* x1, int c1, const float* x2, int c2, const float* w, const float* b, float* y,
                 int CO, int S, int act, cudaStream_t s) {
  vp::unet_tc::ConvArgs a;
  a.x1 = x1;
  a.c1 = c1;
  a.x2 = x2;
  a.c2 = c2;
  a.w = w;
  a.bias = b;
  a.y = y;
  a.co = CO;
  a.S = S;
  a.act = act;
  a.slope = u->slope;
  a.err = u->err;
  a.wait_cycles = u->wait_cycles;
  a.withhold = u->withhold;
  return vp::unet_tc::conv3d(a, s);
}

cudaError_t wgrad(vp_unet u, int layer, const float* x1, int c1, const float* x2, int c2, const float* dz, int S,
                  cudaStream_t s) {
  const int CO = u->co[layer], Ci = u->ci[layer];
  const long long rows = vp::unet_tc::wgrad_rows(S);
  const int nb = rows < u->part_blocks ? (int)rows : u->part_blocks;
  vp::unet_tc::WgradArgs a;
  a.x1 = x1;
  a.c1 = c1;
  a.x2 = x2;
  a.c2 = c2;
  a.dy = dz;
  a.co = CO;
  a.part = u->part;
  a.nblk = nb;
  a.S = S;
  a.err = u->err;
  a.wait_cycles = u->wait_cycles;
  a.withhold = u->withhold;
  cudaError_t e = vp::unet_tc::wgrad3d(a, s);
  if (e != cudaSuccess) return e;
  k_wreduce<<<g1((long long)Ci * 27 * CO + CO), 256, 0, s>>>(u->part, nb, Ci, CO, u->g + u->woff[layer],
                                                             u->g + u->boff[layer]);
  return cudaGetLastError();
}

// input gradient of a layer: conv of dz with the flipped, transposed weights
cudaError_t dgrad(vp_unet u, int layer, const float* dz, float* dx, int S, cudaStream_t s) {
  const int CO = u->co[layer], Ci = u->ci[layer];
  k_flip<<<g1((long long)CO * Ci * 27), 256, 0, s>>>(u->wq + u->woff[layer], u->wf, CO, Ci);
  return conv(u, dz, CO, nullptr, 0, u->wf, nullptr, dx, Ci, S, 0, s);
}

cudaError_t forward(vp_unet u, const float* in, cudaStream_t s) {
  const int S = u->S, C = u->C, S2 = S / 2, S4 = S / 4;
  const long long n2 = (long long)C * S2 * S2 * S2;
  cudaError_t e;
  auto L = [&](int i) { return u->wq + u->woff[i]; };
  auto B = [&](int i) { return u->wq + u->boff[i]; };
  if ((e = conv(u, in, 3, nullptr, 0, L(0), B(0), u->a1, C, S, 1, s)) != cudaSuccess) return e;
  if ((e = conv(u, u->a1, C, nullptr, 0, L(1), B(1), u->s1, C, S, 1, s)) != cudaSuccess) return e;
  k_pool<<<g1(n2), 256, 0, s>>>(u->s1, u->p1, C, S);
  if ((e = conv(u, u->p1, C, nullptr, 0, L(2), B(2), u->a3, C, S2, 1, s)) != cudaSuccess) return e;
  if ((e = conv(u, u->a3, C, nullptr, 0, L(3), B(3), u->s2, C, S2, 1, s)) != cudaSuccess) return e;
  k_pool<<<g1((long long)C * S4 * S4 * S4), 256, 0, s>>>(u->s2, u->p2, C, S2);
  if ((e = conv(u, u->p2, C, nullptr, 0, L(4), B(4), u->a5, C, S4, 1, s)) != cudaSuccess) return e;
  if ((e = conv(u, u->a5, C, nullptr, 0, L(5), B(5), u->a6, C, S4, 1, s)) != cudaSuccess) return e;
  k_up<<<g1(n2), 256, 0, s>>>(u->a6, u->u2, C, S2, 0);
  if ((e = conv(u, u->u2, C, u->s2, C, L(6), B(6), u->a7, C, S2, 1, s)) != cudaSuccess) return e;
  if ((e = conv(u, u->a7, C, nullptr, 0, L(7), B(7), u->a8, C, S2, 1, s)) != cudaSuccess) return e;
  k_up<<<g1((long long)C * S * S * S), 256, 0, s>>>(u->a8, u->u1, C, S, 0);
  if ((e = conv(u, u->u1, C, u->s1, C, L(8), B(8), u->a9, C, S, 1, s)) != cudaSuccess) return e;
  if ((e = conv(u, u->a9, C, nullptr, 0, L(9), B(9), u->out, 2, S, 0, s)) != cudaSuccess) return e;
  return cudaGetLastError();
}

// gradients of the loss for dL/dout = u->dout (stored in u->g)
cudaError_t backward(vp_unet u, const float* in, cudaStream_t s) {
  const int S = u->S, C = u->C, S2 = S / 2, S4 = S / 4;
  const long long n1 = (long long)C * S * S * S, n2 = (long long)C * S2 * S2 * S2, n4 = (long long)C * S4 * S4 * S4;
  cudaError_t e;
  // D1b (linear): input a9
  if ((e = wgrad(u, 9, u->a9, C, nullptr, 0, u->dout, S, s)) != cudaSuccess) return e;
  if ((e = dgrad(u, 9, u->dout, u->gA, S, s)) != cudaSuccess) return e;  // d a9
  // D1a: input concat[u1, s1], output a9
  k_lrelu_back<<<g1(n1), 256, 0, s>>>(u->gA, u->gA, u->a9, n1, u->slope);
  if ((e = wgrad(u, 8, u->u1, C, u->s1, C, u->gA, S, s)) != cudaSuccess) return e;
  if ((e = dgrad(u, 8, u->gA, u->gB, S, s)) != cudaSuccess) return e;  // [d u1, d s1] (2C)
  cudaMemcpyAsync(u->gS1, u->gB + n1, n1 * sizeof(float), cudaMemcpyDeviceToDevice, s);
  k_up<<<g1(n2), 256, 0, s>>>(u->gB, u->gC, C, S, 1);  // d a8 = up^T d u1
  // D2b: input a7, output a8
  k_lrelu_back<<<g1(n2), 256, 0, s>>>(u->gC, u->gC, u->a8, n2, u->slope);
  if ((e = wgrad(u, 7, u->a7, C, nullptr, 0, u->gC, S2, s)) != cudaSuccess) return e;
  if ((e = dgrad(u, 7, u->gC, u->gA, S2, s)) != cudaSuccess) return e;  // d a7
  // D2a: input concat[u2, s2], output a7
  k_lrelu_back<<<g1(n2), 256, 0, s>>>(u->gA, u->gA, u->a7, n2, u->slope);
  if ((e = wgrad(u, 6, u->u2, C, u->s2, C, u->gA, S2, s)) != cudaSuccess) return e;
  if ((e = dgrad(u, 6, u->gA, u->gB, S2, s)) != cudaSuccess) return e;  // [d u2, d s2]
  cudaMemcpyAsync(u->gS2, u->gB + n2, n2 * sizeof(float), cudaMemcpyDeviceToDevice, s);
  k_up<<<g1(n4), 256, 0, s>>>(u->gB, u->gC, C, S2, 1);  // d a6
  // B2: input a5, output a6
  k_lrelu_back<<<g1(n4), 256, 0, s>>>(u->gC, u->gC, u->a6, n4, u->slope);
  if ((e = wgrad(u, 5, u->a5, C, nullptr, 0, u->gC, S4, s)) != cudaSuccess) return e;
  if ((e = dgrad(u, 5, u->gC, u->gA, S4, s)) != cudaSuccess) return e;  // d a5
  // B1: input p2, output a5
  k_lrelu_back<<<g1(n4), 256, 0, s>>>(u->gA, u->gA, u->a5, n4, u->slope);
  if ((e = wgrad(u, 4, u->p2, C, nullptr, 0, u->gA, S4, s)) != cudaSuccess) return e;
  if ((e = dgrad(u, 4, u->gA, u->gC, S4, s)) != cudaSuccess) return e;  // d p2
  k_pool_back<<<g1(n2), 256, 0, s>>>(u->gC, u->gS2, C, S2, 1);        // d s2 += pool^T d p2
  // E2b: input a3, output s2
  k_lrelu_back<<<g1(n2), 256, 0, s>>>(u->gS2, u->gS2, u->s2, n2, u->slope);
  if ((e = wgrad(u, 3, u->a3, C, nullptr, 0, u->gS2, S2, s)) != cudaSuccess) return e;
  if ((e = dgrad(u, 3, u->gS2, u->gA, S2, s)) != cudaSuccess) return e;  // d a3
  // E2a: input p1, output a3
  k_lrelu_back<<<g1(n2), 256, 0, s>>>(u->gA, u->gA, u->a3, n2, u->slope);
  if ((e = wgrad(u, 2, u->p1, C, nullptr, 0, u->gA, S2, s)) != cudaSuccess) return e;
  if ((e = dgrad(u, 2, u->gA, u->gC, S2, s)) != cudaSuccess) return e;  // d p1
  k_pool_back<<<g1(n1), 256, 0, s>>>(u->gC, u->gS1, C, S, 1);          // d s1 += pool^T d p1
  // E1b: input a1, output s1
  k_lrelu_back<<<g1(n1), 256, 0, s>>>(u->gS1, u->gS1, u->s1, n1, u->slope);
  if ((e = wgrad(u, 1, u->a1, C, nullptr, 0, u->gS1, S, s)) != cudaSuccess) return e;
  if ((e = dgrad(u, 1, u->gS1, u->gA, S, s)) != cudaSuccess) return e;  // d a1
  // E1a: input x0, output a1
  k_lrelu_back<<<g1(n1), 256, 0, s>>>(u->gA, u->gA, u->a1, n1, u->slope);
  if ((e = wgrad(u, 0, in, 3, nullptr, 0, u->gA, S, s)) != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

extern "C" {

vp_status vp_unet_create(vp_unet* out, int S, int C) {
  if (!out) return VP_ERR_INVALID_ARG;
  *out = nullptr;
  if (S < 4 || S % 4 || C != 16) return VP_ERR_INVALID_ARG;
  vp_unet u = new vp_unet_s();
  u->S = S;
  u->C = C;
  cudaGetDevice(&u->device);
  const int shapes[kLayers][2] = {{C, 3}, {C, C}, {C, C}, {C, C}, {C, C}, {C, C}, {C, 2 * C}, {C, C}, {C, 2 * C}, {2, C}};
  long long off = 0;
  for (int i = 0; i < kLayers; ++i) {
    u->co[i] = shapes[i][0];
    u->ci[i] = shapes[i][1];
    u->woff[i] = off;
    off += (long long)u->co[i] * u->ci[i] * 27;
    u->boff[i] = off;
    off += u->co[i];
  }
  u->nparams = off;
  const long long S1 = (long long)S * S * S, S2 = S1 / 8, S4 = S1 / 64;
  cudaError_t e = cudaSuccess;
  auto A = [&](float** p, long long n) {
    if (e == cudaSuccess) e = ualloc(u, p, n);
  };
  A(&u->w, off);
  A(&u->wq, off);
  A(&u->g, off);
  A(&u->m, off);
  A(&u->v, off);
  A(&u->wf, (long long)2 * C * C * 27);
  A(&u->x0, 3 * S1);
  A(&u->a1, C * S1);
  A(&u->s1, C * S1);
  A(&u->p1, C * S2);
  A(&u->a3, C * S2);
  A(&u->s2, C * S2);
  A(&u->p2, C * S4);
  A(&u->a5, C * S4);
  A(&u->a6, C * S4);
  A(&u->u2, C * S2);
  A(&u->a7, C * S2);
  A(&u->a8, C * S2);
  A(&u->u1, C * S1);
  A(&u->a9, C * S1);
  A(&u->out, 2 * S1);
  A(&u->gA, 2 * C * S1);
  A(&u->gB, 2 * C * S1);
  A(&u->gC, 2 * C * S1);
  A(&u->gS1, C * S1);
  A(&u->gS2, C * S2);
  A(&u->dout, 2 * S1);
  u->part_blocks = 2 * 152;
  A(&u->part, (long long)u->part_blocks * (2 * C * 27 * C + C));
  if (e == cudaSuccess) e = ualloc(u, &u->red, 2048);
  if (e == cudaSuccess) e = ualloc(u, &u->err, 1);
  if (e == cudaSuccess) e = cudaMemset(u->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(u->m, 0, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(u->v, 0, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(u->w, 0, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(u->wq, 0, off * sizeof(float));
  if (e != cudaSuccess) {
    vp_unet_destroy(u);
    return e == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA;
  }
  if (const double secs = vp::env_timeout_seconds()) vp_unet_set_timeout(u, secs);
  *out = u;
  return VP_OK;
}

vp_status vp_unet_param_count(vp_unet u, size_t* count) {
  if (!u || !count) return VP_ERR_INVALID_ARG;
  *count = (size_t)u->nparams;
  return VP_OK;
}

vp_status vp_unet_set_stream(vp_unet u, void* stream) {
  if (!u) return VP_ERR_INVALID_ARG;
  u->stream = reinterpret_cast<cudaStream_t>(stream);
  return VP_OK;
}

vp_status vp_unet_set_weights(vp_unet u, const float* host, size_t count) {
  if (!u || !host || count != (size_t)u->nparams) return ufail(u, VP_ERR_INVALID_ARG, "weight count mismatch");
  vp::DeviceGuard dg_(u->device);
  if (cudaMemcpy(u->w, host, count * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return VP_ERR_CUDA;
  k_round_bf16<<<g1(u->nparams), 256, 0, u->stream>>>(u->w, u->wq, u->nparams);
  cudaMemsetAsync(u->m, 0, count * sizeof(float), u->stream);
  cudaMemsetAsync(u->v, 0, count * sizeof(float), u->stream);
  u->step = 0;
  return cudaStreamSynchronize(u->stream) == cudaSuccess ? VP_OK : VP_ERR_CUDA;
}

vp_status vp_unet_get_weights(vp_unet u, int which, float* host, size_t count) {
  if (!u || !host || count != (size_t)u->nparams || which < 0 || which > 2) return VP_ERR_INVALID_ARG;
  vp::DeviceGuard dg_(u->device);
  cudaStreamSynchronize(u->stream);
  const float* src = which == 0 ? u->w : (which == 1 ? u->wq : u->g);
  return cudaMemcpy(host, src, count * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? VP_OK : VP_ERR_CUDA;
}

vp_status vp_unet_forward(vp_unet u, const float* in, float* out) {
  vp::NvtxRange range("vp_unet_forward");
  if (!u || !in || !out) return VP_ERR_INVALID_ARG;
  vp::DeviceGuard dg_(u->device);
  cudaError_t e = forward(u, in, u->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, u->out, 2LL * u->S * u->S * u->S * sizeof(float), cudaMemcpyDeviceToDevice, u->stream);
  return e == cudaSuccess ? VP_OK : ufail(u, VP_ERR_CUDA, cudaGetErrorString(e));
}

vp_status vp_unet_loss_grad(vp_unet u, const float* in, const float* target, double* loss) {
  if (!u || !in || !target) return VP_ERR_INVALID_ARG;
  vp::DeviceGuard dg_(u->device);
  cudaStream_t s = u->stream;
  cudaError_t e = forward(u, in, s);
  const long long n = 2LL * u->S * u->S * u->S;
  const int nb = 256;
  if (e == cudaSuccess) {
    k_mse<<<nb, 256, 0, s>>>(u->out, target, u->dout, n, u->red);
    e = backward(u, in, s);
  }
  if (e != cudaSuccess) return ufail(u, VP_ERR_CUDA, cudaGetErrorString(e));
  if (loss) {
    std::vector<double> h(nb);
    if (cudaMemcpyAsync(h.data(), u->red, nb * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return VP_ERR_CUDA;
    int herr = 0;
    if (cudaMemcpy(&herr, u->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return VP_ERR_CUDA;
    if (herr) {  // reported once, then cleared
      if (cudaMemset(u->err, 0, sizeof(int)) != cudaSuccess) return VP_ERR_CUDA;
      return ufail(u, VP_ERR_TIMEOUT, "a tensor-core convolution timed out waiting for its MMAs");
    }
    double acc = 0.0;
    for (double v : h) acc += v;
    *loss = acc / (double)n;
  }
  return VP_OK;
}

vp_status vp_unet_get_adam(vp_unet u, float* m, float* v, size_t count, long long* step) {
  if (!u || !m || !v || !step || count != (size_t)u->nparams)
    return ufail(u, VP_ERR_INVALID_ARG, "Adam state: NULL argument or count mismatch");
  vp::DeviceGuard dg_(u->device);
  if (cudaStreamSynchronize(u->stream) != cudaSuccess ||
      cudaMemcpy(m, u->m, count * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(v, u->v, count * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return ufail(u, VP_ERR_CUDA, "Adam state: copy failed");
  *step = u->step;
  return VP_OK;
}
vp_status vp_unet_set_adam(vp_unet u, const float* m, const float* v, size_t count, long long step) {
  if (!u || !m || !v || count != (size_t)u->nparams || step < 0)
    return ufail(u, VP_ERR_INVALID_ARG, "Adam state: NULL argument, count mismatch or negative step");
  vp::DeviceGuard dg_(u->device);
  if (cudaStreamSynchronize(u->stream) != cudaSuccess ||
      cudaMemcpy(u->m, m, count * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(u->v, v, count * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return ufail(u, VP_ERR_CUDA, "Adam state: copy failed");
  u->step = step;
  return VP_OK;
}
vp_status vp_unet_adam_step(vp_unet u, double lr) {
  if (!u || !(lr > 0)) return VP_ERR_INVALID_ARG;
  vp::DeviceGuard dg_(u->device);
  const float b1 = 0.9f, b2 = 0.999f;
  ++u->step;
  const float c1 = 1.f - powf(b1, (float)u->step), c2 = 1.f - powf(b2, (float)u->step);
  k_adam<<<g1(u->nparams), 256, 0, u->stream>>>(u->w, u->wq, u->g, u->m, u->v, u->nparams, (float)lr, b1, b2, 1e-8f,
                                                 c1, c2);
  return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ERR_CUDA;
}

vp_status vp_unet_set_slope(vp_unet u, double slope) {
  if (!u || !(slope >= 0.0) || slope > 1.0) return VP_ERR_INVALID_ARG;
  u->slope = (float)slope;
  return VP_OK;
}

vp_status vp_unet_bind(vp_unet u, const float* q) {
  if (!u || !q) return VP_ERR_INVALID_ARG;
  u->q = q;
  return VP_OK;
}

// Preconditioner z = r + (||r||/sqrt(n)) net(sqrt(n) r/||r||, q), a vp_precond_fn:
// inputs scaled to unit RMS, the network learns A^-1 - I.
vp_status vp_unet_precond(void* ctx, const void* r, void* z, void* stream) {
  vp_unet u = reinterpret_cast<vp_unet>(ctx);
  if (!u || !u->q || !r || !z) return VP_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long n = (long long)u->S * u->S * u->S;
  const float2* rr = reinterpret_cast<const float2*>(r);
  k_norm2c<<<256, 256, 0, s>>>(rr, n, u->red);
  std::vector<double> h(256);
  int herr = 0;
  if (cudaMemcpyAsync(h.data(), u->red, 256 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&herr, u->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return VP_ERR_CUDA;
  if (herr) {  // reported once, then cleared
    if (cudaMemsetAsync(u->err, 0, sizeof(int), s) != cudaSuccess) return VP_ERR_CUDA;
    return ufail(u, VP_ERR_TIMEOUT, "a tensor-core convolution timed out waiting for its MMAs");
  }
  double nr = 0.0;
  for (double v : h) nr += v;
  nr = sqrt(nr);
  if (!(nr > 0)) {
    cudaMemsetAsync(z, 0, n * sizeof(float2), s);
    return VP_OK;
  }
  const double rms = sqrt((double)n) / nr;
  k_pack_input<<<g1(n), 256, 0, s>>>(u->x0, rr, u->q, rms, n);
  cudaError_t e = forward(u, u->x0, s);
  if (e != cudaSuccess) return VP_ERR_CUDA;
  k_unpack_output<<<g1(n), 256, 0, s>>>(reinterpret_cast<float2*>(z), rr, u->out, 1.0 / rms, n);
  return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ERR_CUDA;
}

vp_status vp_unet_status(vp_unet u) {
  if (!u) return VP_ERR_INVALID_ARG;
  vp::DeviceGuard dg_(u->device);
  int herr = 0;
  if (cudaMemcpyAsync(&herr, u->err, sizeof(int), cudaMemcpyDeviceToHost, u->stream) != cudaSuccess ||
      cudaStreamSynchronize(u->stream) != cudaSuccess)
    return ufail(u, VP_ERR_CUDA, "stream synchronisation failed");
  if (herr) {  // reported once, then cleared
    if (cudaMemsetAsync(u->err, 0, sizeof(int), u->stream) != cudaSuccess ||
        cudaStreamSynchronize(u->stream) != cudaSuccess)
      return ufail(u, VP_ERR_CUDA, "clearing the error word failed");
    return ufail(u, VP_ERR_TIMEOUT, "a tensor-core convolution timed out waiting for its MMAs");
  }
  return VP_OK;
}

vp_status vp_unet_set_timeout(vp_unet u, double seconds) {
  if (!u || !(seconds > 0)) return VP_ERR_INVALID_ARG;
  vp::DeviceGuard dg_(u->device);
  int khz = 0;
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, u->device) != cudaSuccess || khz <= 0) khz = 2000000;
  const double cycles = seconds * khz * 1e3;
  u->wait_cycles = cycles > 4e18 ? 4000000000000000000ll : (long long)cycles;
  return VP_OK;
}

vp_status vp_unet_withhold(vp_unet u, int on) {
  if (!u) return VP_ERR_INVALID_ARG;
  u->withhold = on ? 1 : 0;
  return VP_OK;
}

const char* vp_unet_last_error(vp_unet u) { return u ? u->last_error.c_str() : ""; }

vp_status vp_unet_destroy(vp_unet u) {
  if (!u) return VP_OK;
  vp::DeviceGuard dg_(u->device);
  if (u->stream) cudaStreamSynchronize(u->stream);
  for (void* p : u->allocs) cudaFree(p);
  delete u;
  return VP_OK;
}

}  // extern "C"
