// entries.cu -- Nystrom matrix entries on the fly (Section 4, the remark after
// the discrete convolution of Vico, Greengard & Ferrando).
//
// The precomputed kernel T is the matrix of a high-order Nystrom discretisation
// of the volume integral operator: phi_p = sum_{p'} T(p - p') f_{p'}, so the
// entry for target node p and source node p' is T(p - p') (the quadrature
// weight h^d included).  T is even in every axis (the potential) or odd in axis
// j (the derivative kernel T_j of Section 3); the plan holds it as its FP64
// octant n in [0, N]^d, so an entry is one gather:
//   T(n) = T_oct[|n_0|][|n_1|]([|n_2|])  (times sign(n_j) for T_j).
// Two entry points: a list of integer offsets, and a dense block of the matrix
// for lists of target and source nodes (flat C-order grid indices), the form a
// hierarchical or block preconditioner consumes.  Out-of-range offsets or
// indices write zero and raise a flag the host turns into VP_ERR_INVALID_ARG.
#include <cuda_runtime.h>

#include "../../include/vp.h"
#include "vp_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 152 * 32;

// T(n) for an offset n (|n_j| <= N), from the octant of the output's precision
// (D = d: the loops unroll and the index arrays stay in registers)
struct Dims {
  int N[3];  // points per axis (N_j; 1 beyond d)
};

template <typename C, int D>
__device__ __forceinline__ C gather(const C* __restrict__ oct, const Dims& g, int odd_axis, const int (&n)[3]) {
  long long idx = 0;
  int sgn = 1;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const int a = n[j] < 0 ? -n[j] : n[j];
    idx = idx * (g.N[j] + 1) + a;
    if (j == odd_axis) sgn = n[j] > 0 ? 1 : (n[j] < 0 ? -1 : 0);
  }
  C v = __ldg(oct + idx);
  if (sgn != 1) {
    v.x = sgn ? -v.x : 0;
    v.y = sgn ? -v.y : 0;
  }
  return v;
}

template <typename C, int D>
__global__ void __launch_bounds__(kThreads) k_entries(const C* __restrict__ oct, Dims g, int odd_axis,
                                                      const int* __restrict__ off, long long count, C* __restrict__ out,
                                                      int* __restrict__ bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    int n[3] = {0, 0, 0};
    bool ok = true;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      n[j] = off[i * D + j];
      ok = ok && n[j] >= -g.N[j] && n[j] <= g.N[j];
    }
    if (!ok) {
      out[i] = C{0, 0};
      atomicExch(bad, 1);
      continue;
    }
    out[i] = gather<C, D>(oct, g, odd_axis, n);
  }
}

// out[i][j] = T(p(rows[i]) - p(cols[j])), row-major.  A block owns a tile of
// kTileRows rows x kThreads columns: the rows are decoded once into shared
// memory, each thread decodes its column once and writes that column of every
// row of the tile (consecutive threads write consecutive entries of one row).
constexpr int kTileRows = 16;
constexpr int kGroup = 8;

template <typename C, int D>
__global__ void __launch_bounds__(kThreads, 4) k_block(const C* __restrict__ oct, Dims g, int odd_axis,
                                                    const long long* __restrict__ rows, long long nr,
                                                    const long long* __restrict__ cols, long long nc,
                                                    C* __restrict__ out, int* __restrict__ bad) {
  __shared__ int srow[kTileRows][3];
  __shared__ int sok[kTileRows];
  const long long U = D == 3 ? (long long)g.N[0] * g.N[1] * g.N[2] : (long long)g.N[0] * g.N[1];
  const long long c = blockIdx.x * (long long)kThreads + threadIdx.x;
  int q[3] = {0, 0, 0};
  bool cok = false;
  if (c < nc) {
    long long cc = cols[c];
    cok = cc >= 0 && cc < U;
    if (cok) {
#pragma unroll
      for (int a = D - 1; a >= 0; --a) {
        q[a] = (int)(cc % g.N[a]);
        cc /= g.N[a];
      }
    } else {
      atomicExch(bad, 1);
    }
  }
  for (long long r0 = blockIdx.y * (long long)kTileRows; r0 < nr; r0 += (long long)gridDim.y * kTileRows) {
    __syncthreads();  // the previous tile's rows are no longer read
    if (threadIdx.x < kTileRows) {
      const long long r = r0 + threadIdx.x;
      int ok = 0;
      if (r < nr) {
        long long rr = rows[r];
        ok = rr >= 0 && rr < U;
        if (ok) {
#pragma unroll
          for (int a = D - 1; a >= 0; --a) {
            srow[threadIdx.x][a] = (int)(rr % g.N[a]);
            rr /= g.N[a];
          }
        } else if (blockIdx.x == 0) {
          atomicExch(bad, 1);
        }
      }
      sok[threadIdx.x] = ok;
    }
    __syncthreads();
    if (c >= nc) continue;
    const int nrows = nr - r0 < kTileRows ? (int)(nr - r0) : kTileRows;
    // the gathers of kGroup rows in flight before their stores (kGroup bounds
    // the registers, and so keeps four CTAs resident per SM)
    for (int i0 = 0; i0 < kTileRows; i0 += kGroup) {
      C v[kGroup];
#pragma unroll
      for (int k = 0; k < kGroup; ++k) {
        const int i = i0 + k;
        v[k] = C{0, 0};
        if (i < nrows && cok && sok[i]) {
          int n[3] = {0, 0, 0};
#pragma unroll
          for (int a = 0; a < D; ++a) n[a] = srow[i][a] - q[a];
          v[k] = gather<C, D>(oct, g, odd_axis, n);
        }
      }
#pragma unroll
      for (int k = 0; k < kGroup; ++k)
        if (i0 + k < nrows) out[(r0 + i0 + k) * nc + c] = v[k];
    }
  }
}

unsigned grid_for(long long n) {
  const long long b = (n + kThreads - 1) / kThreads;
  return (unsigned)(b < 1 ? 1 : (b > kMaxBlocks ? kMaxBlocks : b));
}

bool is_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// common checks; *oct (FP64 or FP32 per dtype), *odd_axis, *dflag on success
vp_status prepare(vp_plan plan, int which, int axis, vp_dtype dtype, const void* const* ptrs, int nptr,
                  const void** oct, int* odd_axis, int** dflag) {
  if (!plan) return vp::entries_fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (dtype != VP_C64 && dtype != VP_C128)
    return vp::entries_fail(plan, VP_ERR_INVALID_ARG, "dtype must be VP_C64 or VP_C128");
  for (int i = 0; i < nptr; ++i) {
    if (!ptrs[i]) return vp::entries_fail(plan, VP_ERR_INVALID_ARG, "NULL array");
    if (!is_device(ptrs[i])) return vp::entries_fail(plan, VP_ERR_INVALID_ARG, "arrays must be device pointers");
  }
  vp_status st;
  if (dtype == VP_C128) {
    const double2* o = nullptr;
    st = vp::plan_kernel_octant(plan, which, axis, &o);
    *oct = o;
  } else {
    const float2* o = nullptr;
    st = vp::plan_kernel_octant32(plan, which, axis, &o);
    *oct = o;
  }
  if (st != VP_OK) return st;
  *odd_axis = which == VP_ARRAY_TJ ? axis : -1;
  *dflag = vp::plan_flag_word(plan);
  if (!*dflag) return vp::entries_fail(plan, VP_ERR_OOM, "flag word allocation failed");
  return VP_OK;
}

vp_status finish(vp_plan plan, int* dflag) {
  cudaStream_t s = vp::plan_stream(plan);
  int h = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, dflag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return vp::entries_fail(plan, VP_ERR_CUDA, cudaGetErrorString(e));
  if (h) return vp::entries_fail(plan, VP_ERR_INVALID_ARG, "an offset or grid index is out of range (zeros written)");
  return VP_OK;
}

}  // namespace

extern "C" {

vp_status vp_kernel_entries(vp_plan plan, int which, int axis, const int* offsets, long long count, void* out,
                            vp_dtype dtype) {
  if (count < 0) return vp::entries_fail(plan, VP_ERR_INVALID_ARG, "count < 0");
  if (count == 0) return VP_OK;
  if (!plan) return vp::entries_fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  vp::DeviceGuard dg_(vp::plan_device(plan));
  if (dg_.error() != cudaSuccess) return vp::entries_fail(plan, VP_ERR_CUDA, "cannot make the plan's device current");
  const void* ptrs[2] = {offsets, out};
  const void* oct = nullptr;
  int odd = -1, *flag = nullptr;
  vp_status st = prepare(plan, which, axis, dtype, ptrs, 2, &oct, &odd, &flag);
  if (st != VP_OK) return st;
  int d = 0, N = 0;
  vp_plan_info(plan, &d, &N, nullptr, nullptr, nullptr);
  Dims dims;
  vp::plan_dims(plan, dims.N);
  cudaStream_t s = vp::plan_stream(plan);
  cudaMemsetAsync(flag, 0, sizeof(int), s);
  const unsigned g = grid_for(count);
  if (dtype == VP_C128) {
    auto o = reinterpret_cast<double2*>(out);
    auto t = reinterpret_cast<const double2*>(oct);
    if (d == 3)
      k_entries<double2, 3><<<g, kThreads, 0, s>>>(t, dims, odd, offsets, count, o, flag);
    else
      k_entries<double2, 2><<<g, kThreads, 0, s>>>(t, dims, odd, offsets, count, o, flag);
  } else {
    auto o = reinterpret_cast<float2*>(out);
    auto t = reinterpret_cast<const float2*>(oct);
    if (d == 3)
      k_entries<float2, 3><<<g, kThreads, 0, s>>>(t, dims, odd, offsets, count, o, flag);
    else
      k_entries<float2, 2><<<g, kThreads, 0, s>>>(t, dims, odd, offsets, count, o, flag);
  }
  return finish(plan, flag);
}

vp_status vp_matrix_block(vp_plan plan, int which, int axis, const long long* rows, long long nrows,
                          const long long* cols, long long ncols, void* out, vp_dtype dtype) {
  if (nrows < 0 || ncols < 0) return vp::entries_fail(plan, VP_ERR_INVALID_ARG, "negative block size");
  if (nrows == 0 || ncols == 0) return VP_OK;
  if (!plan) return vp::entries_fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  vp::DeviceGuard dg_(vp::plan_device(plan));
  if (dg_.error() != cudaSuccess) return vp::entries_fail(plan, VP_ERR_CUDA, "cannot make the plan's device current");
  const void* ptrs[3] = {rows, cols, out};
  const void* oct = nullptr;
  int odd = -1, *flag = nullptr;
  vp_status st = prepare(plan, which, axis, dtype, ptrs, 3, &oct, &odd, &flag);
  if (st != VP_OK) return st;
  int d = 0, N = 0;
  vp_plan_info(plan, &d, &N, nullptr, nullptr, nullptr);
  Dims dims;
  vp::plan_dims(plan, dims.N);
  cudaStream_t s = vp::plan_stream(plan);
  cudaMemsetAsync(flag, 0, sizeof(int), s);
  const long long gx = (ncols + kThreads - 1) / kThreads;
  if (gx > 0x7fffffffLL) return vp::entries_fail(plan, VP_ERR_INVALID_ARG, "ncols too large");
  const long long row_tiles = (nrows + kTileRows - 1) / kTileRows;
  // about 32 resident blocks per SM in all; the row tiles are strided over grid.y
  long long gy = (152LL * 32 + gx - 1) / gx;
  gy = gy < 1 ? 1 : (gy > row_tiles ? row_tiles : (gy > 65535 ? 65535 : gy));
  const dim3 grid((unsigned)gx, (unsigned)gy);
  if (dtype == VP_C128) {
    auto o = reinterpret_cast<double2*>(out);
    auto t = reinterpret_cast<const double2*>(oct);
    if (d == 3)
      k_block<double2, 3><<<grid, kThreads, 0, s>>>(t, dims, odd, rows, nrows, cols, ncols, o, flag);
    else
      k_block<double2, 2><<<grid, kThreads, 0, s>>>(t, dims, odd, rows, nrows, cols, ncols, o, flag);
  } else {
    auto o = reinterpret_cast<float2*>(out);
    auto t = reinterpret_cast<const float2*>(oct);
    if (d == 3)
      k_block<float2, 3><<<grid, kThreads, 0, s>>>(t, dims, odd, rows, nrows, cols, ncols, o, flag);
    else
      k_block<float2, 2><<<grid, kThreads, 0, s>>>(t, dims, odd, rows, nrows, cols, ncols, o, flag);
  }
  return finish(plan, flag);
}

}  // extern "C"
