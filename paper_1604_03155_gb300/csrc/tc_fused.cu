// tc_fused.cu -- tensor-core form of the fused axis-0 pass of the 3D apply
// (precision variants VP_TC_BF16X2, VP_TC_FP16X2, VP_TC_BF16X3).
//
// The pass computes, for every pencil along axis 0 (Section 4: zero-pad to 2N,
// transform, multiply by the (2N)^d multiplier, inverse transform, crop):
//
//   y[j] = sum_m G[m] sum_{i<N} x[i] e^{-2 pi i i m/2N} e^{+2 pi i j m/2N},  j < N.
//
// Both 2N-point transforms are factored as 2N = 16 * N2 (Cooley-Tukey,
// four-step): with j = j1 + 16 j2 and m = k2 + N2 k1,
//
//   F1  Y[j1][k2]  = sum_{j2 < N2/2} x[j1 + 16 j2] w_N2^{j2 k2}      (pruned input)
//   T1  Y[j1][k2] *= w_2N^{j1 k2}
//   F3  X[k2 + N2 k1] = sum_{j1} Y[j1][k2] w_16^{j1 k1}
//       Z = X * G
//   I1  W[k2][j1]  = sum_{k1} Z[k2 + N2 k1] w_16^{-j1 k1}
//   T2  W[k2][j1] *= w_2N^{-j1 k2}
//   I3  y[j1 + 16 j2] = sum_{k2} W[k2][j1] w_N2^{-j2 k2},  j2 < N2/2  (cropped output)
//
// and each of F1, F3, I1, I3 runs over a tile of 8 pencils as one real GEMM
// (complex numbers expanded as [re | im] blocks) on the tensor cores:
// tcgen05.mma kind::f16, A (data) and B (DFT matrix) in shared memory, FP32
// accumulators in tensor memory, read back with tcgen05.ld.  FP32 values are
// split into 16-bit parts, x = x_0 + x_1 (+ x_2), and the partial products
// above the split's truncation level are accumulated:
//   BF16X2: a0 b0 + a1 b0 + a0 b1                      (~2^-16 relative)
//   FP16X2: the same in FP16 with a power-of-two scale per row or per pencil
//           (~2^-22 relative)
//   BF16X3: a0 b0 + a1 b0 + a0 b1 + a2 b0 + a1 b1 + a0 b2  (~2^-24 relative)
// The twiddles T1/T2 and the multiply by G run on the CUDA cores in FP32.
//
// Operand layouts are the tensor core's canonical no-swizzle layouts: 8x8
// "core matrices" of 16-bit elements (128 contiguous bytes).  A is K-major
// where one thread writes a whole row (F1, I1) and MN-major where the step
// transposes the data (F3, I3), so every shared-memory store is 16 bytes and
// none has a bank conflict (the F1 operand pads its row groups by 16 bytes).
// Row orders are chosen for the global accesses: the F1 input is loaded as 4
// pencils x 8 positions per warp, and the F3/I1 rows (k2/8)*64 + p*8 + k2%8
// give each warp 4 pencils x 8 frequencies, so the multiplier gathers read
// whole 32-byte sectors.  The output is staged in shared memory and written
// as 64-byte runs (8 pencils) per position.
//
// One CTA of 128 threads (one thread per tensor-memory lane) processes one
// tile at a time and loops over tiles (persistent grid, three CTAs per SM for
// the two-part splits).  Waits on MMA completion are bounded by a clock
// budget; a timeout sets the error word.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "vp_internal.cuh"

namespace vp {
namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_P = 8;             // pencils per tile
constexpr uint32_t TC_TMEM_COLS = 64;
constexpr long long TC_WAIT_CYCLES = 4000000000ll;  // ~2 s at 2 GHz

// Reading of the two stride fields of an MN-major shared-memory descriptor:
// leading byte offset = stride between core matrices along K, stride byte
// offset = stride along M/N (the same assignment as for K-major operands).
constexpr bool kMnLboIsK = true;

template <int SPLIT> struct SplitT;
template <> struct SplitT<0> {  // BF16 x 2
  static constexpr int parts = 2, products = 3;
  static constexpr bool bf16 = true, scaled = false;
};
template <> struct SplitT<1> {  // FP16 x 2, scaled
  static constexpr int parts = 2, products = 3;
  static constexpr bool bf16 = false, scaled = true;
};
template <> struct SplitT<2> {  // BF16 x 3
  static constexpr int parts = 3, products = 6;
  static constexpr bool bf16 = true, scaled = false;
};

// partial products (a part, b part), largest first
__host__ __device__ constexpr int prod_a(int i) { return i == 1 ? 1 : (i == 3 ? 2 : (i == 4 ? 1 : 0)); }
__host__ __device__ constexpr int prod_b(int i) { return i == 2 ? 1 : (i == 4 ? 1 : (i == 5 ? 2 : 0)); }

// Element offset of (row, k) in a K-major canonical operand with K columns.
__host__ __device__ __forceinline__ int ck(int r, int k, int K) {
  return ((r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}
// Element offset of (row, k) in a K-major operand whose groups of 8 rows are
// (K/8)*128 + pad bytes apart (pad = 16 spreads rows 16 apart over the banks).
__host__ __device__ __forceinline__ int ck_pad(int r, int k, int K, int pad) {
  return ((r >> 3) * ((K >> 3) * 128 + pad) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2) >> 1;
}
// Element offset of (m, k) in an MN-major canonical operand with M rows.
__host__ __device__ __forceinline__ int cmn(int m, int k, int M) {
  return ((k >> 3) * (M >> 3) + (m >> 3)) * 64 + (k & 7) * 8 + (m & 7);
}

template <int N2> struct TcGeom {
  static constexpr int n = 16 * N2;
  static constexpr int Nh = n / 2;
  static constexpr int bpart = 4 * N2 * N2 + 2048;  // B elements per part
  static constexpr int b_f1 = 0;                    // (2 N2) x N2
  static constexpr int b_f3 = 2 * N2 * N2;          // 32 x 32
  static constexpr int b_i1 = b_f3 + 1024;          // 32 x 32
  static constexpr int b_i3 = b_i1 + 1024;          // N2 x (2 N2)
  static constexpr int amax = 256 * N2;             // A elements per part
  static constexpr int m3 = 8 * N2;                 // rows of F3 and I1
  static constexpr int nh3 = m3 / 128;              // M=128 MMAs of F3 and I1
};

template <int N2, int SPLIT> constexpr size_t tc_smem_bytes() {
  using G = TcGeom<N2>;
  return (size_t)SplitT<SPLIT>::parts * (G::bpart + G::amax) * 2 + (size_t)32 * N2 * 8 + 768;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor core; no swizzle
  return d;
}

// instruction descriptor: D FP32, A/B BF16 or FP16, M = 128, N = ncols
__device__ __forceinline__ uint32_t idesc_f16(bool bf16, int ncols, bool a_mn) {
  const uint32_t ty = bf16 ? 1u : 0u;
  return (1u << 4) | (ty << 7) | (ty << 10) | (a_mn ? (1u << 15) : 0u) | ((uint32_t)(ncols >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > TC_WAIT_CYCLES) return false;
  }
}

__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Generic-proxy shared stores -> visible to the tensor core; then a CTA barrier.
__device__ __forceinline__ void sync_for_mma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
}

// tcgen05.ld of 8/16/32 consecutive FP32 columns of this warp's 32 lanes
// (lane = thread), waiting for completion inside the same asm statement.
__device__ __forceinline__ void tld8(uint32_t addr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(addr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tld16(uint32_t addr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tld32(uint32_t addr, float* v) {
  tld16(addr, v);
  tld16(addr + 16, v + 16);
}
template <int W> __device__ __forceinline__ void tldw(uint32_t addr, float* v) {
  if constexpr (W == 8) tld8(addr, v);
  else if constexpr (W == 16) tld16(addr, v);
  else tld32(addr, v);
}

// Power-of-two factor that brings mx into [2^13, 2^14) (1 for mx == 0).
__device__ __forceinline__ float pow2_scale(float mx) {
  const int e = (int)((__float_as_uint(mx) >> 23) & 0xFF) - 127;  // exponent of mx (normal numbers)
  int s = 13 - e;
  s = s < -126 ? -126 : (s > 127 ? 127 : s);
  return mx > 0.f ? __uint_as_float((uint32_t)(s + 127) << 23) : 1.f;
}

// Splits a pair (a, b) into 16-bit parts, two lanes per 32-bit word (a in the
// low half): part q of the pair is word[q].
template <int SPLIT> __device__ __forceinline__ void split_pair(float a, float b, uint32_t* word) {
  using S = SplitT<SPLIT>;
  if constexpr (S::bf16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const float ra = a - hf.x, rb = b - hf.y;
    const __nv_bfloat162 m = __floats2bfloat162_rn(ra, rb);
    word[0] = *reinterpret_cast<const uint32_t*>(&h);
    word[1] = *reinterpret_cast<const uint32_t*>(&m);
    if constexpr (S::parts == 3) {
      const float2 mf = __bfloat1622float2(m);
      const __nv_bfloat162 l = __floats2bfloat162_rn(ra - mf.x, rb - mf.y);
      word[2] = *reinterpret_cast<const uint32_t*>(&l);
    }
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    word[0] = *reinterpret_cast<const uint32_t*>(&h);
    word[1] = *reinterpret_cast<const uint32_t*>(&l);
  }
}

// Splits 8 values (times `scale`) and stores each part as one 16-byte row of
// a core matrix at element offset `off` of the part's A buffer.
template <int SPLIT>
__device__ __forceinline__ void store8(unsigned char* abase, int part_bytes, int off, const float* v, float scale) {
  constexpr int PARTS = SplitT<SPLIT>::parts;
  uint32_t w[PARTS][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    uint32_t pw[PARTS];
    split_pair<SPLIT>(v[2 * i] * scale, v[2 * i + 1] * scale, pw);
#pragma unroll
    for (int q = 0; q < PARTS; ++q) w[q][i] = pw[q];
  }
#pragma unroll
  for (int q = 0; q < PARTS; ++q)
    *reinterpret_cast<uint4*>(abase + q * part_bytes + off * 2) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

__device__ __forceinline__ int fold_m(int m, int n) { return m <= n - m ? m : n - m; }

// One GEMM step for 128 rows: all partial products and k-steps of 16.
//   a_addr   shared address of part 0 of A at the first of the 128 rows
//   a_mn     MN-major A (else K-major); m_total = rows of the whole MN-major operand
//   b_addr   shared address of part 0 of this step's B
template <int SPLIT, int K, int NC, int AMAX, int BPART, int KPAD = 0>
__device__ __forceinline__ void issue_step(uint32_t d_tmem, uint32_t a_addr, bool a_mn, int m_total, uint32_t b_addr) {
  using S = SplitT<SPLIT>;
  const uint32_t idesc = idesc_f16(S::bf16, NC, a_mn);
#pragma unroll
  for (int pr = 0; pr < S::products; ++pr) {
    const uint32_t ab = a_addr + prod_a(pr) * AMAX * 2;
    const uint32_t bb = b_addr + prod_b(pr) * BPART * 2;
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks) {
      uint64_t ad;
      if (a_mn) {
        const uint32_t kstride = (uint32_t)(m_total / 8) * 128;  // between core matrices along K
        ad = kMnLboIsK ? sdesc(ab + ks * 2 * kstride, kstride, 128) : sdesc(ab + ks * 2 * kstride, 128, kstride);
      } else {
        ad = sdesc(ab + ks * 256, 128, (K / 8) * 128 + KPAD);
      }
      const uint64_t bd = sdesc(bb + ks * 256, 128, (K / 8) * 128);
      mma_f16(d_tmem, ad, bd, idesc, (pr > 0 || ks > 0) ? 1u : 0u);
    }
  }
}

// Rows of F3 and I1: m = (k2/8)*64 + p*8 + k2%8.  Runs of 8 consecutive rows are
// 8 frequencies of one pencil (one 16-byte MN-major store by the writer of that
// pencil), and a warp's 32 rows are 4 pencils x 8 frequencies, so the multiplier
// gathers of a warp touch 8 full 32-byte sectors.
__device__ __forceinline__ int row3(int p, int k2) { return (k2 >> 3) * 64 + p * 8 + (k2 & 7); }
__device__ __forceinline__ int row3_p(int m) { return (m >> 3) & 7; }
__device__ __forceinline__ int row3_k2(int m) { return (m >> 6) * 8 + (m & 7); }

// Maximum over the 16 lanes of a half warp (lanes 0-15 or 16-31).
__device__ __forceinline__ float half_warp_max(float v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <int N2, int SPLIT>
__global__ void __launch_bounds__(TC_THREADS, SplitT<SPLIT>::parts == 3 ? 2 : 3)
    tc_fused_kernel(const TcFusedArgs a) {
  using S = SplitT<SPLIT>;
  using G = TcGeom<N2>;
  constexpr int n = G::n, Nh = G::Nh, PARTS = S::parts;
  constexpr int AB = G::amax * 2;  // bytes per A part
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sB = smem;
  unsigned char* sA = sB + PARTS * G::bpart * 2;
  float2* s_tw1 = reinterpret_cast<float2*>(sA + PARTS * AB);  // [k2][j1] = w_2N^{j1 k2}
  float2* s_tw2 = s_tw1 + 16 * N2;                             // [j1][k2] = w_2N^{-j1 k2}
  uint64_t* s_mbar = reinterpret_cast<uint64_t*>(s_tw2 + 16 * N2);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_mbar + 1);
  float* s_scale = reinterpret_cast<float*>(s_tmem + 1);  // [0, 8): F3 pencils, [8, 16): I3 pencils
  float* s_rs1 = s_scale + 16;                             // F1 row scales [128]
  unsigned* s_pmax = reinterpret_cast<unsigned*>(s_rs1 + 128);  // I3 pencil maxima (FP32 bits) [8]
  int* s_bad = reinterpret_cast<int*>(s_pmax + 8);
  float2* s_out = reinterpret_cast<float2*>(sA);  // [Nh][9] output staging, aliases A after I3

  const int tid = threadIdx.x, warp = tid >> 5;
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.bmat);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    for (int i = tid; i < PARTS * G::bpart * 2 / 16; i += TC_THREADS) dst[i] = src[i];
  }
  for (int i = tid; i < 16 * N2; i += TC_THREADS) {
    const int k2 = i >> 4, j1 = i & 15;
    const float2 w = a.tw[j1 * k2];  // j1 k2 < 2N
    s_tw1[k2 * 16 + j1] = w;
    s_tw2[j1 * N2 + k2] = make_float2(w.x, -w.y);
  }
  if (tid == 0) *s_bad = 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(s_mbar)));
  sync_for_mma();
  const uint32_t tmem = *s_tmem;
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t mbar = smem_u32(s_mbar);
  const uint32_t aB = smem_u32(sB), aA = smem_u32(sA);
  uint32_t phase = 0;
  bool ok = true;

  const long long ntiles = a.npencils / TC_P;
  const int np1 = Nh + 1;
  // this thread's F1 row r = p*16 + j1 (a half warp = one pencil)
  const int p1 = tid >> 4, j1t = tid & 15;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long pen0 = tile * TC_P;
    if constexpr (S::scaled) {
      if (tid < 8) s_pmax[tid] = 0u;  // read last by the previous tile before its final barrier
    }
    float rs_f1 = 1.f;  // row scales (FP16 split)
    float rs_i1[G::nh3];
#pragma unroll
    for (int h = 0; h < G::nh3; ++h) rs_i1[h] = 1.f;

    // ---- F1 operand: row r = p*16 + j1, K = N2 (re j2 | im j2), K-major with
    // padded row groups; loaded with 4 pencils x 8 positions per warp (coalesced) ----
    {
      const int pl = (tid & 3) + 4 * (tid >> 6), jl = (tid >> 2) & 15, rl = pl * 16 + jl;
      float xr[N2 / 2], xi[N2 / 2];
      const float2* src = a.in + pen0 + pl + (long long)jl * a.pitch_pos;
#pragma unroll
      for (int j2 = 0; j2 < N2 / 2; ++j2) {
        const float2 v = __ldg(src + (long long)(16 * j2) * a.pitch_pos);
        xr[j2] = v.x;
        xi[j2] = v.y;
      }
      if constexpr (S::scaled) {
        float mx = 0.f;
#pragma unroll
        for (int j2 = 0; j2 < N2 / 2; ++j2) mx = fmaxf(mx, fmaxf(fabsf(xr[j2]), fabsf(xi[j2])));
        rs_f1 = pow2_scale(mx);
        s_rs1[rl] = rs_f1;
      }
#pragma unroll
      for (int c = 0; c < N2 / 16; ++c) {
        store8<SPLIT>(sA, AB, ck_pad(rl, 8 * c, N2, 16), &xr[8 * c], rs_f1);
        store8<SPLIT>(sA, AB, ck_pad(rl, N2 / 2 + 8 * c, N2, 16), &xi[8 * c], rs_f1);
      }
    }
    sync_for_mma();
    if (tid == 0) {
      issue_step<SPLIT, N2, 2 * N2, G::amax, G::bpart, 16>(tmem, aA, false, 128, aB + G::b_f1 * 2);
      mma_commit(mbar);
    }
    ok = mbar_wait(mbar, phase) && ok;
    phase ^= 1;
    tc_after_sync();
    if constexpr (S::scaled) rs_f1 = s_rs1[tid];  // scale of the D row this thread reads

    // ---- T1 and the F3 operand: rows m = p*N2 + k2, K = 32 (re j1 | im j1), MN-major ----
    {
      float yr[N2], yi[N2];
      tldw<N2>(lane_base + 0, yr);
      tldw<N2>(lane_base + N2, yi);
      const float inv = 1.f / rs_f1;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const float2 w = s_tw1[k2 * 16 + j1t];
        const float r = yr[k2] * inv, i = yi[k2] * inv;
        yr[k2] = r * w.x - i * w.y;
        yi[k2] = r * w.y + i * w.x;
      }
      float sc = 1.f;
      if constexpr (S::scaled) {
        float mx = 0.f;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) mx = fmaxf(mx, fmaxf(fabsf(yr[k2]), fabsf(yi[k2])));
        sc = pow2_scale(half_warp_max(mx));  // the half warp holds the whole pencil
        if (j1t == 0) s_scale[p1] = sc;
      }
#pragma unroll
      for (int c = 0; c < N2 / 8; ++c) {
        const int m0 = row3(p1, 8 * c);
        store8<SPLIT>(sA, AB, cmn(m0, j1t, G::m3), &yr[8 * c], sc);
        store8<SPLIT>(sA, AB, cmn(m0, 16 + j1t, G::m3), &yi[8 * c], sc);
      }
    }
    sync_for_mma();
    if (tid == 0) {
#pragma unroll
      for (int h = 0; h < G::nh3; ++h)
        issue_step<SPLIT, 32, 32, G::amax, G::bpart>(tmem + 32 * h, aA + h * 2048, true, G::m3, aB + G::b_f3 * 2);
      mma_commit(mbar);
    }
    // multiplier gathers for this thread's rows (m = 128 h + tid) while the MMAs run
    float2 g[G::nh3][16];
#pragma unroll
    for (int h = 0; h < G::nh3; ++h) {
      const int r = 128 * h + tid, p = row3_p(r), k2 = row3_k2(r);
      const long long pen = pen0 + p;
      const int m1 = (int)(pen / n), m2 = (int)(pen % n);
      const long long rest = (long long)fold_m(m1, n) * np1 + fold_m(m2, n);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) {
        const int m0 = k2 + N2 * k1;
        g[h][k1] = __ldg(a.mult + (long long)fold_m(m0, n) * np1 * np1 + rest);
      }
    }
    ok = mbar_wait(mbar, phase) && ok;
    phase ^= 1;
    tc_after_sync();

    // ---- multiply and the I1 operand: rows m = p*N2 + k2, K = 32 (re k1 | im k1), K-major ----
#pragma unroll
    for (int h = 0; h < G::nh3; ++h) {
      const int r = 128 * h + tid, p = row3_p(r);
      float zr[16], zi[16];
      tld16(lane_base + 32 * h, zr);
      tld16(lane_base + 32 * h + 16, zi);
      float inv = 1.f;
      if constexpr (S::scaled) inv = 1.f / s_scale[p];
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) {
        const float xr = zr[k1] * inv, xi = zi[k1] * inv;
        zr[k1] = xr * g[h][k1].x - xi * g[h][k1].y;
        zi[k1] = xr * g[h][k1].y + xi * g[h][k1].x;
      }
      if constexpr (S::scaled) {
        float mx = 0.f;
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) mx = fmaxf(mx, fmaxf(fabsf(zr[k1]), fabsf(zi[k1])));
        rs_i1[h] = pow2_scale(mx);
      }
      store8<SPLIT>(sA, AB, ck(r, 0, 32), &zr[0], rs_i1[h]);
      store8<SPLIT>(sA, AB, ck(r, 8, 32), &zr[8], rs_i1[h]);
      store8<SPLIT>(sA, AB, ck(r, 16, 32), &zi[0], rs_i1[h]);
      store8<SPLIT>(sA, AB, ck(r, 24, 32), &zi[8], rs_i1[h]);
    }
    sync_for_mma();
    if (tid == 0) {
#pragma unroll
      for (int h = 0; h < G::nh3; ++h)
        issue_step<SPLIT, 32, 32, G::amax, G::bpart>(tmem + 32 * h, aA + h * 8192, false, G::m3, aB + G::b_i1 * 2);
      mma_commit(mbar);
    }
    ok = mbar_wait(mbar, phase) && ok;
    phase ^= 1;
    tc_after_sync();

    // ---- T2 and the I3 operand: rows m = p*16 + j1, K = 2 N2 (re k2 | im k2), MN-major ----
    {
      float wr[G::nh3][16], wi[G::nh3][16];
#pragma unroll
      for (int h = 0; h < G::nh3; ++h) {
        const int r = 128 * h + tid, k2 = row3_k2(r);
        tld16(lane_base + 32 * h, wr[h]);
        tld16(lane_base + 32 * h + 16, wi[h]);
        const float inv = 1.f / rs_i1[h];
#pragma unroll
        for (int j1 = 0; j1 < 16; ++j1) {
          const float2 w = s_tw2[j1 * N2 + k2];
          const float xr = wr[h][j1] * inv, xi = wi[h][j1] * inv;
          wr[h][j1] = xr * w.x - xi * w.y;
          wi[h][j1] = xr * w.y + xi * w.x;
        }
        if constexpr (S::scaled) {
          float mx = 0.f;
#pragma unroll
          for (int j1 = 0; j1 < 16; ++j1) mx = fmaxf(mx, fmaxf(fabsf(wr[h][j1]), fabsf(wi[h][j1])));
          atomicMax(&s_pmax[row3_p(r)], __float_as_uint(mx));  // a pencil's rows span warps
        }
      }
      if constexpr (S::scaled) __syncthreads();
#pragma unroll
      for (int h = 0; h < G::nh3; ++h) {
        const int r = 128 * h + tid, p = row3_p(r), k2 = row3_k2(r);
        float sc = 1.f;
        if constexpr (S::scaled) sc = pow2_scale(__uint_as_float(s_pmax[p]));
        store8<SPLIT>(sA, AB, cmn(p * 16, k2, 128), &wr[h][0], sc);
        store8<SPLIT>(sA, AB, cmn(p * 16 + 8, k2, 128), &wr[h][8], sc);
        store8<SPLIT>(sA, AB, cmn(p * 16, N2 + k2, 128), &wi[h][0], sc);
        store8<SPLIT>(sA, AB, cmn(p * 16 + 8, N2 + k2, 128), &wi[h][8], sc);
      }
    }
    sync_for_mma();
    if (tid == 0) {
      issue_step<SPLIT, 2 * N2, N2, G::amax, G::bpart>(tmem, aA, true, 128, aB + G::b_i3 * 2);
      mma_commit(mbar);
    }
    ok = mbar_wait(mbar, phase) && ok;
    phase ^= 1;
    tc_after_sync();

    // ---- output: row r = p*16 + j1 holds y[j1 + 16 j2], j2 < N2/2 ----
    {
      float yr[N2 / 2], yi[N2 / 2];
      tldw<N2 / 2>(lane_base + 0, yr);
      tldw<N2 / 2>(lane_base + N2 / 2, yi);
      float inv = 1.f;
      if constexpr (S::scaled) inv = 1.f / pow2_scale(__uint_as_float(s_pmax[p1]));
#pragma unroll
      for (int j2 = 0; j2 < N2 / 2; ++j2)
        s_out[(j1t + 16 * j2) * 9 + p1] = make_float2(yr[j2] * inv, yi[j2] * inv);
    }
    __syncthreads();
    for (int i = tid; i < Nh * TC_P; i += TC_THREADS) {
      const int pos = i >> 3, pp = i & 7;
      a.out[pen0 + pp + (long long)pos * a.pitch_pos] = s_out[pos * 9 + pp];
    }
    if (!ok) atomicOr(s_bad, 1);
    __syncthreads();
    if (*s_bad) break;
  }
  if (tid == 0 && *s_bad) atomicOr(a.err, 1);
  tc_before_sync();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// DFT matrices of the four steps, real-expanded, K-major canonical, split into
// 16-bit parts computed from the FP64 values.
template <int SPLIT> __device__ __forceinline__ void split_store64(uint16_t* out, int bpart, int off, double v) {
  using S = SplitT<SPLIT>;
  double r = v;
#pragma unroll
  for (int q = 0; q < S::parts; ++q) {
    uint16_t bits;
    double back;
    if constexpr (S::bf16) {
      const __nv_bfloat16 h = __double2bfloat16(r);
      bits = __bfloat16_as_ushort(h);
      back = (double)__bfloat162float(h);
    } else {
      const __half h = __double2half(r);
      bits = __half_as_ushort(h);
      back = (double)__half2float(h);
    }
    out[q * bpart + off] = bits;
    r -= back;
  }
}

template <int N2, int SPLIT> __global__ void tc_bmat_kernel(uint16_t* out) {
  using G = TcGeom<N2>;
  const int total = G::bpart;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int step, local, K, Kc, Nc, L, sgn, base;
    if (idx < G::b_f3) {
      step = 0, local = idx, K = N2, Kc = N2 / 2, Nc = N2, L = N2, sgn = -1, base = G::b_f1;
    } else if (idx < G::b_i1) {
      step = 1, local = idx - G::b_f3, K = 32, Kc = 16, Nc = 16, L = 16, sgn = -1, base = G::b_f3;
    } else if (idx < G::b_i3) {
      step = 2, local = idx - G::b_i1, K = 32, Kc = 16, Nc = 16, L = 16, sgn = 1, base = G::b_i1;
    } else {
      step = 3, local = idx - G::b_i3, K = 2 * N2, Kc = N2, Nc = N2 / 2, L = N2, sgn = 1, base = G::b_i3;
    }
    (void)step;
    const int nn = local / K, kk = local % K;
    const int c = nn % Nc, imo = nn / Nc, kc = kk % Kc, imi = kk / Kc;
    double s, co;
    sincospi((double)sgn * 2.0 * (double)((kc * c) % L) / (double)L, &s, &co);
    const double v = imo == 0 ? (imi == 0 ? co : -s) : (imi == 0 ? s : co);
    split_store64<SPLIT>(out, G::bpart, base + ck(nn, kk, K), v);
  }
}

template <int N2, int SPLIT> cudaError_t launch_tc_t(const TcFusedArgs& a, cudaStream_t s) {
  constexpr size_t smem = tc_smem_bytes<N2, SPLIT>();
  static int grid_cap[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (grid_cap[dev] == 0) {
    e = cudaFuncSetAttribute(tc_fused_kernel<N2, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // ask for the largest shared-memory carveout: without it the occupancy query
    // (and the launch) can settle on one CTA per SM
    e = cudaFuncSetAttribute(tc_fused_kernel<N2, SPLIT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int occ = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tc_fused_kernel<N2, SPLIT>, TC_THREADS, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // the residency the register file and shared memory allow (CTAs never wait
    // on one another, so a grid above the true residency only queues)
    cudaFuncAttributes fa;
    int smem_sm = 0;
    if (cudaFuncGetAttributes(&fa, tc_fused_kernel<N2, SPLIT>) == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess) {
      const int regs = ((fa.numRegs > 0 ? fa.numRegs : 1) + 7) / 8 * 8;
      const int by_regs = 65536 / (TC_THREADS * regs);
      const int by_smem = smem_sm / (int)(smem + 1024);
      const int est = by_regs < by_smem ? by_regs : by_smem;
      if (est > occ) occ = est;
    }
    // tensor memory: occ x 64 columns of 512 per SM
    if (occ > 8) occ = 8;
    grid_cap[dev] = (occ > 0 ? occ : 1) * sms;
  }
  const long long ntiles = a.npencils / TC_P;
  if (ntiles <= 0) return cudaSuccess;
  const long long grid = ntiles < grid_cap[dev] ? ntiles : grid_cap[dev];
  tc_fused_kernel<N2, SPLIT><<<(unsigned)grid, TC_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int N2> cudaError_t launch_tc_n(int split, const TcFusedArgs& a, cudaStream_t s) {
  switch (split) {
    case 0: return launch_tc_t<N2, 0>(a, s);
    case 1: return launch_tc_t<N2, 1>(a, s);
    case 2: return launch_tc_t<N2, 2>(a, s);
  }
  return cudaErrorInvalidValue;
}

template <int N2> cudaError_t build_bmat_n(int split, uint16_t* out, cudaStream_t s) {
  const int blocks = (TcGeom<N2>::bpart + 255) / 256;
  switch (split) {
    case 0: tc_bmat_kernel<N2, 0><<<blocks, 256, 0, s>>>(out); break;
    case 1: tc_bmat_kernel<N2, 1><<<blocks, 256, 0, s>>>(out); break;
    case 2: tc_bmat_kernel<N2, 2><<<blocks, 256, 0, s>>>(out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

bool tc_length_supported(int n) { return n == 256 || n == 512; }

size_t tc_bmat_bytes(int n, int split) {
  const int parts = split == 2 ? 3 : 2;
  if (n == 256) return (size_t)parts * TcGeom<16>::bpart * 2;
  if (n == 512) return (size_t)parts * TcGeom<32>::bpart * 2;
  return 0;
}

cudaError_t tc_build_bmat(int n, int split, uint16_t* out, cudaStream_t s) {
  if (n == 256) return build_bmat_n<16>(split, out, s);
  if (n == 512) return build_bmat_n<32>(split, out, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_tc_fused(int n, int split, const TcFusedArgs& a, cudaStream_t s) {
  if (a.npencils % TC_P != 0) return cudaErrorInvalidValue;
  if (n == 256) return launch_tc_n<16>(split, a, s);
  if (n == 512) return launch_tc_n<32>(split, a, s);
  return cudaErrorInvalidValue;
}

}  // namespace vp
