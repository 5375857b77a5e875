// fourstep.cuh -- FP32 pencil passes of the apply as four-step FFTs
// (Section 4: zero-pad f to (2N)^d, FFT, multiply by the kernel spectrum,
// inverse FFT, crop; here one pass transforms one axis of a batch of pencils).
//
// A pencil of length n = P Q is held by Q threads, P complex values each, in
// registers.  With j = t + Q q (t < Q, q < P) and k = k1 + P k2 (k1 < P, k2 < Q):
//
//   X[k1 + P k2] = sum_t w_Q^(t k2) w_n^(t k1) sum_q x[t + Q q] w_P^(q k1)
//
// Step A: thread t takes the P-point DFT of x[t + Q q] over q, multiplies by
// the twiddles w_n^(t k1) and writes the P results to shared memory.  Step B:
// thread u reads the Q values of columns k1 = u + Q c (c < P/Q) and takes their
// Q-point DFTs over t, giving X[u + Q c + P k2].  The inverse transform is the
// transpose: Q-point inverse DFTs over k2 (step B'), one exchange, the
// conjugate twiddles and P-point inverse DFTs over k1 (step A').  So a pencil
// costs one shared-memory exchange per transform, and the twiddles w_n^(t k1)
// come from a (Q x P) table in shared memory built once per CTA.
//
// Pruning: the forward input is f zero-padded from n/2 to n, i.e. q < P/2, and
// the P-point DFT of a half-zero input is two P/2-point DFTs (of x and of
// x w_P^q); the inverse output is cropped to n/2, i.e. q < P/2, and the
// cropped P-point inverse DFT is two P/2-point inverse DFTs and one
// combination per kept output.  The fused pass runs step A, step B, the
// multiply by the kernel spectrum, step B' and step A' on one pencil in
// registers: the forward's output layout is the inverse's input layout.
//
// Memory pipeline: persistent CTAs walk the tiles (W pencils each) with a grid
// stride; each tile's input is staged into shared memory by 16-byte cp.async
// copies NSTG - 1 tiles ahead, and the fused pass stages the tile's rows of
// the multiplier octant at the start of the tile (8-byte copies), so they
// arrive while steps A and B run.
#pragma once

#include <cuda.h>

#include "pencil_fft.cuh"

namespace vp {
namespace fs {

// n = P x Q with P the values per thread: Q threads per pencil.
__host__ __device__ constexpr int fs_P(int n) {
  return n == 64 ? 8 : n == 128 ? 16 : n == 256 ? 16 : n == 512 ? 32 : n == 1024 ? 32 : 0;
}
__host__ __device__ constexpr bool fs_length(int n) { return fs_P(n) > 0; }

// cos(pi m / 16) and sin(pi m / 16) for any integer m (period 32)
__host__ __device__ constexpr double cos_pi16_base(int m) {  // m in [0, 8]
  return m == 0   ? 1.0
         : m == 1 ? 0.98078528040323044913
         : m == 2 ? 0.92387953251128675613
         : m == 3 ? 0.83146961230254523708
         : m == 4 ? 0.70710678118654752440
         : m == 5 ? 0.55557023301960222474
         : m == 6 ? 0.38268343236508977173
         : m == 7 ? 0.19509032201612826785
                  : 0.0;
}
__host__ __device__ constexpr double cos_pi16(int m) {
  return (m = ((m % 32) + 32) % 32, m <= 8 ? cos_pi16_base(m)
                                    : m <= 16 ? -cos_pi16_base(16 - m)
                                    : m <= 24 ? -cos_pi16_base(m - 16)
                                              : cos_pi16_base(32 - m));
}
__host__ __device__ constexpr double sin_pi16(int m) { return cos_pi16(8 - m); }

// x * exp(-i pi m/16) (INV: exp(+i pi m/16)); m is a compile-time constant
// after unrolling, so the trivial angles cost nothing.
template <bool INV>
__device__ __forceinline__ float2 rot_pi16(float2 x, int m) {
  m = ((m % 32) + 32) % 32;
  if (m == 0) return x;
  if (m == 16) return float2{-x.x, -x.y};
  if (m == 8) return mul_mi<INV>(x);
  if (m == 24) return mul_mi<!INV>(x);
  const float c = (float)cos_pi16(m), s = (float)sin_pi16(m);
  return INV ? float2{c * x.x - s * x.y, c * x.y + s * x.x} : float2{c * x.x + s * x.y, c * x.y - s * x.x};
}

// v[k1] *= w_n^(t k1) (CONJ: its conjugate) for k1 = 1..P-1, the twiddles
// read two at a time from the thread's row of the table.
template <int P, bool CONJ>
__device__ __forceinline__ void apply_twiddles(float2* v, const float4* row) {
#pragma unroll
  for (int h = 0; h < P / 2; ++h) {
    const float4 p = row[h];
    if (h > 0) v[2 * h] = CONJ ? cconjmul(v[2 * h], float2{p.x, p.y}) : cmul(v[2 * h], float2{p.x, p.y});
    v[2 * h + 1] = CONJ ? cconjmul(v[2 * h + 1], float2{p.z, p.w}) : cmul(v[2 * h + 1], float2{p.z, p.w});
  }
}

// P-point forward DFT of v[0, P/2) (v[P/2, P) is zero and not read), natural
// order out in v[0, P): X[2m] = DFT_{P/2}(x)[m], X[2m+1] = DFT_{P/2}(x w_P^j)[m].
template <int P>
__device__ __forceinline__ void dft_fwd_halfzero(float2* v) {
  constexpr int H = P / 2;
  float2 e[H], o[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = v[j];
    o[j] = rot_pi16<false>(v[j], (32 / P) * j);
  }
  Dft<H, false>::run(e);
  Dft<H, false>::run(o);
#pragma unroll
  for (int m = 0; m < H; ++m) {
    v[2 * m] = e[m];
    v[2 * m + 1] = o[m];
  }
}

// P-point inverse DFT of v[0, P), only outputs q < P/2, into v[0, P/2):
// y[q] = E[q] + w_P^(-q) O[q] with E, O the P/2-point inverse DFTs of the even
// and odd samples.
template <int P>
__device__ __forceinline__ void idft_cropped(float2* v) {
  constexpr int H = P / 2;
  float2 e[H], o[H];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    e[m] = v[2 * m];
    o[m] = v[2 * m + 1];
  }
  Dft<H, true>::run(e);
  Dft<H, true>::run(o);
#pragma unroll
  for (int q = 0; q < H; ++q) v[q] = cadd(e[q], rot_pi16<true>(o[q], (32 / P) * q));
}

// ---------------------------------------------------------------------------
// launch configuration and shared-memory layout of a pass
//   W pencils per tile, Q threads each; NSTG-deep input staging ring.
// Exchange element (k1, t, w):
//   strided pencils (lanes run over w): k1 RP + t W + w, RP = Q W + (W mod 16),
//     so that the step-B reads (lanes over w and u) of 32/W column rows fall
//     in distinct bank halves/quarters;
//   contiguous pencils (lanes run over t): w WP + k1 (Q + 1) + t, an odd
//     column pitch for the step-B reads and WP = Q (mod 16) between pencils.
// Twiddle table: (t, k1) at t (P + 2) + k1, read in pairs of k1.
// Staging slot: strided [pos][w] (the rows of W pencils as in global memory),
//   contiguous [w][pos] with pitch NIN (+ 8 when Q < 16).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr size_t round128(size_t b) { return (b + 127) / 128 * 128; }

template <int n, bool CONTIG, int MODE, int W_, int NSTG_, bool ALIAS_ = false>
struct Cfg {
  static constexpr int n_ = n;
  static constexpr bool CONTIG_ = CONTIG;
  static constexpr int P = fs_P(n);
  static constexpr int Q = n / P;
  static constexpr int CC = P / Q;  // columns per thread in step B
  static constexpr int W = W_;
  static constexpr int NSTG = NSTG_;
  static constexpr int threads = W * Q;
  static constexpr int NIN = stage_in_len(n, MODE);  // n/2 forward and fused, n inverse
  static constexpr bool FUSED = (MODE == MODE_FUSED1);
  // ALIAS: the exchange runs in the current tile's staging slot (free once the
  // tile's input is in registers), in XR rounds of P/XR columns k1, laid out
  // (k1r, t, w) -> k1r Q W + ((t W + w) xor ((k1r & SWZ) W)) (no padding; the
  // xor sends the step-B reads of neighbouring columns to other bank groups).
  static constexpr bool ALIAS = ALIAS_;
  static constexpr int XR = (MODE == MODE_INV) ? 1 : P / Q;
  static constexpr int SWZ = W >= 16 ? 0 : 16 / W - 1;
  static constexpr int TP = P + 2;  // even: entries (k1, k1 + 1) are one 16-byte load
  static constexpr int RP = Q * W + (W % 16);
  static constexpr int QP = Q + 1;
  static constexpr int WP0 = P * QP;
  static constexpr int WP = Q >= 16 ? WP0 : WP0 + (((Q - WP0) % 16) + 16) % 16;
  static constexpr int XELEMS = CONTIG ? W * WP : P * RP;
  static constexpr int SPITCH = NIN + (Q < 16 ? 8 : 0);
  static constexpr size_t tw_bytes = round128((size_t)Q * TP * 8);
  static constexpr size_t x_bytes = ALIAS ? 0 : round128((size_t)XELEMS * 8);
  static constexpr size_t g_bytes = FUSED ? round128((size_t)(n / 2 + 1) * W * 8) : 0;
  static constexpr size_t in_bytes = CONTIG ? (size_t)W * SPITCH * 8 : (size_t)NIN * W * 8;
  static constexpr size_t xr_bytes = ALIAS ? (size_t)(P / XR) * Q * W * 8 : 0;
  static constexpr size_t slot_bytes = round128(in_bytes > xr_bytes ? in_bytes : xr_bytes);
  static constexpr size_t off_tw = 0;
  static constexpr size_t off_x = tw_bytes;
  static constexpr size_t off_g = off_x + x_bytes;
  static constexpr size_t off_stg = off_g + g_bytes;
  static constexpr size_t smem = off_stg + NSTG * slot_bytes;
  static_assert(P > 0 && P % Q == 0, "unsupported length");
  static_assert(W % 2 == 0 && NSTG >= 2, "W even (16-byte staging), at least two stages");
  static_assert(!FUSED || !CONTIG, "the fused pass runs on strided pencils");
  static_assert(MODE != MODE_FUSEDN, "one field per fused launch");
  static_assert(!ALIAS || (!CONTIG && W <= 16), "aliased exchange: strided pencils, W <= 16");
  __host__ __device__ static int xi(int k1, int t, int w) {
    return CONTIG ? w * WP + k1 * QP + t : k1 * RP + t * W + w;
  }
  __host__ __device__ static int si(int pos, int w) { return CONTIG ? w * SPITCH + pos : pos * W + w; }
  __host__ __device__ static int ai(int k1r, int t, int w) { return k1r * (Q * W) + ((t * W + w) ^ ((k1r & SWZ) * W)); }
};

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}

// Stages the input of one tile into a slot with 16-byte copies (complex input;
// rows 16-byte aligned, checked by the launcher).
template <typename K>
__device__ __forceinline__ void stage_input(const PassArgs<float>& a, int tile, float2* slot) {
  const float2* gin = reinterpret_cast<const float2*>(a.in);
  if constexpr (K::CONTIG_) {
    constexpr int cpr = K::NIN / 2;  // 16-byte chunks per row
    const long long row0 = (long long)tile * K::W;
    for (int c = threadIdx.x; c < K::W * cpr; c += K::threads) {
      const int w = c / cpr, k = c % cpr;
      if (row0 + w < a.O) cp_async16(slot + K::si(2 * k, w), gin + (row0 + w) * a.in_pitch_o + 2 * k);
    }
  } else {
    constexpr int cpr = K::W / 2;
    const int o = tile / a.nblk_i;
    const int inner0 = (tile - o * a.nblk_i) * K::W;
    const float2* base = gin + (long long)o * a.in_pitch_o + inner0;
    for (int c = threadIdx.x; c < K::NIN * cpr; c += K::threads) {
      const int pos = c / cpr, k = c % cpr;
      if (inner0 + 2 * k < a.I) cp_async16(slot + K::si(pos, 2 * k), base + pos * a.in_pitch_pos + 2 * k);
    }
  }
}

// stage_input with the input pointer given apart from the pass arguments (the
// batched kernel's first pass reads the caller's density)
template <typename K>
__device__ __forceinline__ void stage_input_from(const PassArgs<float>& a, const float2* gin, int tile, float2* slot) {
  if constexpr (K::CONTIG_) {
    constexpr int cpr = K::NIN / 2;
    const long long row0 = (long long)tile * K::W;
    for (int c = threadIdx.x; c < K::W * cpr; c += K::threads) {
      const int w = c / cpr, k = c % cpr;
      if (row0 + w < a.O) cp_async16(slot + K::si(2 * k, w), gin + (row0 + w) * a.in_pitch_o + 2 * k);
    }
  } else {
    constexpr int cpr = K::W / 2;
    const int o = tile / a.nblk_i;
    const int inner0 = (tile - o * a.nblk_i) * K::W;
    const float2* base = gin + (long long)o * a.in_pitch_o + inner0;
    for (int c = threadIdx.x; c < K::NIN * cpr; c += K::threads) {
      const int pos = c / cpr, k = c % cpr;
      if (inner0 + 2 * k < a.I) cp_async16(slot + K::si(pos, 2 * k), base + pos * a.in_pitch_pos + 2 * k);
    }
  }
}

// Stages rows 0..n/2 of the multiplier octant for the W pencils of a tile
// (8-byte copies; entry (row, w) at row W + w).  A thread's copies all belong
// to pencil w = threadIdx.x mod W.
template <typename K>
__device__ __forceinline__ void stage_mult(const PassArgs<float>& a, int tile, float2* gs) {
  const int w = threadIdx.x % K::W;
  const int inner = (tile % a.nblk_i) * K::W + w;
  if (inner >= a.I) return;
  const int n1 = a.nn[1], n2 = a.nn[2];
  long long rest, pitch0;
  if (a.d == 3) {
    const int m1 = inner / n2, m2 = inner % n2;
    rest = (long long)fold_freq(m1, n1) * (a.Nhs[2] + 1) + fold_freq(m2, n2);
    pitch0 = (long long)(a.Nhs[1] + 1) * (a.Nhs[2] + 1);
  } else {
    rest = fold_freq(inner, n1);
    pitch0 = a.Nhs[1] + 1;
  }
  const float2* src = reinterpret_cast<const float2*>(a.fields[0].mult) + rest;
  for (int r = threadIdx.x / K::W; r <= K::n_ / 2; r += K::threads / K::W) cp_async8(gs + r * K::W + w, src + r * pitch0);
}

// ---------------------------------------------------------------------------
// the pass kernel
//   MODE_FWD:    n/2 inputs (zero-padded to n) -> n outputs
//   MODE_INV:    n inputs -> the first n/2 outputs
//   MODE_FUSED1: n/2 inputs -> forward -> x multiplier -> inverse -> n/2 outputs
// Thread (w, t) of a tile: contiguous w = tid / Q, t = tid mod Q; strided
// w = tid mod W, t = tid / W (lanes over pencils: coalesced rows).  In step B
// the same thread is column thread u = t.
// ---------------------------------------------------------------------------
template <int n, bool CONTIG, int MODE, int W, int NSTG, int MINB, bool ALIAS = false>
__global__ void __launch_bounds__(W*(n / fs_P(n)), MINB) fourstep_pass(const PassArgs<float> a) {
  using K = Cfg<n, CONTIG, MODE, W, NSTG, ALIAS>;
  constexpr int P = K::P, Q = K::Q, CC = K::CC, H = P / 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* tws = reinterpret_cast<float2*>(smem_raw + K::off_tw);
  float2* xs = reinterpret_cast<float2*>(smem_raw + K::off_x);
  float2* gs = reinterpret_cast<float2*>(smem_raw + K::off_g);
  float2* stg = reinterpret_cast<float2*>(smem_raw + K::off_stg);
  constexpr int SLOT = (int)(K::slot_bytes / 8);

  const int tid = threadIdx.x;
  const int w = CONTIG ? tid / Q : tid % W;
  const int t = CONTIG ? tid % Q : tid / W;
  const int ntiles = CONTIG ? (a.O + W - 1) / W : a.O * a.nblk_i;  // < 2^31 (checked by usable)

  // prologue: inputs of the first NSTG - 1 tiles (the fused pass pairs each
  // with an empty group, so that every tile's groups are (multiplier, input))
#pragma unroll
  for (int s = 0; s < NSTG - 1; ++s) {
    const int tl = blockIdx.x + s * gridDim.x;
    if constexpr (K::FUSED) cp_async_commit();
    if (tl < ntiles) stage_input<K>(a, tl, stg + s * SLOT);
    cp_async_commit();
  }
  // twiddles w_n^(t k1), published by the first tile's barrier
  const float2* gtw = reinterpret_cast<const float2*>(a.tw);
  for (int i = tid; i < Q * P; i += K::threads) {
    const int tt = i / P, k1 = i % P;
    tws[tt * K::TP + k1] = gtw[(tt * k1) % n];
  }
  const float4* twt = reinterpret_cast<const float4*>(tws + t * K::TP);

  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    // groups per tile: [multiplier rows of this tile,] input of tile + NSTG - 1
    if constexpr (K::FUSED) {
      stage_mult<K>(a, tile, gs);
      cp_async_commit();
    }
    {
      const int tl = tile + (NSTG - 1) * gridDim.x;
      if (tl < ntiles) stage_input<K>(a, tl, stg + ((it + NSTG - 1) % NSTG) * SLOT);
      cp_async_commit();
    }
    cp_async_wait<K::FUSED ? 2 * (NSTG - 1) : NSTG - 1>();
    __syncthreads();
    float2* slot = stg + (it % NSTG) * SLOT;

    bool valid;
    long long out_base;
    if (CONTIG) {
      const int row = tile * W + w;
      valid = row < a.O;
      out_base = (long long)row * a.out_pitch_o;
    } else {
      const int o = tile / a.nblk_i;
      const int inner = (tile - o * a.nblk_i) * W + w;
      valid = inner < a.I;
      out_base = (long long)o * a.out_pitch_o + inner;
    }
    float2* outp = reinterpret_cast<float2*>(a.out) + out_base;
    const long long op = CONTIG ? 1 : a.out_pitch_pos;

    // step-B columns of this thread: t + Q c; in the fused pass with two
    // columns, t and its mirror P - t (Q for t = 0), so that frequencies k and
    // n - k (one octant row) meet in one thread
    constexpr bool MIRROR = K::FUSED && CC == 2;
    auto col = [&](int c) { return (MIRROR && c == 1) ? (t == 0 ? Q : P - t) : t + Q * c; };

    float2 v[P];
    if constexpr (MODE != MODE_INV) {
      // step A: pruned P-point DFT over q, twiddles
#pragma unroll
      for (int q = 0; q < H; ++q) v[q] = slot[K::si(t + Q * q, w)];
      dft_fwd_halfzero<P>(v);
      apply_twiddles<P, false>(v, twt);
      // exchange, step B: Q-point DFTs of columns k1 = t + Q c
      if constexpr (ALIAS) {
        // round c moves columns [Q c, Q c + Q) through the slot
#pragma unroll
        for (int c = 0; c < CC; ++c) {
          __syncthreads();  // the slot's previous readers are done
#pragma unroll
          for (int r = 0; r < Q; ++r) slot[K::ai(r, t, w)] = v[Q * c + r];
          if (K::FUSED && c == 0) cp_async_wait<1>();  // this tile's multiplier rows
          __syncthreads();
#pragma unroll
          for (int j = 0; j < Q; ++j) v[Q * c + j] = slot[K::ai(col(c) - Q * c, j, w)];
        }
      } else {
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) xs[K::xi(k1, t, w)] = v[k1];
        if constexpr (K::FUSED) cp_async_wait<1>();  // this tile's multiplier rows
        __syncthreads();
#pragma unroll
        for (int c = 0; c < CC; ++c)
#pragma unroll
          for (int j = 0; j < Q; ++j) v[c * Q + j] = xs[K::xi(col(c), j, w)];
      }
#pragma unroll
      for (int c = 0; c < CC; ++c) Dft<Q, false>::run(v + c * Q);
      if constexpr (MODE == MODE_FWD) {
        if (valid) {
#pragma unroll
          for (int c = 0; c < CC; ++c)
#pragma unroll
            for (int k2 = 0; k2 < Q; ++k2) outp[(t + Q * c + P * k2) * op] = v[c * Q + k2];
        }
      } else {
        // multiply by the kernel spectrum at k = col + P k2: octant row k
        // for k2 < Q/2, n - k above; step B'
        if constexpr (MIRROR) {
          if (t != 0) {
            // (0, k2) and (1, Q - 1 - k2) are frequencies k and n - k
            const float2* gp = gs + t * W + w;
            const float2* gn = gs + (n - t) * W + w;
#pragma unroll
            for (int k2 = 0; k2 < Q; ++k2) {
              const float2 g = k2 < Q / 2 ? gp[P * k2 * W] : gn[-P * k2 * W];
              v[k2] = cmul(v[k2], g);
              v[Q + Q - 1 - k2] = cmul(v[Q + Q - 1 - k2], g);
            }
          } else {
            // columns 0 and Q: each is its own mirror
#pragma unroll
            for (int k2 = 0; k2 < Q; ++k2) {
              const int r0 = P * (k2 < Q - k2 ? k2 : Q - k2);
              const int r1 = k2 < Q / 2 ? Q + P * k2 : n - Q - P * k2;
              v[k2] = cmul(v[k2], gs[r0 * W + w]);
              v[Q + k2] = cmul(v[Q + k2], gs[r1 * W + w]);
            }
          }
        } else {
#pragma unroll
          for (int c = 0; c < CC; ++c) {
            const float2* gp = gs + (t + Q * c) * W + w;
            const float2* gn = gs + (n - t - Q * c) * W + w;
#pragma unroll
            for (int k2 = 0; k2 < Q; ++k2)
              v[c * Q + k2] = cmul(v[c * Q + k2], k2 < Q / 2 ? gp[P * k2 * W] : gn[-P * k2 * W]);
          }
        }
#pragma unroll
        for (int c = 0; c < CC; ++c) Dft<Q, true>::run(v + c * Q);
        // exchange back: thread t gathers all k1 of its t
        if constexpr (ALIAS) {
#pragma unroll
          for (int c = 0; c < CC; ++c) {
            __syncthreads();
#pragma unroll
            for (int j = 0; j < Q; ++j) slot[K::ai(col(c) - Q * c, j, w)] = v[c * Q + j];
            __syncthreads();
#pragma unroll
            for (int r = 0; r < Q; ++r) v[Q * c + r] = slot[K::ai(r, t, w)];
          }
        } else {
          __syncthreads();  // step-B reads of the exchange buffer are done
#pragma unroll
          for (int c = 0; c < CC; ++c)
#pragma unroll
            for (int j = 0; j < Q; ++j) xs[K::xi(col(c), j, w)] = v[c * Q + j];
          __syncthreads();
#pragma unroll
          for (int k1 = 0; k1 < P; ++k1) v[k1] = xs[K::xi(k1, t, w)];
        }
        apply_twiddles<P, true>(v, twt);
        idft_cropped<P>(v);
        if (valid) {
#pragma unroll
          for (int q = 0; q < H; ++q) outp[(t + Q * q) * op] = v[q];
        }
      }
    } else {
      // step B': Q-point inverse DFTs over k2 of columns k1 = t + Q c, exchange
#pragma unroll
      for (int c = 0; c < CC; ++c) {
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) v[c * Q + k2] = slot[K::si(t + Q * c + P * k2, w)];
        Dft<Q, true>::run(v + c * Q);
      }
      if constexpr (ALIAS) {
        __syncthreads();  // every thread's input reads of the slot are done
#pragma unroll
        for (int c = 0; c < CC; ++c)
#pragma unroll
          for (int j = 0; j < Q; ++j) slot[K::ai(t + Q * c, j, w)] = v[c * Q + j];
        __syncthreads();
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) v[k1] = slot[K::ai(k1, t, w)];
      } else {
#pragma unroll
        for (int c = 0; c < CC; ++c)
#pragma unroll
          for (int j = 0; j < Q; ++j) xs[K::xi(t + Q * c, j, w)] = v[c * Q + j];
        __syncthreads();
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) v[k1] = xs[K::xi(k1, t, w)];
      }
      // step A': conjugate twiddles, cropped P-point inverse DFT over k1
      apply_twiddles<P, true>(v, twt);
      idft_cropped<P>(v);
      if (valid) {
#pragma unroll
        for (int q = 0; q < H; ++q) outp[(t + Q * q) * op] = v[q];
      }
    }
    __syncthreads();  // slot, exchange buffer and multiplier rows are free again
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// TMA fused pass (n = 512, P = 32, Q = 16; the fused axis of spectra laid out
// [N0 = 256 rows][I pencils], in place).  A tile is W = 8 or 16 pencils x 256
// rows moved by the tensor memory accelerator: a cp.async.bulk.tensor load
// completes on an mbarrier, and the results leave by a bulk tensor store from
// the same slot.  Warp i owns pencils 2i and 2i + 1 (lane = w' + 2 (t mod 8) +
// 16 (t / 8): a half-warp, the unit of 64-bit bank conflicts, covers 8 values
// of t of both pencils), so both exchanges of a pencil stay inside the warp,
// through its private 8 KB buffer, with __syncwarp; the multiplier rows of a
// tile are staged by all threads with 8-byte cp.async copies that arrive on a
// second mbarrier; so the one CTA barrier per tile orders only the slot's
// reuse and the bulk store.  With W = 8 two CTAs share an SM and drift apart,
// so that the shared-memory traffic of one overlaps the arithmetic of the
// other.  Each thread's twiddles w_n^(t k1) stay in registers (t is fixed).
// Shared layouts, in 8-byte elements:
//   slot and multiplier rows: rows of W pencils (8 W bytes), the pair of
//     pencils (2c, 2c + 1) in 16-byte chunk c xor swz(row) -- the tensor map's
//     128-byte (W = 16) or 64-byte (W = 8) swizzle;
//   exchange (warp-private): element (k1, j) of pencil w' at
//     2 (16 k1 + ((j + k1) mod 16)) + w', the skew spreading both directions of
//     the exchange over the banks.
// Waits are bounded (clock64); on timeout the kernel sets *err and runs out
// its loop without waiting.
// ---------------------------------------------------------------------------
template <int W_, int NSTG_ = 2>
struct TmaFusedCfg {
  static constexpr int n_ = 512, P = 32, Q = 16, W = W_, threads = 16 * W_, NIN = 256;
  static constexpr int NSTG = NSTG_;  // input slots: tiles in flight ahead of the one computed
  static constexpr int ROW = W;                              // elements per row: 64 or 128 bytes
  static constexpr size_t slot_bytes = (size_t)NIN * W * 8;  // 16 or 32 KB, 1024-byte aligned
  static constexpr size_t off_slot = 0;
  static constexpr size_t off_x = NSTG * slot_bytes;
  static constexpr size_t x_bytes = (size_t)(W / 2) * 8192;  // 8 KB per warp
  static constexpr size_t off_g = off_x + x_bytes;
  static constexpr size_t g_bytes = round128((size_t)(n_ / 2 + 1) * W * 8);
  static constexpr size_t off_bar = off_g + g_bytes;
  static constexpr size_t smem = off_bar + 8 * (NSTG + 1) + 1024;  // + alignment slack of the base
  static_assert(NSTG >= 2 && NSTG <= 4, "2 to 4 input slots");
  static_assert(W == 8 || W == 16, "tiles of 8 (64-byte swizzle) or 16 (128-byte swizzle) pencils");
  // 16-byte chunk column of row `row` holding the pencil pair c: c xor swz(row)
  __host__ __device__ static int swz(int row) { return W == 16 ? (row & 7) : ((row >> 1) & 3); }
  // (row, pencil w) in the swizzled slot / multiplier rows
  __host__ __device__ static int eb(int row, int w) { return row * ROW + (((w >> 1) ^ swz(row)) << 1) + (w & 1); }
  // exchange element (k1, j) of pencil wp in a warp's buffer
  __host__ __device__ static int xe(int k1, int j, int wp) { return 2 * (16 * k1 + ((j + k1) & 15)) + wp; }
  __host__ __device__ static int lane_t(int lane) { return ((lane >> 4) << 3) | ((lane >> 1) & 7); }
};
constexpr long long FS_WAIT_CYCLES = 1LL << 31;  // about one second

__device__ __forceinline__ void fs_mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fs_mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool fs_mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > FS_WAIT_CYCLES) return false;
  }
}
__device__ __forceinline__ void fs_tma_load2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fs_tma_store2d(const CUtensorMap* map, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(src)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
template <int W, int MINB, int NSTG = 2>
__global__ void __launch_bounds__(16 * W, MINB)
    fourstep_tma_fused(const PassArgs<float> a, const __grid_constant__ CUtensorMap map) {
  using K = TmaFusedCfg<W, NSTG>;
  constexpr int P = K::P, Q = K::Q, H = P / 2, n = K::n_;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // swizzled slots: 1024-byte aligned
  unsigned char* sb = smem_raw + (base - raw);
  float2* slots = reinterpret_cast<float2*>(sb + K::off_slot);
  float2* gs = reinterpret_cast<float2*>(sb + K::off_g);
  const uint32_t bar_in0 = base + (uint32_t)K::off_bar, bar_g = bar_in0 + 8 * NSTG;
  constexpr int SLOT = (int)(K::slot_bytes / 8);

  const int tid = threadIdx.x;
  const int wi = tid >> 5, lane = tid & 31;
  const int t = K::lane_t(lane), wp = lane & 1;
  const int w = 2 * wi + wp;
  float2* xw = reinterpret_cast<float2*>(sb + K::off_x) + wi * 1024;  // this warp's exchange buffer
  const int ntiles = a.nblk_i;
  bool ok = true;
  // work units: a tile and, in 3D, its mirror tile (m1 -> n1 - m1, the same m2
  // block), whose pencils read the same multiplier rows: staged once per unit
  const int n1 = a.nn[1], n2 = a.nn[2];
  const bool pair = (a.d == 3) && (n2 % W == 0) && (a.I == n1 * n2);
  const int rowblk = pair ? n2 / W : 1;  // tiles per m1 row
  const int nunits = pair ? (n1 / 2 + 1) * rowblk : ntiles;
  auto unit_ntiles = [&](int u) {
    if (!pair) return 1;
    const int m = u / rowblk;
    return (m == 0 || m == n1 / 2) ? 1 : 2;
  };
  auto unit_tile = [&](int u, int kk) {
    if (!pair) return u;
    const int m = u / rowblk, bb = u - m * rowblk;
    return (kk == 0 ? m : n1 - m) * rowblk + bb;
  };
  // thread 0's load cursor: the next tile of this CTA's sequence to load
  int lu = blockIdx.x, lk = 0;
  auto load_next = [&](int slot_index) {
    if (lu >= nunits) return;
    const int tl = unit_tile(lu, lk);
    fs_mbar_expect_tx(bar_in0 + 8 * slot_index, (uint32_t)K::slot_bytes);
    fs_tma_load2d(base + (uint32_t)(K::off_slot + slot_index * K::slot_bytes), &map, 2 * W * tl, 0,
                  bar_in0 + 8 * slot_index);
    if (++lk == unit_ntiles(lu)) {
      lk = 0;
      lu += gridDim.x;
    }
  };

  if (tid == 0) {
    for (int s = 0; s < NSTG; ++s) fs_mbar_init(bar_in0 + 8 * s, 1);
    fs_mbar_init(bar_g, K::threads);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < NSTG; ++s) load_next(s);
  // multiplier rows of a tile: thread tid copies rows tid/W + 16 m of pencil tid mod W
  const int gw = tid % W;
  auto stage_g = [&](int tile) {
    const int inner = tile * K::W + gw;
    if (inner < a.I) {
      const int n1 = a.nn[1], n2 = a.nn[2];
      long long rest, pitch0;
      if (a.d == 3) {
        const int m1 = inner / n2, m2 = inner % n2;
        rest = (long long)fold_freq(m1, n1) * (a.Nhs[2] + 1) + fold_freq(m2, n2);
        pitch0 = (long long)(a.Nhs[1] + 1) * (a.Nhs[2] + 1);
      } else {
        rest = fold_freq(inner, n1);
        pitch0 = a.Nhs[1] + 1;
      }
      const float2* src = reinterpret_cast<const float2*>(a.fields[0].mult) + rest;
      for (int r = tid / W; r <= n / 2; r += K::threads / W) cp_async8(gs + K::eb(r, gw), src + r * pitch0);
    }
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar_g) : "memory");
  };
  if ((int)blockIdx.x < nunits) stage_g(unit_tile(blockIdx.x, 0));
  // this thread's twiddles w_n^(t k1), k1 = 1..P-1: t is fixed for the
  // kernel's lifetime, so they stay in registers
  const float2* gtw = reinterpret_cast<const float2*>(a.tw);
  float2 twr[P];
#pragma unroll
  for (int k1 = 1; k1 < P; ++k1) twr[k1] = __ldg(gtw + ((t * k1) & (n - 1)));
  __syncthreads();
  // step-B columns t and its mirror P - t (Q for t = 0): frequencies k and n - k meet in a thread
  const int col1 = t == 0 ? Q : P - t;
  // multiplier rows of column t (octant row k for k2 < Q/2, n - k above)
  const float2* gp = gs + K::eb(t, w);       // rows t + P k2 keep t's chunk column
  const float2* gn = gs + K::eb(n - t, w);   // rows n - t - P k2 keep n - t's

  int it = 0, ui = 0;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++ui)
  for (int kk = 0, nt = unit_ntiles(u); kk < nt; ++kk, ++it) {
    const int tile = unit_tile(u, kk);
    const int s = it % NSTG;
    float2* slot = slots + s * SLOT;
    if (ok) ok = fs_mbar_wait(bar_in0 + 8 * s, (it / NSTG) & 1);

    float2 v[P];
    // step A: pruned 32-point DFT over q, twiddles, exchange
#pragma unroll
    for (int q = 0; q < H; ++q) v[q] = slot[K::eb(t + Q * q, w)];
    dft_fwd_halfzero<P>(v);
#pragma unroll
    for (int k1 = 1; k1 < P; ++k1) v[k1] = cmul(v[k1], twr[k1]);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) xw[K::xe(k1, t, wp)] = v[k1];
    __syncwarp();
    // step B: 16-point DFTs of columns t and col1
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      v[j] = xw[K::xe(t, j, wp)];
      v[Q + j] = xw[K::xe(col1, j, wp)];
    }
    Dft<Q, false>::run(v);
    Dft<Q, false>::run(v + Q);
    // multiply: element (0, k2) is frequency t + P k2, element (1, Q - 1 - k2)
    // its mirror n - k, one octant row; for t = 0 column Q is its own mirror
    if (kk == 0 && ok) ok = fs_mbar_wait(bar_g, ui & 1);  // this unit's multiplier rows
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
      const float2 g0 = k2 < Q / 2 ? gp[P * k2 * W] : gn[-P * k2 * W];
      v[k2] = cmul(v[k2], g0);
      const int j1 = Q - 1 - k2;
      float2 g1 = g0;
      if (t == 0) g1 = gs[K::eb(j1 < Q / 2 ? Q + P * j1 : n - Q - P * j1, w)];
      v[Q + j1] = cmul(v[Q + j1], g1);
    }
    Dft<Q, true>::run(v);
    Dft<Q, true>::run(v + Q);
    __syncwarp();  // the step-B reads of the buffer are done
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      xw[K::xe(t, j, wp)] = v[j];
      xw[K::xe(col1, j, wp)] = v[Q + j];
    }
    __syncwarp();
    // step A': conjugate twiddles, cropped 32-point inverse DFT over k1
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) v[k1] = xw[K::xe(k1, t, wp)];
#pragma unroll
    for (int k1 = 1; k1 < P; ++k1) v[k1] = cconjmul(v[k1], twr[k1]);
    idft_cropped<P>(v);
#pragma unroll
    for (int q = 0; q < H; ++q) slot[K::eb(t + Q * q, w)] = v[q];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> bulk store
    __syncthreads();  // the tile's results are in the slot; every warp is done with the multiplier rows
    if (tid == 0) fs_tma_store2d(&map, 2 * W * tile, 0, base + (uint32_t)(K::off_slot + s * K::slot_bytes));
    if (kk == nt - 1 && u + (int)gridDim.x < nunits) stage_g(unit_tile(u + gridDim.x, 0));
    if (tid == 0) {
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // the slot has been read out
      load_next(s);
    }
  }
  if (!ok && a.err) atomicOr(a.err, 1);
  if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// One tile of a pass inside the batched persistent kernel (batch.cu): W
// pencils of length n, read straight from global memory through L2 (the data
// may have been written earlier in the same launch, so not through the
// read-only path), one exchange per transform through xs (layout Cfg::xi,
// synchronised with __syncthreads: the caller's CTA is W Q threads), and
// written back.  tws is the (Q x P) twiddle table of this n (pitch Cfg::TP).
// With `slot`, the tile's input was staged there by stage_input_from (layout
// Cfg::si) and is read from shared memory instead.
// The fused pass gathers its multiplier values from the octant in global
// memory before the forward transform, so their latency hides behind it.
// ---------------------------------------------------------------------------
template <int n, bool CONTIG, int MODE, int W>
__device__ __forceinline__ void batch_tile(const PassArgs<float>& a, const float2* in, float2* out, int tile,
                                           float2* xs, const float2* tws, const float2* slot = nullptr) {
  using K = Cfg<n, CONTIG, MODE, W, 2>;
  constexpr int P = K::P, Q = K::Q, CC = K::CC, H = P / 2;
  const int tid = threadIdx.x;
  const int w = CONTIG ? tid / Q : tid % W;
  const int t = CONTIG ? tid % Q : tid / W;
  bool valid;
  long long in_base, out_base;
  int inner = 0;
  if (CONTIG) {
    const int row = tile * W + w;
    valid = row < a.O;
    in_base = (long long)row * a.in_pitch_o;
    out_base = (long long)row * a.out_pitch_o;
  } else {
    const int o = tile / a.nblk_i;
    inner = (tile - o * a.nblk_i) * W + w;
    valid = inner < a.I;
    in_base = (long long)o * a.in_pitch_o + inner;
    out_base = (long long)o * a.out_pitch_o + inner;
  }
  const long long ip = CONTIG ? 1 : a.in_pitch_pos, op = CONTIG ? 1 : a.out_pitch_pos;
  const float2* gin = in + in_base;
  float2* gout = out + out_base;
  const float4* twt = reinterpret_cast<const float4*>(tws + t * K::TP);
  float2 v[P];
  if constexpr (MODE != MODE_INV) {
    float2 g[K::FUSED ? P : 1];
    if constexpr (K::FUSED) {
      // octant row of frequency k = t + Q c + P k2 (k for k2 < Q/2, n - k above)
      const int n1 = a.nn[1], n2 = a.nn[2];
      long long rest, pitch0;
      if (a.d == 3) {
        const int m1 = inner / n2, m2 = inner % n2;
        rest = (long long)fold_freq(m1, n1) * (a.Nhs[2] + 1) + fold_freq(m2, n2);
        pitch0 = (long long)(a.Nhs[1] + 1) * (a.Nhs[2] + 1);
      } else {
        rest = fold_freq(inner, n1);
        pitch0 = a.Nhs[1] + 1;
      }
      const float2* mult = reinterpret_cast<const float2*>(a.fields[0].mult) + rest;
#pragma unroll
      for (int c = 0; c < CC; ++c)
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) {
          const int k = t + Q * c + P * k2;
          const int row = k2 < Q / 2 ? k : n - k;
          g[c * Q + k2] = valid ? __ldg(mult + row * pitch0) : float2{0.f, 0.f};
        }
    }
    if (slot) {
#pragma unroll
      for (int q = 0; q < H; ++q) v[q] = slot[K::si(t + Q * q, w)];
    } else {
#pragma unroll
      for (int q = 0; q < H; ++q) v[q] = valid ? __ldcg(gin + (t + Q * q) * ip) : float2{0.f, 0.f};
    }
    dft_fwd_halfzero<P>(v);
    apply_twiddles<P, false>(v, twt);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) xs[K::xi(k1, t, w)] = v[k1];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CC; ++c)
#pragma unroll
      for (int j = 0; j < Q; ++j) v[c * Q + j] = xs[K::xi(t + Q * c, j, w)];
#pragma unroll
    for (int c = 0; c < CC; ++c) Dft<Q, false>::run(v + c * Q);
    if constexpr (MODE == MODE_FWD) {
      if (valid) {
#pragma unroll
        for (int c = 0; c < CC; ++c)
#pragma unroll
          for (int k2 = 0; k2 < Q; ++k2) gout[(t + Q * c + P * k2) * op] = v[c * Q + k2];
      }
    } else {
#pragma unroll
      for (int c = 0; c < CC; ++c) {
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) v[c * Q + k2] = cmul(v[c * Q + k2], g[c * Q + k2]);
        Dft<Q, true>::run(v + c * Q);
      }
      __syncthreads();  // the step-B reads of xs are done
#pragma unroll
      for (int c = 0; c < CC; ++c)
#pragma unroll
        for (int j = 0; j < Q; ++j) xs[K::xi(t + Q * c, j, w)] = v[c * Q + j];
      __syncthreads();
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) v[k1] = xs[K::xi(k1, t, w)];
      apply_twiddles<P, true>(v, twt);
      idft_cropped<P>(v);
      if (valid) {
#pragma unroll
        for (int q = 0; q < H; ++q) gout[(t + Q * q) * op] = v[q];
      }
    }
  } else {
    if (slot) {
#pragma unroll
      for (int c = 0; c < CC; ++c)
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) v[c * Q + k2] = slot[K::si(t + Q * c + P * k2, w)];
    } else {
#pragma unroll
      for (int c = 0; c < CC; ++c)
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2)
          v[c * Q + k2] = valid ? __ldcg(gin + (t + Q * c + P * k2) * ip) : float2{0.f, 0.f};
    }
#pragma unroll
    for (int c = 0; c < CC; ++c) Dft<Q, true>::run(v + c * Q);
#pragma unroll
    for (int c = 0; c < CC; ++c)
#pragma unroll
      for (int j = 0; j < Q; ++j) xs[K::xi(t + Q * c, j, w)] = v[c * Q + j];
    __syncthreads();
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) v[k1] = xs[K::xi(k1, t, w)];
    apply_twiddles<P, true>(v, twt);
    idft_cropped<P>(v);
    if (valid) {
#pragma unroll
      for (int q = 0; q < H; ++q) gout[(t + Q * q) * op] = v[q];
    }
  }
}

// Tensor map of a fused pass's spectra: rows of I complex pencils (2 I
// floats), N0 rows pitch_pos elements apart; boxes of W pencils x 256 rows
// with the 128-byte (W = 16) or 64-byte (W = 8) swizzle.  cuTensorMapEncodeTiled comes from the driver
// through the runtime (no link against libcuda).
inline cudaError_t encode_fused_map(CUtensorMap* map, void* base, long long pencils, long long rows,
                                    long long pitch_pos, int W) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !f) return cudaErrorNotSupported;
    fn = reinterpret_cast<EncodeFn>(f);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * pencils), (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(pitch_pos * 8)};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * W), 256};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  W == 16 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The TMA fused pass serves n = 512 in place on one slab (O = 1) whose rows
// hold exactly N0 = 256 positions, with a 16-byte aligned base and pitch.
inline bool tma_fused_usable(int n, const PassArgs<float>& a) {
  return n == 512 && a.in == a.out && a.O == 1 && a.nfields == 1 && a.fields[0].odd_axis < 0 &&
         a.fields[0].spectral_axis < 0 && !a.in_real && !a.out_real && a.nout <= 1 && a.Nhs[0] == 256 &&
         a.in_pitch_pos == a.out_pitch_pos && a.in_pitch_pos >= a.I && (reinterpret_cast<uintptr_t>(a.in) % 16) == 0 &&
         (a.in_pitch_pos * 8) % 16 == 0 && a.I % 2 == 0;
}

template <int W, int MINB, int NSTG = 2>
cudaError_t launch_tma_fused(const PassArgs<float>& a0, cudaStream_t s) {
  using K = TmaFusedCfg<W, NSTG>;
  auto kern = fourstep_tma_fused<W, MINB, NSTG>;
  static int grid_cap[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64) return cudaErrorInvalidDevice;
  if (!grid_cap[dev]) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K::threads, K::smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    grid_cap[dev] = sms * per_sm;
  }
  PassArgs<float> a = a0;
  a.nblk_i = (a.I + K::W - 1) / K::W;
  if (a.nblk_i <= 0) return cudaSuccess;
  CUtensorMap map;
  e = encode_fused_map(&map, const_cast<void*>(a.in), a.I, a.Nhs[0], a.in_pitch_pos, W);
  if (e != cudaSuccess) return e;
  const int grid = a.nblk_i < grid_cap[dev] ? a.nblk_i : grid_cap[dev];
  kern<<<grid, K::threads, K::smem, s>>>(a, map);
  return cudaGetLastError();
}

// Whether a pass can run on the four-step kernel: a served length, complex
// input and output staged with 16-byte copies, one output, and for the fused
// pass one plain field (no odd extension, no spectral factor).
inline bool usable(int n, int mode, bool contig, const PassArgs<float>& a) {
  if (!fs_length(n) || !a.async_ok || a.in_real || a.out_real || a.nout > 1) return false;
  if (!contig && (a.I % 2 != 0)) return false;
  if ((long long)a.O * (contig ? 1 : a.I) >= (1LL << 31) - 1024) return false;  // 32-bit tile indices
  if (mode == MODE_FUSEDN) return false;
  if (mode == MODE_FUSED1)
    return !contig && a.nfields == 1 && a.fields[0].odd_axis < 0 && a.fields[0].spectral_axis < 0;
  return true;
}

template <int n, bool CONTIG, int MODE, int W, int NSTG, int MINB, bool ALIAS = false>
cudaError_t launch(const PassArgs<float>& a0, cudaStream_t s) {
  using K = Cfg<n, CONTIG, MODE, W, NSTG, ALIAS>;
  auto kern = fourstep_pass<n, CONTIG, MODE, W, NSTG, MINB, ALIAS>;
  // per device: shared-memory opt-in and the persistent grid (SMs x resident CTAs)
  static int grid_cap[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64) return cudaErrorInvalidDevice;
  if (!grid_cap[dev]) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K::threads, K::smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    grid_cap[dev] = sms * per_sm;
  }
  PassArgs<float> a = a0;
  long long tiles;
  if (CONTIG) {
    a.nblk_i = 1;
    tiles = (a.O + W - 1) / W;
  } else {
    a.nblk_i = (a.I + W - 1) / W;
    tiles = (long long)a.O * a.nblk_i;
  }
  if (tiles <= 0) return cudaSuccess;
  const long long grid = tiles < grid_cap[dev] ? tiles : grid_cap[dev];
  kern<<<(unsigned)grid, K::threads, K::smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fs
}  // namespace vp
