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

// ---------------------------------------------------------------------------
// compile-time plan: radices chosen greedily (16, 8, 4, 3, 2) dividing both the
// remaining length and the per-thread count E.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pick_radix(int rem, int E) {
  return (rem % 16 == 0 && E % 16 == 0)  ? 16
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
// shared-memory tile: W pencils of n elements, element (w, pos) at
// w*P + pos + (pos >> SH), P = n + (n >> SH) + 1.  The 1-in-2^SH padding makes
// radix-strided accesses within a pencil conflict-free; the odd pitch P makes
// same-position accesses across pencils conflict-free.
// ---------------------------------------------------------------------------
template <typename Real> struct SmemLayout {
  static constexpr int SH = sizeof(Real) == 4 ? 4 : 3;
};
template <typename Real> __host__ __device__ constexpr int smem_pitch(int n) {
  return n + (n >> SmemLayout<Real>::SH) + 1;
}

enum PassMode { MODE_FWD = 0, MODE_INV = 1, MODE_FUSED = 2 };

// Pencils per CTA: 256 threads' worth, at least 16 for strided passes (to fill
// 128-byte rows), bounded by a 72 KB exchange buffer.
template <typename Real> __host__ __device__ constexpr int pencils_per_cta(int n, bool contig) {
  int Tp = n / elems_per_thread<Real>(n);
  int w = 256 / Tp;
  if (w < 1) w = 1;
  if (!contig) {
    if (w < 16) w = 16;
    if (w > 64) w = 64;
  } else if (w > 32) {
    w = 32;
  }
  while (w > 1 && (long)w * smem_pitch<Real>(n) * 2 * (long)sizeof(Real) > 72 * 1024) w >>= 1;
  while (w > 1 && w * Tp > 1024) w >>= 1;
  return w;
}

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
  const C* tw;  // twiddles exp(-2 pi i q/n), q in [0, n)
  // fused pass only
  int nfields;
  int d;
  int Nh;  // N = n/2
  FieldDesc fields[4];
};

template <typename Real, typename C> __device__ __forceinline__ C ld_in(const PassArgs<Real>& a, long long idx) {
  if (a.in_real) return C{__ldg(reinterpret_cast<const Real*>(a.in) + idx), (Real)0};
  return __ldg(reinterpret_cast<const C*>(a.in) + idx);
}
template <typename Real, typename C> __device__ __forceinline__ void st_out(const PassArgs<Real>& a, long long idx, C v) {
  if (a.out_real)
    reinterpret_cast<Real*>(a.out)[idx] = v.x;
  else
    reinterpret_cast<C*>(a.out)[idx] = v;
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

template <typename Real, int n> __device__ __forceinline__ int saddr(int w, int pos) {
  return w * smem_pitch<Real>(n) + pos + (pos >> SmemLayout<Real>::SH);
}

// Exchange after stage S (compute done) into stage S+1 (loads done).
template <typename Real, typename C, int n, int E, bool INV, int S>
__device__ __forceinline__ void exchange(C (&v)[E], C* sm, int w, int t) {
  constexpr int R0 = stage_radix(n, E, INV, S);
  constexpr int R1 = stage_radix(n, E, INV, S + 1);
  constexpr int Tp = n / E;
  __syncthreads();  // previous readers of sm are done
#pragma unroll
  for (int q = 0; q < E / R0; ++q)
#pragma unroll
    for (int r = 0; r < R0; ++r) sm[saddr<Real, n>(w, stage_out_pos<n, E, INV, S>(t + q * Tp, r))] = v[q * R0 + r];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < E / R1; ++q)
#pragma unroll
    for (int r = 0; r < R1; ++r) v[q * R1 + r] = sm[saddr<Real, n>(w, stage_in_pos<n, E, INV, S + 1>(t + q * Tp, r))];
}

// Runs stages [S, NS) of a transform whose stage S inputs are already loaded.
template <typename Real, typename C, int n, int E, bool INV, int S, int NS> struct StageRun {
  __device__ __forceinline__ static void run(C (&v)[E], C* sm, int w, int t, const C* tw) {
    stage_compute<C, n, E, INV, S>(v, t, tw);
    if constexpr (S + 1 < NS) {
      exchange<Real, C, n, E, INV, S>(v, sm, w, t);
      StageRun<Real, C, n, E, INV, S + 1, NS>::run(v, sm, w, t, tw);
    }
  }
};

__device__ __forceinline__ int fold_freq(int m, int n) { return m <= n - m ? m : n - m; }

// ---------------------------------------------------------------------------
// the pass kernel
//   MODE_FWD:   N valid inputs -> n outputs       (forward, pruned input)
//   MODE_INV:   n inputs -> N outputs             (inverse, cropped output)
//   MODE_FUSED: N inputs -> fwd -> x multiplier -> inv -> N outputs, per field
// CONTIG: pencils are contiguous rows; otherwise pencils are strided and the
// W pencils of a CTA are W consecutive inner indices (coalesced).
// ---------------------------------------------------------------------------
template <typename Real, int n, bool CONTIG, int MODE>
__global__ void __launch_bounds__(pencils_per_cta<Real>(n, CONTIG) * (n / elems_per_thread<Real>(n)))
    pencil_pass(const PassArgs<Real> a) {
  using C = typename CxT<Real>::T;
  constexpr int E = elems_per_thread<Real>(n);
  constexpr int Tp = n / E;
  constexpr int W = pencils_per_cta<Real>(n, CONTIG);
  constexpr int NS = plan_nstages(n, E);
  static_assert(NS > 0, "unsupported FFT length");
  constexpr bool FWD_FIRST = (MODE != MODE_INV);
  constexpr int R_first = stage_radix(n, E, !FWD_FIRST, 0);
  constexpr int R_lastinv = stage_radix(n, E, true, NS - 1);
  static_assert(!FWD_FIRST || R_first % 2 == 0, "pruned first stage needs an even radix");
  static_assert(MODE == MODE_FWD || R_lastinv % 2 == 0, "cropped last stage needs an even radix");

  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);

  const int tid = threadIdx.x;
  const int w = CONTIG ? tid / Tp : tid % W;
  const int t = CONTIG ? tid % Tp : tid / W;

  // tile -> pencil coordinates
  long long in_base, out_base;
  bool valid;
  int inner = 0;
  if (CONTIG) {
    const long long row = (long long)blockIdx.x * W + w;
    valid = row < a.O;
    in_base = row * a.in_pitch_o;
    out_base = row * a.out_pitch_o;
  } else {
    const int o = blockIdx.x / a.nblk_i;
    inner = (blockIdx.x % a.nblk_i) * W + w;
    valid = inner < a.I;
    in_base = (long long)o * a.in_pitch_o + inner;
    out_base = (long long)o * a.out_pitch_o + inner;
  }
  const C* tw = a.tw;

  C v[E];
  // ---- first stage loads straight from global memory ----
  {
    constexpr int R = R_first;
#pragma unroll
    for (int q = 0; q < E / R; ++q) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int pos = stage_in_pos<n, E, !FWD_FIRST, 0>(t + q * Tp, r);
        C x = {(Real)0, (Real)0};
        if (valid && (!FWD_FIRST || r < R / 2)) x = ld_in<Real, C>(a, in_base + (long long)pos * a.in_pitch_pos);
        v[q * R + r] = x;
      }
    }
  }

  if constexpr (MODE == MODE_FWD) {
    StageRun<Real, C, n, E, false, 0, NS>::run(v, sm, w, t, tw);
    constexpr int R = stage_radix(n, E, false, NS - 1);
    if (valid) {
#pragma unroll
      for (int q = 0; q < E / R; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int pos = stage_out_pos<n, E, false, NS - 1>(t + q * Tp, r);
          st_out<Real, C>(a, out_base + (long long)pos * a.out_pitch_pos, v[q * R + r]);
        }
    }
  } else if constexpr (MODE == MODE_INV) {
    StageRun<Real, C, n, E, true, 0, NS>::run(v, sm, w, t, tw);
    constexpr int R = R_lastinv;
    if (valid) {
#pragma unroll
      for (int q = 0; q < E / R; ++q)
#pragma unroll
        for (int r = 0; r < R / 2; ++r) {
          const int pos = stage_out_pos<n, E, true, NS - 1>(t + q * Tp, r);
          st_out<Real, C>(a, out_base + (long long)pos * a.out_pitch_pos, v[q * R + r]);
        }
    }
  } else {
    StageRun<Real, C, n, E, false, 0, NS>::run(v, sm, w, t, tw);
    // frequencies of the other axes (fused axis = axis 0, the slowest)
    const int Nh = a.Nh;
    const int np1 = Nh + 1;
    int m1 = 0, m2 = 0;
    if (a.d == 3) {
      m1 = inner / n;
      m2 = inner % n;
    } else {
      m1 = inner;
    }
    const int f1 = fold_freq(m1, n), f2 = fold_freq(m2, n);
    const long long oct_rest = (a.d == 3) ? (long long)f1 * np1 + f2 : f1;
    const long long oct_pitch0 = (a.d == 3) ? (long long)np1 * np1 : np1;
    constexpr int RL = stage_radix(n, E, false, NS - 1);  // == first inverse radix
    for (int fi = 0; fi < a.nfields; ++fi) {
      const FieldDesc fd = a.fields[fi];
      const C* mult = reinterpret_cast<const C*>(fd.mult);
      C y[E];
#pragma unroll
      for (int q = 0; q < E / RL; ++q)
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int m0 = stage_out_pos<n, E, false, NS - 1>(t + q * Tp, r);
          C g = {(Real)0, (Real)0};
          if (valid) g = __ldg(mult + fold_freq(m0, n) * oct_pitch0 + oct_rest);
          if (fd.odd_axis >= 0) {
            const int mj = fd.odd_axis == 0 ? m0 : (fd.odd_axis == 1 ? m1 : m2);
            if (mj > Nh) g = C{-g.x, -g.y};
          }
          if (fd.spectral_axis >= 0) {
            const int mj = fd.spectral_axis == 0 ? m0 : (fd.spectral_axis == 1 ? m1 : m2);
            const int ms = mj < Nh ? mj : (mj == Nh ? 0 : mj - n);
            const Real f = (Real)3.14159265358979323846 * (Real)ms;
            g = C{-g.y * f, g.x * f};  // i pi m_j * g
          }
          y[q * RL + r] = cmul(v[q * RL + r], g);
        }
      if (fi > 0) __syncthreads();  // the previous field's last exchange readers
      StageRun<Real, C, n, E, true, 0, NS>::run(y, sm, w, t, tw);
      constexpr int R = R_lastinv;
      if (valid) {
        const long long ob = out_base + (long long)fi * a.out_field_stride;
#pragma unroll
        for (int q = 0; q < E / R; ++q)
#pragma unroll
          for (int r = 0; r < R / 2; ++r) {
            const int pos = stage_out_pos<n, E, true, NS - 1>(t + q * Tp, r);
            st_out<Real, C>(a, ob + (long long)pos * a.out_pitch_pos, y[q * R + r]);
          }
      }
    }
  }
}

template <typename Real, int n, bool CONTIG> struct PassCfg {
  static constexpr int E = elems_per_thread<Real>(n);
  static constexpr int W = pencils_per_cta<Real>(n, CONTIG);
  static constexpr int threads = W * (n / E);
  static constexpr size_t smem = (size_t)W * smem_pitch<Real>(n) * 2 * sizeof(Real);
  static constexpr int nstages = plan_nstages(n, E);
};

}  // namespace vp
