// precompute.cu -- FP64 precompute of the discrete kernel and its (2N)^d
// multiplier on the device (Sections 2 and 4 of Vico, Greengard & Ferrando).
//
// 1. Sample G^L(|s_m|) at s_m = (pi/2) m for m in [0, 2N]^d: the nonnegative
//    octant of the 4N-oversampled grid (Section 2).  G^L is radial, so the
//    octant determines the whole (4N)^d array.
// 2. T(n) = (4N)^{-d} sum_{m in [-2N,2N)^d} G e^{2 pi i m.n/(4N)} for n in
//    [0, N]^d (Section 4).  By evenness in each m_j this is a separable cosine
//    sum over the octant with weights 1 (m_j = 0, 2N) and 2 (otherwise).
//    Derivative kernels (Section 3) use i s_{m,j} G: along axis j the sum of
//    the pairs (m_j, -m_j) is -pi m_j sin(2 pi m_j n_j/(4N)), Nyquist zeroed.
// 3. Multiplier at m in [0, N]^d: the (2N)^d DFT of T cropped to (-N, N]^d
//    (Section 4): weights 1 (n_j = 0, N), 2 otherwise on cos(pi m n/N); an odd
//    kernel (value 0 at n_j = N) gives -2i sum sin(pi m n/N).
// Each separable step is one batched matrix product along one axis.
#include <cuda_runtime.h>
#include <math.h>

#include "vp_internal.cuh"

namespace vp {

__constant__ double c_gl_x[GL_NODES];
__constant__ double c_gl_w[GL_NODES];

// ---------------------------------------------------------------------------
// Bessel functions J0, J1, Y0, Y1 of a real argument x > 0, FP64, accurate to a
// few units of 1e-16 of their amplitude min(1, sqrt(2/(pi x))) for all x.
//  * x >= 25: Hankel's asymptotic expansion (DLMF 10.17.3-10.17.4)
//      J_nu = sqrt(2/(pi x)) (P cos w - Q sin w),  Y_nu = sqrt(2/(pi x)) (P sin w + Q cos w),
//      w = x - nu pi/2 - pi/4,  P = sum_k (-1)^k a_2k x^-2k,  Q = sum_k (-1)^k a_2k+1 x^-2k-1,
//      a_k(nu) = prod_{j<=k} (4 nu^2 - (2j-1)^2) / (k! 8^k); summed to the smallest term.
//      cos w and sin w are formed from sin x, cos x without rounding x - pi/4.
//  * x < 25: Miller's backward recurrence J_{n-1} = (2n/x) J_n - J_{n+1} from an
//    even order M ~ x + 60, normalised by J_0 + 2 sum_k J_2k = 1 (DLMF 10.12.4);
//    Y0 by Neumann's series (2/pi)(log(x/2) + gamma) J0 - (4/pi) sum_k (-1)^k J_2k/k
//    (A&S 9.1.88) and Y1 = -Y0' from the same series with
//    J_2k' = (J_2k-1 - J_2k+1)/2.  All sums are accumulated during the recurrence.
// ---------------------------------------------------------------------------
struct Bessel01 {
  double j0, j1, y0, y1;
};

__device__ Bessel01 bessel01(double x) {
  const double two_over_pi = 0.63661977236758134308;
  Bessel01 b;
  if (x >= 25.0) {
    double sn, cs;
    sincos(x, &sn, &cs);
    const double r = 0.70710678118654752440;
    const double amp = sqrt(two_over_pi / x);
    double res[4];
    for (int nu = 0; nu < 2; ++nu) {
      const double mu = 4.0 * nu * nu;
      double P = 1.0, Q = 0.0, a = 1.0, xp = 1.0, prev = 1e300;
      for (int k = 1; k < 40; ++k) {
        a *= (mu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (8.0 * k);
        xp /= x;
        const double t = a * xp;
        if (fabs(t) > prev) break;
        prev = fabs(t);
        if (k % 2 == 0)
          P += ((k / 2) % 2 ? -t : t);
        else
          Q += (((k - 1) / 2) % 2 ? -t : t);
        if (fabs(t) < 1e-18) break;
      }
      // nu = 0: w = x - pi/4; nu = 1: w = x - 3 pi/4
      const double cw = nu == 0 ? (cs + sn) * r : (sn - cs) * r;
      const double sw = nu == 0 ? (sn - cs) * r : (-sn - cs) * r;
      res[2 * nu] = amp * (P * cw - Q * sw);
      res[2 * nu + 1] = amp * (P * sw + Q * cw);
    }
    b.j0 = res[0];
    b.y0 = res[1];
    b.j1 = res[2];
    b.y1 = res[3];
    return b;
  }
  const int M = 2 * (int)((x + 60.0) * 0.5);
  double jp1 = 0.0, j = 1e-30;
  double norm = 0.0, s0 = 0.0, s1 = 0.0, jn1 = 0.0;
  // the order-M value is even: account for it before recurring
  norm += 2.0 * j;
  s0 += (((M / 2) % 2) ? -j : j) / (M / 2);
  for (int n = M; n > 0; --n) {
    const double jm1 = (2.0 * n / x) * j - jp1;
    jp1 = j;
    j = jm1;
    const int m = n - 1;  // order of j
    if (m >= 2 && (m % 2) == 0) {
      const int k = m / 2;
      norm += 2.0 * j;
      s0 += ((k % 2) ? -j : j) / k;
    } else if (m % 2 == 1) {
      // odd J_m enters sum_k (-1)^k (J_{2k-1} - J_{2k+1})/k at k = (m+1)/2 and k = (m-1)/2
      const int ka = (m + 1) / 2;
      double c = ((ka % 2) ? -1.0 : 1.0) / ka;
      if (m >= 3) {
        const int kb = (m - 1) / 2;
        c -= ((kb % 2) ? -1.0 : 1.0) / kb;
      }
      s1 += c * j;
      if (m == 1) jn1 = j;
    }
    if (fabs(j) > 1e200) {
      j *= 1e-200;
      jp1 *= 1e-200;
      norm *= 1e-200;
      s0 *= 1e-200;
      s1 *= 1e-200;
      jn1 *= 1e-200;
    }
  }
  norm += j;  // J_0
  const double J0 = j / norm, J1 = jn1 / norm;
  const double lg = log(0.5 * x) + 0.57721566490153286061;
  b.j0 = J0;
  b.j1 = J1;
  b.y0 = two_over_pi * (lg * J0 - 2.0 * s0 / norm);
  b.y1 = -two_over_pi * (J0 / x - lg * J1) + two_over_pi * s1 / norm;
  return b;
}

// ---------------------------------------------------------------------------
// truncated spectra (Tables 1-2), FP64, stable at s = 0 and s = k
// ---------------------------------------------------------------------------
__device__ double2 g_laplace3(double s, double L) {
  if (s == 0.0) return make_double2(0.5 * L * L, 0.0);
  const double t = sin(0.5 * L * s) / s;
  return make_double2(2.0 * t * t, 0.0);
}

// E(a) = int_0^L e^{iar} dr = L e^{iaL/2} sin(aL/2)/(aL/2)
__device__ double2 e_int(double a, double L) {
  const double x = 0.5 * a * L;
  double sn, cs;
  sincos(x, &sn, &cs);
  const double sinc = (x == 0.0) ? 1.0 : sn / x;
  return make_double2(L * sinc * cs, L * sinc * sn);
}

__device__ double2 g_helmholtz3(double s, double k, double L) {
  if (s == 0.0) {
    const double x = k * L;
    if (x >= 0.5) {  // (e^{ix}(1 - ix) - 1)/k^2
      double sn, cs;
      sincos(x, &sn, &cs);
      const double re = cs + x * sn - 1.0, im = sn - x * cs;
      return make_double2(re / (k * k), im / (k * k));
    }
    // L^2 sum_{n>=2} (1 - n) i^n x^{n-2}/n!
    double re = 0.0, im = 0.0, xp = 1.0, fact = 2.0;
    for (int nn = 2; nn < 30; ++nn) {
      const double c = (1.0 - nn) * xp / fact;
      switch (nn & 3) {
        case 0: re += c; break;
        case 1: im += c; break;
        case 2: re -= c; break;
        default: im -= c; break;
      }
      xp *= x;
      fact *= (nn + 1);
    }
    return make_double2(L * L * re, L * L * im);
  }
  // [E(k+s) - E(k-s)]/(2 i s): no pole at s = k
  const double2 ep = e_int(k + s, L), em = e_int(k - s, L);
  const double dx = ep.x - em.x, dy = ep.y - em.y;
  return make_double2(dy / (2.0 * s), -dx / (2.0 * s));
}

__device__ double2 g_laplace2(double s, double L) {
  const double x = L * s;
  const double lnL = log(L);
  if (x < 0.5) {
    // (1 - J0(x))/x^2 and J1(x)/x by their power series
    double a = 0.0, ta = 0.25, b = 0.0, tb = 0.5;
    for (int nn = 1; nn < 30; ++nn) {
      a += ta;
      ta = -ta * x * x / (4.0 * (nn + 1) * (nn + 1));
    }
    for (int nn = 0; nn < 30; ++nn) {
      b += tb;
      tb = -tb * x * x / (4.0 * (nn + 1) * (nn + 2));
    }
    return make_double2(L * L * (a - lnL * b), 0.0);
  }
  const Bessel01 b = bessel01(x);
  return make_double2((1.0 - b.j0) / (s * s) - L * lnL * b.j1 / s, 0.0);
}

__device__ double2 g_helmholtz2(double s, double k, double L) {
  const Bessel01 h = bessel01(L * k);
  const double H0r = h.j0, H0i = h.y0;
  const double H1r = h.j1, H1i = h.y1;
  const double hp = 0.5 * 3.14159265358979323846 * L;  // (pi/2) L
  if (fabs(s - k) >= HELM2D_NEAR_K) {
    // 1 + i hp s J1(Ls) H0 - i hp k J0(Ls) H1, over s^2 - k^2
    double jl0 = 1.0, jl1 = 0.0;
    if (s > 0.0) {
      const Bessel01 bs = bessel01(L * s);
      jl0 = bs.j0;
      jl1 = bs.j1;
    }
    const double a = hp * s * jl1, b = hp * k * jl0;
    const double re = 1.0 - a * H0i + b * H1i;
    const double im = a * H0r - b * H1r;
    const double den = (s - k) * (s + k);
    return make_double2(re / den, im / den);
  }
  // numerator / (s - k) = i hp [H0 <L u J0(Lu)> + k H1 <L J1(Lu)>], means over u in [k, s]
  const double mid = 0.5 * (s + k), half = 0.5 * (s - k);
  double mA = 0.0, mB = 0.0;
  for (int g = 0; g < GL_NODES; ++g) {
    const double u = mid + half * c_gl_x[g];
    const double w = 0.5 * c_gl_w[g];
    double ju0 = 1.0, ju1 = 0.0;
    if (u > 0.0) {
      const Bessel01 bu = bessel01(L * u);
      ju0 = bu.j0;
      ju1 = bu.j1;
    }
    mA += w * L * u * ju0;
    mB += w * L * ju1;
  }
  const double cr = H0r * mA + k * H1r * mB, ci = H0i * mA + k * H1i * mB;
  // i hp (cr + i ci) / (s + k)
  return make_double2(-hp * ci / (s + k), hp * cr / (s + k));
}

// Biharmonic (row Delta^2 of Tables 1-2; g_b = r/(8 pi) in 3D,
// -r^2 (log r - 1)/(8 pi) in 2D).  For x = Ls < 2 the printed closed forms
// cancel (terms of order x^-4 and x^-2 against an O(L^4) value); there the
// power series of the defining radial integral is summed instead:
//   3D: (L^4/2) sum_n (-1)^n x^{2n} / ((2n+1)! (2n+4))
//   2D: -(L^4/4) sum_m (-1)^m (x/2)^{2m} / (m!)^2 [(log L - 1)/(2m+4) - 1/(2m+4)^2]
__device__ double2 g_biharm3(double s, double L) {
  const double x = L * s;
  if (x < BIHARM_SERIES_X) {
    double acc = 0.0, term = 1.0;
    for (int n = 0; n < 30; ++n) {
      acc += ((n & 1) ? -term : term) / (2 * n + 4);
      term *= x * x / ((2.0 * n + 2.0) * (2.0 * n + 3.0));
    }
    return make_double2(0.5 * L * L * L * L * acc, 0.0);
  }
  double sn, cs;
  sincos(x, &sn, &cs);
  const double s2 = s * s;
  return make_double2(((2.0 - x * x) * cs + 2.0 * x * sn - 2.0) / (2.0 * s2 * s2), 0.0);
}

__device__ double2 g_biharm2(double s, double L) {
  const double x = L * s;
  const double lnL = log(L);
  if (x < BIHARM_SERIES_X) {
    double acc = 0.0, term = 1.0;
    for (int m = 0; m < 30; ++m) {
      const double p = 2.0 * m + 4.0;
      acc += ((m & 1) ? -term : term) * ((lnL - 1.0) / p - 1.0 / (p * p));
      term *= 0.25 * x * x / ((m + 1.0) * (m + 1.0));
    }
    return make_double2(-0.25 * L * L * L * L * acc, 0.0);
  }
  const Bessel01 b = bessel01(x);
  const double s2 = s * s;
  return make_double2((b.j0 - 1.0) / (s2 * s2) - L * L * L * (lnL - 1.0) * b.j1 / (4.0 * s) +
                          L * lnL * b.j1 / (s2 * s) - L * L * (2.0 * lnL - 1.0) * b.j0 / (4.0 * s2),
                      0.0);
}

// G at m in prod_j [0, 2N_j]: extents e0 x e1 (x e2), e_j = 2 N_j + 1 (e2 = 1 in 2D),
// the last axis fastest
__global__ void spectrum_octant_kernel(double2* __restrict__ G, int d, int e0, int e1, int e2, int kernel, double k,
                                       double L) {
  const long long total = (long long)e0 * e1 * e2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx;
    const int m2 = (int)(r % e2);
    r /= e2;
    const int m1 = (int)(r % e1);
    const int m0 = (int)(r / e1);
    const double msq = (double)m0 * m0 + (double)m1 * m1 + (double)m2 * m2;
    const double s = 0.5 * 3.14159265358979323846 * sqrt(msq);
    double2 v;
    if (kernel == 2)
      v = (d == 3) ? g_biharm3(s, L) : g_biharm2(s, L);
    else if (d == 3)
      v = (kernel == 0) ? g_laplace3(s, L) : g_helmholtz3(s, k, L);
    else
      v = (kernel == 0) ? g_laplace2(s, L) : g_helmholtz2(s, k, L);
    G[idx] = v;
  }
}

// ---------------------------------------------------------------------------
// transform matrices (row-major Q x P), FP64, with exact integer phase reduction
// ---------------------------------------------------------------------------
__global__ void matrix_kernel(double* __restrict__ M, int N, int type) {
  // type 0: C4 (N+1)x(2N+1); 1: S4 (N+1)x(2N+1); 2: C2 (N+1)x(N+1); 3: S2 (N+1)x(N+1)
  const int Q = N + 1;
  const int P = (type <= 1) ? 2 * N + 1 : N + 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Q * P) return;
  const int n = idx / P, m = idx % P;  // output index n (row), summation index m (column)
  double v;
  if (type == 0) {
    const long long ph = ((long long)m * n) % (4 * N);
    const double c = (m == 0 || m == 2 * N) ? 1.0 : 2.0;
    v = c * cospi((double)ph / (2.0 * N)) / (4.0 * N);
  } else if (type == 1) {
    const long long ph = ((long long)m * n) % (4 * N);
    v = (m == 2 * N) ? 0.0 : -3.14159265358979323846 * m * sinpi((double)ph / (2.0 * N)) / (4.0 * N);
  } else if (type == 2) {
    // row = multiplier frequency, column = kernel offset
    const long long ph = ((long long)m * n) % (2 * N);
    const double c = (m == 0 || m == N) ? 1.0 : 2.0;
    v = c * cospi((double)ph / (double)N);
  } else {
    const long long ph = ((long long)m * n) % (2 * N);
    v = (m == 0 || m == N) ? 0.0 : 2.0 * sinpi((double)ph / (double)N);
  }
  M[idx] = v;
}

// out[o][q][i] = sum_p M[q][p] in[o][p][i].  CONTIG_P: I == 1 (the summed axis
// is the contiguous one), tiles then run over o.
template <bool CONTIG_P>
__global__ void __launch_bounds__(256) axis_transform_kernel(const double2* __restrict__ in, double2* __restrict__ out,
                                                             const double* __restrict__ M, long long O, int P, int Q,
                                                             long long I) {
  __shared__ double As[32][17];
  __shared__ double2 Bs[16][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int q0 = blockIdx.y * 32;
  long long o0;
  long long i0 = 0;
  if (CONTIG_P) {
    o0 = (long long)blockIdx.x * 32;
  } else {
    const long long nbi = (I + 31) / 32;
    o0 = blockIdx.x / nbi;
    i0 = (blockIdx.x % nbi) * 32;
  }
  double2 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_double2(0.0, 0.0);
  for (int p0 = 0; p0 < P; p0 += 16) {
    for (int e = threadIdx.x; e < 512; e += 256) {
      const int qq = e >> 4, pp = e & 15;
      As[qq][pp] = (q0 + qq < Q && p0 + pp < P) ? M[(long long)(q0 + qq) * P + p0 + pp] : 0.0;
    }
    for (int e = threadIdx.x; e < 512; e += 256) {
      int pp, cc;
      if (CONTIG_P) {
        pp = e & 15;
        cc = e >> 4;
      } else {
        cc = e & 31;
        pp = e >> 5;
      }
      double2 val = make_double2(0.0, 0.0);
      if (p0 + pp < P) {
        if (CONTIG_P) {
          const long long oo = o0 + cc;
          if (oo < O) val = in[oo * P + p0 + pp];
        } else {
          const long long ii = i0 + cc;
          if (ii < I) val = in[(o0 * P + p0 + pp) * I + ii];
        }
      }
      Bs[pp][cc] = val;
    }
    __syncthreads();
#pragma unroll
    for (int pp = 0; pp < 16; ++pp) {
      const double2 b = Bs[pp][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double a = As[ty * 4 + u][pp];
        acc[u].x = fma(a, b.x, acc[u].x);
        acc[u].y = fma(a, b.y, acc[u].y);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int q = q0 + ty * 4 + u;
    if (q >= Q) continue;
    if (CONTIG_P) {
      const long long oo = o0 + tx;
      if (oo < O) out[oo * Q + q] = acc[u];
    } else {
      const long long ii = i0 + tx;
      if (ii < I) out[(o0 * Q + q) * I + ii] = acc[u];
    }
  }
}

// scaled copies for the apply: s * x (times -i for an odd kernel) in FP64 and FP32
__global__ void finalize_kernel(const double2* __restrict__ in, double2* __restrict__ out_u, double2* __restrict__ out64,
                                float2* __restrict__ out32, long long count, double scale, int times_minus_i) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    double2 v = in[i];
    if (times_minus_i) v = make_double2(v.y, -v.x);
    if (out_u) out_u[i] = v;
    const double2 s = make_double2(v.x * scale, v.y * scale);
    out64[i] = s;
    out32[i] = make_float2((float)s.x, (float)s.y);
  }
}

__global__ void twiddle_kernel(double2* __restrict__ tw64, float2* __restrict__ tw32, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  double sn, cs;
  sincospi(2.0 * (double)q / (double)n, &sn, &cs);  // exp(-2 pi i q/n)
  tw64[q] = make_double2(cs, -sn);
  tw32[q] = make_float2((float)cs, (float)-sn);
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
cudaError_t set_gauss_legendre(const double* x, const double* w) {
  cudaError_t e = cudaMemcpyToSymbol(c_gl_x, x, sizeof(double) * GL_NODES);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_gl_w, w, sizeof(double) * GL_NODES);
}

cudaError_t launch_spectrum(double2* G, int d, const int* M1s, int kernel, double k, double L, cudaStream_t s) {
  const int e0 = M1s[0], e1 = M1s[1], e2 = d == 3 ? M1s[2] : 1;
  const long long total = (long long)e0 * e1 * e2;
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  spectrum_octant_kernel<<<(unsigned)blocks, 256, 0, s>>>(G, d, e0, e1, e2, kernel, k, L);
  return cudaGetLastError();
}

cudaError_t launch_matrix(double* M, int N, int type, cudaStream_t s) {
  const int P = (type <= 1) ? 2 * N + 1 : N + 1;
  const int total = (N + 1) * P;
  matrix_kernel<<<(total + 255) / 256, 256, 0, s>>>(M, N, type);
  return cudaGetLastError();
}

cudaError_t launch_axis_transform(const double2* in, double2* out, const double* M, long long O, int P, int Q,
                                  long long I, cudaStream_t s) {
  dim3 block(256);
  if (I == 1) {
    dim3 grid((unsigned)((O + 31) / 32), (unsigned)((Q + 31) / 32));
    axis_transform_kernel<true><<<grid, block, 0, s>>>(in, out, M, O, P, Q, I);
  } else {
    dim3 grid((unsigned)(O * ((I + 31) / 32)), (unsigned)((Q + 31) / 32));
    axis_transform_kernel<false><<<grid, block, 0, s>>>(in, out, M, O, P, Q, I);
  }
  return cudaGetLastError();
}

// out = in rounded to FP32 (the FP32 copy of a kernel octant)
__global__ void narrow_kernel(const double2* __restrict__ in, float2* __restrict__ out, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

cudaError_t launch_narrow(const double2* in, float2* out, long long count, cudaStream_t s) {
  long long blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  narrow_kernel<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(in, out, count);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double2* in, double2* out_u, double2* out64, float2* out32, long long count,
                            double scale, int times_minus_i, cudaStream_t s) {
  long long blocks = (count + 255) / 256;
  if (blocks > 152LL * 32) blocks = 152LL * 32;
  finalize_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, out_u, out64, out32, count, scale, times_minus_i);
  return cudaGetLastError();
}

cudaError_t launch_twiddles(double2* tw64, float2* tw32, int n, cudaStream_t s) {
  twiddle_kernel<<<(n + 255) / 256, 256, 0, s>>>(tw64, tw32, n);
  return cudaGetLastError();
}

}  // namespace vp
