"""Truncated Green's-function spectra G^L(s) (float64), oracle side.

Convention (paper Section 1 and Tables 1-2): g_k is the free-space Green's
function of -(Delta + k^2): e^{ikr}/(4 pi r) in 3D, (i/4) H_0^(1)(kr) in 2D;
k = 0 gives 1/(4 pi r) and -log(r)/(2 pi).  The truncated kernel is
g^L = g * rect(r/(2L)) (Section 1, eq. for g^L_k) and G^L is its Fourier
transform, a function of s = |s| only.

Definitions (Section 2, radial transforms):
    3D:  G^L(s) = 4 pi int_0^L sin(sr)/(sr) g(r) r^2 dr
    2D:  G^L(s) = 2 pi int_0^L J_0(sr)     g(r) r   dr
``G_quadrature`` evaluates these integrals numerically; the closed forms below
are Tables 1-2 evaluated so that no removable singularity loses digits:

* 3D Laplace (Table 1, row Delta): 2 (sin(Ls/2)/s)^2, limit L^2/2 at s = 0.
* 3D Helmholtz (Table 1, row Delta+k^2).  The printed form has a removable pole
  at s = k.  Writing sin(sr) = (e^{isr} - e^{-isr})/(2i) in the defining integral
  gives G = [E(k+s) - E(k-s)]/(2 i s) with E(a) = int_0^L e^{iar} dr
  = L e^{iaL/2} sinc(aL/2): the same function with no pole at s = k.
  At s = 0 the limit is (e^{ikL}(1 - ikL) - 1)/k^2.
* 2D Laplace (Table 2, row Delta): (1 - J_0(Ls))/s^2 - L log(L) J_1(Ls)/s; for
  small x = Ls both quotients use their power series, limit L^2(1 - 2 log L)/4.
* 2D Helmholtz (Table 2, row Delta+k^2):
  [1 + (i pi/2) L s J_1(Ls) H_0(Lk) - (i pi/2) L k J_0(Ls) H_1(Lk)]/(s^2 - k^2).
  The numerator vanishes at s = k (Wronskian J_1 Y_0 - J_0 Y_1 = 2/(pi x)); near
  there it is written as an integral over u in [k, s] of its derivative,
  using d/du[u J_1(Lu)] = L u J_0(Lu) and d/du J_0(Lu) = -L J_1(Lu), and the
  mean of the integrand is taken by Gauss-Legendre quadrature.
* Biharmonic (Tables 1-2, row Delta^2): g_b = r/(8 pi) (3D) and
  -r^2 (log r - 1)/(8 pi) (2D), so that Delta^2 g_b = -delta (the sign
  convention of the other rows: g solves -L g = delta).  3D:
  ((2 - x^2) cos x + 2 x sin x - 2)/(2 s^4), x = Ls; 2D: (J_0(x) - 1)/s^4
  - L^3 (log L - 1) J_1(x)/(4s) + L log L J_1(x)/s^3 - L^2 (2 log L - 1) J_0(x)/(4 s^2).
  Both lose digits to cancellation as x -> 0 (the terms grow like x^-4 and
  x^-2 while G^L stays O(L^4)); for x < 2 each is summed from the power series
  of its defining radial integral,
    3D: (L^4/2) sum_n (-1)^n x^{2n} / ((2n+1)! (2n+4)),
    2D: -(L^4/4) sum_m (-1)^m (x/2)^{2m}/(m!)^2 [(log L - 1)/(2m+4) - 1/(2m+4)^2],
  whose first terms are the s = 0 limits L^4/8 and -L^4 (4 log L - 5)/64.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special

LAPLACE, HELMHOLTZ, BIHARMONIC = "laplace", "helmholtz", "biharmonic"

# x = Ls below which the biharmonic spectra are summed from their power series
BIHARM_SERIES_X = 2.0

# |s - k| below which the 2D Helmholtz numerator is evaluated as a divided difference.
HELM2D_NEAR_K = 1.0
_GL_NODES, _GL_WEIGHTS = np.polynomial.legendre.leggauss(24)


def default_L(d: int) -> float:
    """Section 2: L = 1.8 > sqrt(3) in 3D, L = 1.5 > sqrt(2) in 2D."""
    return 1.8 if d == 3 else 1.5


def G_laplace3(s, L: float) -> np.ndarray:
    s = np.asarray(s, dtype=np.float64)
    out = np.empty(s.shape, dtype=np.complex128)
    z = s == 0
    out[z] = L * L / 2.0
    sn = s[~z]
    out[~z] = 2.0 * (np.sin(L * sn / 2.0) / sn) ** 2
    return out


def _E(a: np.ndarray, L: float) -> np.ndarray:
    """E(a) = int_0^L e^{iar} dr = L e^{iaL/2} sin(aL/2)/(aL/2)."""
    return L * np.exp(0.5j * a * L) * np.sinc(a * L / (2.0 * np.pi))


def G_helmholtz3(s, k: float, L: float) -> np.ndarray:
    s = np.asarray(s, dtype=np.float64)
    out = np.empty(s.shape, dtype=np.complex128)
    z = s == 0
    out[z] = _helm3_at_zero(k, L)
    sn = s[~z]
    out[~z] = (_E(k + sn, L) - _E(k - sn, L)) / (2j * sn)
    return out


def _helm3_at_zero(k: float, L: float) -> complex:
    """(e^{ikL}(1 - ikL) - 1)/k^2; for small x = kL by its series
    L^2 sum_{n>=2} (1 - n) i^n x^{n-2}/n!."""
    x = k * L
    if x >= 0.5:
        return (np.exp(1j * x) * (1.0 - 1j * x) - 1.0) / (k * k)
    acc, fact = 0j, 2.0
    for n in range(2, 30):
        acc += (1 - n) * (1j ** n) * x ** (n - 2) / fact
        fact *= n + 1
    return L * L * acc


def G_helmholtz3_table(s, k: float, L: float) -> np.ndarray:
    """Table 1 as printed (valid away from s = 0 and s = k)."""
    s = np.asarray(s, dtype=np.float64)
    num = -1.0 + np.exp(1j * L * k) * (np.cos(L * s) - 1j * (k / s) * np.sin(L * s))
    return num / ((k - s) * (k + s))


def _one_minus_j0_over_x2(x: np.ndarray) -> np.ndarray:
    """(1 - J_0(x))/x^2 = sum_{n>=1} (-1)^{n+1} x^{2n-2} / (4^n (n!)^2) for small x."""
    acc = np.zeros_like(x)
    term = np.full_like(x, 0.25)  # n = 1
    for n in range(1, 30):
        acc += term
        term = -term * x * x / (4.0 * (n + 1) ** 2)
    return acc


def _j1_over_x(x: np.ndarray) -> np.ndarray:
    """J_1(x)/x = sum_{n>=0} (-1)^n x^{2n} / (2^{2n+1} n! (n+1)!) for small x."""
    acc = np.zeros_like(x)
    term = np.full_like(x, 0.5)
    for n in range(0, 30):
        acc += term
        term = -term * x * x / (4.0 * (n + 1) * (n + 2))
    return acc


def G_laplace2(s, L: float) -> np.ndarray:
    s = np.asarray(s, dtype=np.float64)
    x = L * s
    small = x < 0.5
    out = np.empty(s.shape, dtype=np.complex128)
    xs = x[small]
    out[small] = L * L * (_one_minus_j0_over_x2(xs) - math.log(L) * _j1_over_x(xs))
    sb, xb = s[~small], x[~small]
    out[~small] = (1.0 - special.j0(xb)) / sb ** 2 - L * math.log(L) * special.j1(xb) / sb
    return out


def G_helmholtz2(s, k: float, L: float) -> np.ndarray:
    s = np.asarray(s, dtype=np.float64)
    H0 = special.hankel1(0, L * k)
    H1 = special.hankel1(1, L * k)
    out = np.empty(s.shape, dtype=np.complex128)
    near = np.abs(s - k) < HELM2D_NEAR_K
    sf = s[~near]
    num = (1.0 + 0.5j * np.pi * L * sf * special.j1(L * sf) * H0
           - 0.5j * np.pi * L * k * special.j0(L * sf) * H1)
    out[~near] = num / (sf * sf - k * k)
    sn = s[near]
    if sn.size:
        # mean over u in [k, s] of L u J0(Lu) and of L J1(Lu) (Gauss-Legendre)
        mid = 0.5 * (sn + k)[:, None]
        half = 0.5 * (sn - k)[:, None]
        u = mid + half * _GL_NODES[None, :]
        w = 0.5 * _GL_WEIGHTS[None, :]
        mA = np.sum(w * L * u * special.j0(L * u), axis=1)
        mB = np.sum(w * L * special.j1(L * u), axis=1)
        out[near] = 0.5j * np.pi * L * (H0 * mA + k * H1 * mB) / (sn + k)
    return out


def G_helmholtz2_table(s, k: float, L: float) -> np.ndarray:
    """Table 2 as printed (valid away from s = k)."""
    s = np.asarray(s, dtype=np.float64)
    H0 = special.hankel1(0, L * k)
    H1 = special.hankel1(1, L * k)
    num = (1.0 + 0.5j * np.pi * L * s * special.j1(L * s) * H0
           - 0.5j * np.pi * L * k * special.j0(L * s) * H1)
    return num / (s * s - k * k)


def G_biharm3(s, L: float) -> np.ndarray:
    s = np.asarray(s, dtype=np.float64)
    x = L * s
    out = np.empty(s.shape, dtype=np.complex128)
    small = x < BIHARM_SERIES_X
    xs = x[small]
    acc = np.zeros_like(xs)
    term = np.ones_like(xs)  # x^{2n}/(2n+1)!, n = 0
    for n in range(30):
        acc += (-1) ** n * term / (2 * n + 4)
        term = term * xs * xs / ((2 * n + 2) * (2 * n + 3))
    out[small] = 0.5 * L ** 4 * acc
    sb, xb = s[~small], x[~small]
    out[~small] = ((2.0 - xb * xb) * np.cos(xb) + 2.0 * xb * np.sin(xb) - 2.0) / (2.0 * sb ** 4)
    return out


def G_biharm2(s, L: float) -> np.ndarray:
    s = np.asarray(s, dtype=np.float64)
    x = L * s
    lnL = math.log(L)
    out = np.empty(s.shape, dtype=np.complex128)
    small = x < BIHARM_SERIES_X
    xs = x[small]
    acc = np.zeros_like(xs)
    term = np.ones_like(xs)  # (x/2)^{2m}/(m!)^2, m = 0
    for m in range(30):
        p = 2 * m + 4
        acc += (-1) ** m * term * ((lnL - 1.0) / p - 1.0 / p ** 2)
        term = term * (xs / 2) ** 2 / ((m + 1) ** 2)
    out[small] = -0.25 * L ** 4 * acc
    sb, xb = s[~small], x[~small]
    j0, j1 = special.j0(xb), special.j1(xb)
    out[~small] = ((j0 - 1.0) / sb ** 4 - L ** 3 * (lnL - 1.0) * j1 / (4.0 * sb)
                   + L * lnL * j1 / sb ** 3 - L ** 2 * (2.0 * lnL - 1.0) * j0 / (4.0 * sb ** 2))
    return out


def G_truncated(d: int, kernel: str, k: float, L: float, s) -> np.ndarray:
    """G^L(s) for the six supported kernels (three operators, two dimensions)."""
    if d not in (2, 3):
        raise ValueError("d must be 2 or 3")
    if kernel == BIHARMONIC:
        return G_biharm3(s, L) if d == 3 else G_biharm2(s, L)
    if d == 3:
        return G_laplace3(s, L) if kernel == LAPLACE else G_helmholtz3(s, k, L)
    return G_laplace2(s, L) if kernel == LAPLACE else G_helmholtz2(s, k, L)


def green(d: int, kernel: str, k: float, r):
    """Free-space Green's function (Tables 1-2, column 2): of -(Delta + k^2)
    (k = 0: Laplace), or of -Delta^2 (biharmonic)."""
    r = np.asarray(r, dtype=np.float64)
    if kernel == BIHARMONIC:
        return (r / (8 * np.pi) if d == 3 else -r * r * (np.log(r) - 1.0) / (8 * np.pi)) + 0j
    if d == 3:
        return (1.0 / (4 * np.pi * r)) * (np.exp(1j * k * r) if kernel == HELMHOLTZ else 1.0)
    if kernel == LAPLACE:
        return -np.log(r) / (2 * np.pi) + 0j
    return 0.25j * special.hankel1(0, k * r)


def G_quadrature(d: int, kernel: str, k: float, L: float, s: float) -> complex:
    """The radial transform of the truncated kernel (Section 2) by adaptive
    quadrature, independent of the closed forms."""
    def integrand(r, part):
        if d == 3 and kernel == BIHARMONIC:
            v = 4 * np.pi * (np.sin(s * r) / (s * r) if s > 0 else 1.0) * green(3, kernel, k, r) * r * r
        elif d == 3:
            # 4 pi sin(sr)/(sr) g(r) r^2 with g = e^{ikr}/(4 pi r): sin(sr)/s e^{ikr}
            kern = (np.sin(s * r) / s) if s > 0 else r
            v = kern * (np.exp(1j * k * r) if kernel == HELMHOLTZ else 1.0)
        else:
            v = 2 * np.pi * special.j0(s * r) * green(2, kernel, k, r) * r
        return float(np.real(v) if part == 0 else np.imag(v))

    n_osc = int((s + k) * L / np.pi) + 4
    pts = np.linspace(0.0, L, n_osc + 1)
    re = im = 0.0
    for a, b in zip(pts[:-1], pts[1:]):
        re += integrate.quad(integrand, a, b, args=(0,), epsabs=0, epsrel=2e-14, limit=200)[0]
        im += integrate.quad(integrand, a, b, args=(1,), epsabs=0, epsrel=2e-14, limit=200)[0]
    return complex(re, im)
