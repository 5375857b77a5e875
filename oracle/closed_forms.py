"""Gaussian-source potentials (Section 5.1), oracle side, float64.

The source is the unit-mass Gaussian rho(r) = (2 pi sigma^2)^{-d/2}
exp(-r^2/(2 sigma^2)) and the potential is g_k * rho with g_k the Green's
function of -(Delta + k^2) (the convention of Tables 1-2).

Readings of garbled printed formulas (each checked by ``radial_convolution``):
* eq. (test_helm_3D) as printed equals minus the potential; the sign of the
  bracket is flipped here.
* eq. (test_lapl_2D) prints Ei; the exponential integral that makes the formula
  finite and correct is E_1 (scipy.special.exp1).
* eq. (test_helm_2D) misses the factor i of g_k = (i/4) H_0^(1) and writes
  H_0(kr) inside the outer integral where H_0(ky) is meant.
* eq. (test_biharm_3D) misses the factor e^{-r^2/(2 sigma^2)} on its
  sigma sqrt(2/pi) term (the printed form tends to r/(8 pi) plus a constant
  instead of r/(8 pi) + sigma^2/(8 pi r) far from the source).
* eq. (test_biharm_2D) prints c_1 r where the constant c_1 is meant, and its
  Ei~(x) = Ei(x) + log x + gamma is finite and correct with E_1 in place of
  Ei (the entire function Ein(x) = int_0^x (1 - e^{-t})/t dt).
The biharmonic potentials use g_b of Tables 1-2 (Delta^2 g_b = -delta).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special

EULER_GAMMA = 0.5772156649015329


def laplace3(r, sigma: float) -> np.ndarray:
    """Eq. (test_lapl_3D): erf(r/(sqrt 2 sigma))/(4 pi r); value at r = 0 is the limit."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty(r.shape)
    z = r == 0
    out[z] = 1.0 / (2.0 * math.pi * math.sqrt(2.0 * math.pi) * sigma)
    rn = r[~z]
    out[~z] = special.erf(rn / (math.sqrt(2.0) * sigma)) / (4.0 * math.pi * rn)
    return out


def laplace3_dr(r, sigma: float) -> np.ndarray:
    """d/dr of ``laplace3`` (r > 0); the gradient is this times x/r."""
    r = np.asarray(r, dtype=np.float64)
    a = math.sqrt(2.0) * sigma
    return (2.0 / (math.sqrt(math.pi) * a) * np.exp(-(r / a) ** 2) / r
            - special.erf(r / a) / r ** 2) / (4.0 * math.pi)


def helmholtz3(r, sigma: float, k: float) -> np.ndarray:
    """Eq. (test_helm_3D) with its sign corrected:
    (e^{-sigma^2 k^2/2}/(4 pi r)) [-Re(e^{-ikr} erf((i sigma^2 k - r)/(sqrt 2 sigma))) + i sin kr].
    At r = 0 the limit (derivative of the bracket) is used."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty(r.shape, dtype=np.complex128)
    pref = math.exp(-0.5 * sigma * sigma * k * k)
    z = r == 0
    out[z] = pref / (4 * math.pi) * (math.sqrt(2 / math.pi) * math.exp(0.5 * sigma * sigma * k * k) / sigma
                                     - k * special.erfi(sigma * k / math.sqrt(2)) + 1j * k)
    rn = r[~z]
    arg = (1j * sigma * sigma * k - rn) / (math.sqrt(2.0) * sigma)
    br = -np.real(np.exp(-1j * k * rn) * special.erf(arg)) + 1j * np.sin(k * rn)
    out[~z] = pref * br / (4 * math.pi * rn)
    return out


def laplace2(r, sigma: float) -> np.ndarray:
    """Eq. (test_lapl_2D) with E_1: -(1/(4 pi)) [E_1(r^2/(2 sigma^2)) + log r^2];
    at r = 0 the limit -(1/(4 pi)) (log(2 sigma^2) - gamma)."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty(r.shape)
    z = r == 0
    out[z] = -(math.log(2 * sigma * sigma) - EULER_GAMMA) / (4 * math.pi)
    rn = r[~z]
    out[~z] = -(special.exp1(rn ** 2 / (2 * sigma * sigma)) + np.log(rn ** 2)) / (4 * math.pi)
    return out


def helmholtz2(r, sigma: float, k: float) -> np.ndarray:
    """Eq. (test_helm_2D), corrected: (i/(4 sigma^2)) [H_0(kr) int_0^r J_0(ky) e^{-y^2/2sigma^2} y dy
    + J_0(kr) int_r^inf H_0(ky) e^{-y^2/2sigma^2} y dy]  (H_0 = H_0^(1)), by quadrature."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    out = np.empty(r.shape, dtype=np.complex128)
    w = lambda y: math.exp(-y * y / (2 * sigma * sigma)) * y
    top = r.max() + 12 * sigma + 1.0
    for i, rv in enumerate(r):
        inner = integrate.quad(lambda y: special.j0(k * y) * w(y), 0, rv, epsabs=0, epsrel=1e-13,
                               limit=400)[0] if rv > 0 else 0.0
        lo = max(rv, 0.0)
        hr = integrate.quad(lambda y: special.j0(k * y) * w(y), lo, top, epsabs=0, epsrel=1e-13, limit=400)[0]
        hi = integrate.quad(lambda y: special.y0(k * y) * w(y), lo, top, epsabs=0, epsrel=1e-13, limit=400)[0]
        h0 = special.hankel1(0, k * rv) if rv > 0 else 0.0
        out[i] = 0.25j / (sigma * sigma) * (h0 * inner + special.j0(k * rv) * complex(hr, hi))
    return out


def biharmonic3(r, sigma: float) -> np.ndarray:
    """Eq. (test_biharm_3D), corrected: (1/(8 pi)) [sigma sqrt(2/pi) e^{-r^2/(2 sigma^2)}
    + erf(r/(sqrt 2 sigma)) (sigma^2/r + r)]; at r = 0 the limit sigma sqrt(2/pi)/(4 pi)."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty(r.shape)
    z = r == 0
    out[z] = sigma * math.sqrt(2 / math.pi) / (4 * math.pi)
    rn = r[~z]
    out[~z] = (sigma * math.sqrt(2 / math.pi) * np.exp(-rn ** 2 / (2 * sigma * sigma))
               + special.erf(rn / (math.sqrt(2) * sigma)) * (sigma * sigma / rn + rn)) / (8 * math.pi)
    return out


def biharmonic2(r, sigma: float) -> np.ndarray:
    """Eq. (test_biharm_2D), corrected: -(sigma^2/(8 pi)) [(x + 1) Ein(x) - e^{-x}] + c_2 r^2 + c_1,
    x = r^2/(2 sigma^2), Ein(x) = E_1(x) + log x + gamma (the series for small x)."""
    r = np.asarray(r, dtype=np.float64)
    x = r ** 2 / (2 * sigma * sigma)
    ein = np.empty(r.shape)
    small = x < 1.0
    xs = x[small]
    acc = np.zeros_like(xs)
    term = xs.copy()
    for n in range(1, 40):  # Ein(x) = sum_{n>=1} (-1)^{n+1} x^n/(n n!)
        acc += (-1) ** (n + 1) * term / n
        term = term * xs / (n + 1)
    ein[small] = acc
    xb = x[~small]
    ein[~small] = special.exp1(xb) + np.log(xb) + EULER_GAMMA
    lg = math.log(1.0 / (2 * sigma * sigma))
    c1 = sigma * sigma / (8 * math.pi) * (EULER_GAMMA + lg)
    c2 = (EULER_GAMMA / 2 + lg / 2 + 1.0) / (8 * math.pi)
    return -sigma * sigma / (8 * math.pi) * ((x + 1.0) * ein - np.exp(-x)) + c2 * r ** 2 + c1


def radial_convolution(d: int, kernel: str, k: float, sigma: float, r: float) -> complex:
    """(g_k * rho)(r) by direct 1D quadrature, independent of the closed forms.
    3D: (2 pi/r) int t rho(t) int_{|r-t|}^{r+t} u g(u) du dt with
        int u g du = (e^{ik(r+t)} - e^{ik|r-t|})/(4 pi i k)  (Laplace: (r+t-|r-t|)/(4 pi)).
    2D Laplace: mean of -log|x-y|/(2 pi) over a circle of radius t is -log(max(r,t))/(2 pi)."""
    rho = lambda t: (2 * math.pi * sigma * sigma) ** (-d / 2) * math.exp(-t * t / (2 * sigma * sigma))
    top = r + 14 * sigma
    if d == 3:
        def inner(t, part):
            if kernel == "biharmonic":  # int u (u/(8 pi)) du
                v = ((r + t) ** 3 - abs(r - t) ** 3) / (24 * math.pi)
            elif kernel == "laplace":
                v = (r + t - abs(r - t)) / (4 * math.pi)
            else:
                v = (np.exp(1j * k * (r + t)) - np.exp(1j * k * abs(r - t))) / (4j * math.pi * k)
            v = 2 * math.pi / r * t * rho(t) * v
            return float(np.real(v) if part == 0 else np.imag(v))
        pts = [r] if r < top else None
        re = integrate.quad(inner, 0, top, args=(0,), points=pts, epsabs=0, epsrel=1e-13, limit=400)[0]
        im = integrate.quad(inner, 0, top, args=(1,), points=pts, epsabs=0, epsrel=1e-13, limit=400)[0]
        return complex(re, im)
    if kernel == "laplace":
        f = lambda t: 2 * math.pi * t * rho(t) * (-math.log(max(r, t)) / (2 * math.pi))
        return complex(integrate.quad(f, 0, top, points=[r], epsabs=0, epsrel=1e-13, limit=400)[0], 0.0)
    if kernel == "biharmonic":
        # the circle mean of g_b(|x - y|) over |y| = t, by quadrature in the angle
        def g(u):
            return -u * u * (math.log(u) - 1.0) / (8 * math.pi) if u > 0 else 0.0

        def circle(t):
            f = lambda th: g(math.sqrt(max(r * r + t * t - 2 * r * t * math.cos(th), 0.0)))
            return 2 * integrate.quad(f, 0, math.pi, epsabs=0, epsrel=1e-13, limit=200)[0]
        f = lambda t: t * rho(t) * circle(t)
        return complex(integrate.quad(f, 0, top, points=[r], epsabs=0, epsrel=1e-12, limit=200)[0], 0.0)
    raise ValueError("2D Helmholtz uses helmholtz2 (Graf addition) directly")
