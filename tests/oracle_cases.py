"""Oracle results for the GPU parity tests, cached per process (test helper)."""
import functools

import numpy as np

from oracle import apply as A
from oracle import kernel as K

KNAME = {0: "laplace", 1: "helmholtz"}


@functools.lru_cache(maxsize=64)
def octants(d, N, kernel, k, L):
    """(T, Ghat) octants by the cosine-sum route."""
    T = K.T_octant_by_sums(d, N, kernel, k, L)
    return T, K.ghat_octant_by_sums(T, N)


@functools.lru_cache(maxsize=64)
def grad_octants(d, N, kernel, k, L, j):
    Tj = K.T_octant_by_sums(d, N, kernel, k, L, deriv_axis=j)
    return Tj, K.ghat_octant_by_sums(Tj, N, odd_axis=j)


def potential(d, N, kernel, k, L, f, grad_mode=None):
    """phi (and the stacked gradient) of the FP64 oracle by the 2N FFT form."""
    T, G = octants(d, N, kernel, k, L)
    Gf = K.ghat_full_from_octant(G)
    f = np.asarray(f, dtype=np.complex128)
    phi = A.apply_fft2n(Gf, f)
    if grad_mode is None:
        return phi, None
    if grad_mode == "exact":
        g = np.stack([A.apply_fft2n(K.ghat_full_from_octant(grad_octants(d, N, kernel, k, L, j)[1], odd_axis=j), f)
                      for j in range(d)])
    else:
        g = A.grad_spectral2n(Gf, f)
    return phi, g


def condition(d, N, kernel, k, L, f, odd_axis=None):
    """kappa = || |T| * |f| ||_2 / || T * f ||_2 >= 1: the scale of rounding
    errors in a discrete convolution relative to its result.  A relative error
    bar eps on well-conditioned data (kappa ~ 1) becomes eps * kappa when the
    result cancels (e.g. an oscillatory kernel on an under-resolved grid)."""
    if odd_axis is None:
        T, _ = octants(d, N, kernel, k, L)
    else:
        T, _ = grad_octants(d, N, kernel, k, L, odd_axis)
    Tabs = np.abs(K.T_full_from_octant(T, odd_axis))
    Gabs = K.ghat_by_fft(Tabs, N)
    f = np.asarray(f, dtype=np.complex128)
    top = np.linalg.norm(A.apply_fft2n(Gabs, np.abs(f)).ravel())
    phi = A.apply_fft2n(K.ghat_full_from_octant(octants(d, N, kernel, k, L)[1]) if odd_axis is None else
                        K.ghat_full_from_octant(grad_octants(d, N, kernel, k, L, odd_axis)[1], odd_axis), f)
    return max(1.0, top / np.linalg.norm(phi.ravel()))


# Relative-L2 bars of the parity sweeps.  A discrete convolution computed in
# floating point with unit roundoff u has forward error of order
# u * log(n) * || |T| * |f| ||, i.e. a relative error of order u * log(n) * kappa
# (kappa from condition()).  kappa is printed beside every case to show how
# much the case's result cancels; the bar asserted is the plain one (1e-5 FP32,
# 1e-12 FP64) for every case, whatever its kappa.


def check(name, err, tol, kappa):
    """Prints the case's error, kappa and bar (pytest -s shows it) and returns
    whether the error is under the plain bar tol."""
    print(f"PARITY {name} rel_l2={err:.3e} kappa={kappa:.2f} bar={tol:.0e}")
    return err < tol
