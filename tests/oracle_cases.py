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
