"""The oracle's own discrete Fourier transforms (float64 / complex128).

The method needs the (4N)^d inverse transform of the sampled spectrum (Section 4,
precompute) and the (2N)^d forward/inverse pair of the apply (Section 4).  This
module provides both without numpy.fft:

* ``dft_direct``: the O(n^2) definition X_k = sum_j x_j exp(-+2 pi i jk/n);
* ``fft``/``ifft``/``fftn``/``ifftn``: recursive decimation-in-time mixed-radix
  transforms for factors 2, 3, 5, falling back to the direct DFT for any other
  prime factor.

Normalisation follows the common convention: forward unscaled, inverse scaled
by 1/n per axis.  Twiddles are evaluated from exact integer phases (jk mod n) so
each is correctly rounded up to the accuracy of exp.
"""
from __future__ import annotations

import numpy as np

_SMALL_PRIMES = (2, 3, 5)


def _twiddle(num: np.ndarray, n: int, sign: float) -> np.ndarray:
    """exp(sign * 2 pi i * num / n) with num reduced mod n first."""
    return np.exp(sign * 2j * np.pi * (np.mod(num, n) / n))


def dft_direct(x, axis: int = -1, inverse: bool = False) -> np.ndarray:
    """The DFT by its definition (O(n^2) per vector)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    j = np.arange(n)
    W = _twiddle(np.outer(j, j), n, 1.0 if inverse else -1.0)  # W[k, j]
    y = x @ W.T
    if inverse:
        y = y / n
    return np.moveaxis(y, -1, axis)


def _fft_last(x: np.ndarray, sign: float) -> np.ndarray:
    """Unnormalised DFT along the last axis, sign -1 forward, +1 inverse."""
    n = x.shape[-1]
    if n == 1:
        return x.copy()
    p = next((q for q in _SMALL_PRIMES if n % q == 0), None)
    if p is None:  # other prime factor: direct DFT of the whole length
        j = np.arange(n)
        return x @ _twiddle(np.outer(j, j), n, sign).T
    m = n // p
    # x[..., p*j1 + j2] -> sub[..., j2, j1]; transform each decimated sequence.
    sub = np.swapaxes(x.reshape(x.shape[:-1] + (m, p)), -1, -2)
    Y = _fft_last(np.ascontiguousarray(sub), sign)  # [..., j2, k1]
    Y = Y * _twiddle(np.outer(np.arange(p), np.arange(m)), n, sign)
    # X[k1 + m*k2] = sum_j2 Y[j2, k1] * exp(sign 2 pi i j2 k2 / p)
    Wp = _twiddle(np.outer(np.arange(p), np.arange(p)), p, sign)  # [k2, j2]
    X = np.einsum("...jk,lj->...lk", Y, Wp)
    return X.reshape(x.shape[:-1] + (n,))


def fft(x, axis: int = -1) -> np.ndarray:
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    return np.moveaxis(_fft_last(np.ascontiguousarray(x), -1.0), -1, axis)


def ifft(x, axis: int = -1) -> np.ndarray:
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    return np.moveaxis(_fft_last(np.ascontiguousarray(x), 1.0) / n, -1, axis)


def fftn(x) -> np.ndarray:
    y = np.asarray(x, dtype=np.complex128)
    for ax in range(y.ndim):
        y = fft(y, ax)
    return y


def ifftn(x) -> np.ndarray:
    y = np.asarray(x, dtype=np.complex128)
    for ax in range(y.ndim):
        y = ifft(y, ax)
    return y
