"""The volume potential on the grid (Section 4), oracle side, float64.

phi_p = sum_{p'} T(p - p') f_{p'} for p, p' in [0, N)^d (storage index
p = i + N/2 - 1, Section 4), i.e. an aperiodic discrete convolution with the
kernel of ``oracle.kernel``.  Three independent evaluations:

* ``apply_direct``: the sum as written (brute force, small grids only);
* ``apply_fft2n``: zero-pad to (2N)^d, DFT, multiply by the cropped-kernel
  multiplier, inverse DFT, keep [0, N)^d ("standard aperiodic convolution,
  which only requires zero-padding by a factor of 2", Section 4);
* ``apply_fft4n``: the un-precomputed form of Section 2: zero-pad to (4N)^d and
  multiply by the sampled spectrum G^L itself.

Gradients (spectral differentiation, Section 3 and the abstract's "any
derivative ... at the cost of an additional FFT"):
* exact mode: the same sums with the derivative kernels T_j;
* 2N mode: multiply the (2N)^d product by i s'_{m,j} = i pi m_j (the 2N grid's
  own frequencies, m_j in [-N, N), Nyquist m_j = -N set to 0).
"""
from __future__ import annotations

import numpy as np

from . import fft as offt
from .kernel import signed_freq


def _pad(f: np.ndarray, n: int) -> np.ndarray:
    out = np.zeros((n,) * f.ndim, dtype=np.complex128)
    out[tuple(slice(0, s) for s in f.shape)] = f
    return out


def _crop(x: np.ndarray, N: int) -> np.ndarray:
    return x[tuple(slice(0, N) for _ in range(x.ndim))]


def apply_direct(T_full: np.ndarray, f: np.ndarray) -> np.ndarray:
    """phi_p = sum_{p'} T(p - p') f_{p'}; T_full indexed by offset + N."""
    N, d = f.shape[0], f.ndim
    phi = np.zeros(f.shape, dtype=np.complex128)
    for src in np.ndindex(*f.shape):
        fv = f[src]
        if fv == 0:
            continue
        # offsets p - src for p in [0, N): indices N - src .. 2N - 1 - src
        sl = tuple(slice(N - s, 2 * N - s) for s in src)
        phi += T_full[sl] * fv
    return phi


def apply_direct_at(T_full: np.ndarray, f: np.ndarray, points) -> np.ndarray:
    """phi at the listed storage points only (each by its full sum)."""
    N = f.shape[0]
    out = []
    for p in points:
        # T(p - p') for p' in [0, N): offsets p .. p - N + 1, indices p + N .. p + 1
        sl = tuple(slice(pj + 1, pj + N + 1) for pj in p)
        Tw = T_full[sl][tuple(slice(None, None, -1) for _ in p)]
        out.append(np.sum(Tw * f))
    return np.array(out)


def apply_direct_at_octant(T_oct: np.ndarray, f: np.ndarray, points, odd_axis=None) -> np.ndarray:
    """phi at the listed storage points, each by its full sum over the grid, with
    T(n) read from its octant [0, N]^d by evenness in every n_j (oddness along
    ``odd_axis``): T(p - p') = T_oct[|p_0 - p'_0|, ...] (times sign(p_j - p'_j)
    on the odd axis).  Needs no (2N+1)^d array, so it serves full-size grids."""
    d = f.ndim
    out = []
    for p in points:
        a = [np.abs(int(pj) - np.arange(f.shape[j])) for j, pj in enumerate(p)]
        Tw = T_oct[np.ix_(*a)]
        if odd_axis is not None:
            sgn = np.sign(int(p[odd_axis]) - np.arange(f.shape[odd_axis])).astype(np.float64)
            shape = [1] * d
            shape[odd_axis] = f.shape[odd_axis]
            Tw = Tw * sgn.reshape(shape)
        out.append(np.sum(Tw * f))
    return np.array(out)


def apply_fft2n(ghat_full: np.ndarray, f: np.ndarray) -> np.ndarray:
    N = f.shape[0]
    X = offt.fftn(_pad(f, 2 * N))
    return _crop(offt.ifftn(ghat_full * X), N)


def apply_fft4n(G4: np.ndarray, f: np.ndarray, deriv_axis=None) -> np.ndarray:
    """Section 2's form on the 4N grid (G4 = sampled G^L in DFT order)."""
    N, d = f.shape[0], f.ndim
    mult = G4
    if deriv_axis is not None:
        m = signed_freq(4 * N).astype(np.float64)
        m[m == -2 * N] = 0.0
        shape = [1] * d
        shape[deriv_axis] = 4 * N
        mult = G4 * (1j * 0.5 * np.pi * m).reshape(shape)
    X = offt.fftn(_pad(f, 4 * N))
    return _crop(offt.ifftn(mult * X), N)


def spectral2n_factor(N: int, d: int, j: int) -> np.ndarray:
    """i pi m_j on the 2N grid, Nyquist zeroed (2N-mode gradient multiplier)."""
    m = signed_freq(2 * N).astype(np.float64)
    m[m == -N] = 0.0
    shape = [1] * d
    shape[j] = 2 * N
    return (1j * np.pi * m).reshape(shape)


def grad_spectral2n(ghat_full: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Stacked d gradient fields of the 2N mode."""
    N, d = f.shape[0], f.ndim
    X = ghat_full * offt.fftn(_pad(f, 2 * N))
    return np.stack([_crop(offt.ifftn(spectral2n_factor(N, d, j) * X), N) for j in range(d)])


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_2 / ||b||_2 over all entries."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
