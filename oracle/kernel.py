"""Discrete kernels of the method (Section 4), oracle side, float64.

Grid and sampling (Sections 2 and 4): N points per axis, h = 1/N; the spectrum
is sampled on the 4N-oversampled grid s_m = 2 pi m/(4N h) = (pi/2) m,
m in [-2N, 2N)^d.  Trapezoidal quadrature of the inverse Fourier integral with
the forward integral also discretised on the grid gives a discrete convolution
(Section 4) with kernel

    T(n) = (4N)^{-d} sum_m G^L(|s_m|) exp(2 pi i m.n/(4N)),   n in [-N, N]^d,

i.e. the inverse (4N)^d DFT of the samples (the factor h^d of the forward
integral and (2 pi)^{-d} ds^d of the inverse cancel to (4N)^{-d}).  Derivative
kernels (spectral differentiation, Section 3) multiply the samples by i s_{m,j};
the Nyquist sample m_j = -2N of that odd factor is set to zero.

Only offsets |n_j| <= N - 1 enter an apply on the N^d grid; the (2N)^d
multiplier is the DFT of T cropped to the window (-N, N]^d ("only an FFT of
dimension (2N)^d is required", Section 4).  At the window edge n_j = N the even
kernel keeps T(N); the odd derivative kernels store 0 there (the edge offset
never reaches a grid point, so the cropped potential does not depend on it).

Each quantity is computed by two routes that share nothing but G^L:
  * full transforms with the oracle's own FFT (``*_by_fft``), and
  * separable cosine/sine sums over the nonnegative octant, which follow from
    the evenness of G^L in every m_j (``*_by_sums``).
"""
from __future__ import annotations

import numpy as np

from . import fft as offt
from .spectrum import G_truncated


def signed_freq(n_fft: int) -> np.ndarray:
    """Frequencies of an n-point DFT in natural storage order: q or q - n."""
    q = np.arange(n_fft)
    return np.where(q < (n_fft + 1) // 2, q, q - n_fft)


# ---------------------------------------------------------------------------
# route 1: full transforms with the oracle FFT
# ---------------------------------------------------------------------------

def spectrum_4n(d: int, N: int, kernel: str, k: float, L: float) -> np.ndarray:
    """G^L(|s_m|) on the full (4N)^d grid in DFT storage order."""
    m = signed_freq(4 * N).astype(np.float64)
    m2 = np.zeros((4 * N,) * d)
    for j in range(d):
        shape = [1] * d
        shape[j] = 4 * N
        m2 = m2 + (m ** 2).reshape(shape)
    s = 0.5 * np.pi * np.sqrt(m2)
    return G_truncated(d, kernel, k, L, s.ravel()).reshape(m2.shape)


def _deriv_factor_4n(d: int, N: int, j: int) -> np.ndarray:
    """i s_{m,j} on the 4N grid, zero at the Nyquist sample m_j = -2N."""
    m = signed_freq(4 * N).astype(np.float64)
    m[m == -2 * N] = 0.0
    shape = [1] * d
    shape[j] = 4 * N
    return (1j * 0.5 * np.pi * m).reshape(shape)


def T_by_fft(d: int, N: int, kernel: str, k: float, L: float, deriv_axis=None,
             G4: np.ndarray | None = None) -> np.ndarray:
    """T (or T_j) on offsets [-N, N]^d, array index n + N, by the inverse 4N DFT."""
    if G4 is None:
        G4 = spectrum_4n(d, N, kernel, k, L)
    if deriv_axis is not None:
        G4 = G4 * _deriv_factor_4n(d, N, deriv_axis)
    t = offt.ifftn(G4)
    idx = np.arange(-N, N + 1) % (4 * N)
    return t[np.ix_(*([idx] * d))]


def window_2n(T_full: np.ndarray, N: int, odd_axis=None) -> np.ndarray:
    """The 2N-periodic array of T cropped to (-N, N]^d (storage q <-> offset q or q-2N)."""
    d = T_full.ndim
    off = signed_freq(2 * N)
    off[N] = N  # the window keeps +N
    t = T_full[np.ix_(*([off + N] * d))].copy()
    if odd_axis is not None:
        sl = [slice(None)] * d
        sl[odd_axis] = N
        t[tuple(sl)] = 0.0
    return t


def ghat_by_fft(T_full: np.ndarray, N: int, odd_axis=None) -> np.ndarray:
    """(2N)^d multiplier: the DFT of the cropped kernel, natural storage order."""
    return offt.fftn(window_2n(T_full, N, odd_axis))


# ---------------------------------------------------------------------------
# route 2: separable sums over the nonnegative octant
# ---------------------------------------------------------------------------

def spectrum_octant(d: int, N: int, kernel: str, k: float, L: float) -> np.ndarray:
    """G^L(|s_m|) for m in [0, 2N]^d.  G^L depends on |m|^2 only; each distinct
    integer |m|^2 is evaluated once and gathered."""
    m = np.arange(2 * N + 1, dtype=np.int64)
    msq = np.zeros((2 * N + 1,) * d, dtype=np.int64)
    for j in range(d):
        shape = [1] * d
        shape[j] = 2 * N + 1
        msq = msq + (m * m).reshape(shape)
    table = G_truncated(d, kernel, k, L, 0.5 * np.pi * np.sqrt(np.arange(d * 4 * N * N + 1,
                                                                         dtype=np.float64)))
    return table[msq]


def _apply_axis(mat: np.ndarray, x: np.ndarray, ax: int) -> np.ndarray:
    """y[..., a, ...] = sum_b mat[a, b] x[..., b, ...] along axis ``ax`` (real mat)."""
    xr = np.moveaxis(x, ax, -1)
    if np.iscomplexobj(xr):
        y = (xr.real @ mat.T) + 1j * (xr.imag @ mat.T)
    else:
        y = xr @ mat.T
    return np.moveaxis(y, -1, ax)


def cos_matrix_4n(N: int) -> np.ndarray:
    """C[n, m] = c(m) cos(2 pi m n/(4N))/(4N), n in [0, N], m in [0, 2N];
    c = 1 at m = 0 and m = 2N (each appears once in [-2N, 2N)), else 2."""
    n = np.arange(N + 1)[:, None]
    m = np.arange(2 * N + 1)[None, :]
    c = np.where((m == 0) | (m == 2 * N), 1.0, 2.0)
    return c * np.cos(2 * np.pi * np.mod(n * m, 4 * N) / (4 * N)) / (4 * N)


def sin_matrix_4n(N: int) -> np.ndarray:
    """Axis factor of T_j: pairs (m, -m) of i (pi/2) m e^{2 pi i m n/(4N)} sum to
    -pi m sin(2 pi m n/(4N)); m = 0 contributes nothing and the Nyquist m = -2N is
    zeroed.  S[n, m] for n in [0, N], m in [0, 2N], including 1/(4N)."""
    n = np.arange(N + 1)[:, None]
    m = np.arange(2 * N + 1)[None, :]
    S = -np.pi * m * np.sin(2 * np.pi * np.mod(n * m, 4 * N) / (4 * N)) / (4 * N)
    S[:, 2 * N] = 0.0
    return S


def T_octant_by_sums(d: int, N: int, kernel: str, k: float, L: float, deriv_axis=None,
                     Goct: np.ndarray | None = None) -> np.ndarray:
    """T (or T_j) for n in [0, N]^d by separable cosine (sine on axis j) sums."""
    x = spectrum_octant(d, N, kernel, k, L) if Goct is None else Goct
    C, S = cos_matrix_4n(N), sin_matrix_4n(N)
    for ax in range(d):
        x = _apply_axis(S if ax == deriv_axis else C, x, ax)
    return x


def ghat_octant_by_sums(T_oct: np.ndarray, N: int, odd_axis=None) -> np.ndarray:
    """Multiplier at m in [0, N]^d from the kernel octant.
    Even axis: sum over n in (-N, N] of T(n) e^{-i pi m n/N} = sum_{n=0}^{N} c'(n)
    cos(pi m n/N) T(n), c' = 1 at 0 and N, else 2.
    Odd axis (T_j(N) := 0): -2i sum_{n=1}^{N-1} T_j(n) sin(pi m n/N)."""
    d = T_oct.ndim
    n = np.arange(N + 1)[None, :]
    m = np.arange(N + 1)[:, None]
    cp = np.where((n == 0) | (n == N), 1.0, 2.0)
    Cm = cp * np.cos(np.pi * np.mod(m * n, 2 * N) / N)
    Sm = 2.0 * np.sin(np.pi * np.mod(m * n, 2 * N) / N)
    Sm[:, 0] = 0.0
    Sm[:, N] = 0.0
    x = T_oct.astype(np.complex128)
    for ax in range(d):
        x = _apply_axis(Sm if ax == odd_axis else Cm, x, ax)
    if odd_axis is not None:
        x = -1j * x
    return x


# ---------------------------------------------------------------------------
# octant <-> full conversions
# ---------------------------------------------------------------------------

def T_full_from_octant(T_oct: np.ndarray, odd_axis=None) -> np.ndarray:
    """Offsets [-N, N]^d (index n + N) from the octant, by evenness (oddness on
    ``odd_axis``)."""
    d = T_oct.ndim
    N = T_oct.shape[0] - 1
    n = np.arange(-N, N + 1)
    out = T_oct[np.ix_(*([np.abs(n)] * d))].astype(np.complex128)
    if odd_axis is not None:
        shape = [1] * d
        shape[odd_axis] = 2 * N + 1
        out = out * np.sign(n).reshape(shape)
    return out


def ghat_full_from_octant(G_oct: np.ndarray, odd_axis=None) -> np.ndarray:
    """(2N)^d multiplier in natural storage order from its [0, N]^d octant."""
    d = G_oct.ndim
    N = G_oct.shape[0] - 1
    q = np.arange(2 * N)
    fold = np.minimum(q, 2 * N - q)
    out = G_oct[np.ix_(*([fold] * d))].astype(np.complex128)
    if odd_axis is not None:
        sgn = np.where(q < N, 1.0, -1.0)
        sgn[0] = 0.0
        sgn[N] = 0.0
        shape = [1] * d
        shape[odd_axis] = 2 * N
        out = out * sgn.reshape(shape)
    return out


def nystrom_block(T_oct: np.ndarray, rows, cols, odd_axis=None) -> np.ndarray:
    """The Nystrom matrix of the discretised volume integral (Section 4, the
    remark after the discrete convolution): A[i][j] = T(p_i - p'_j) for target
    nodes rows[i] and source nodes cols[j], flat C-order grid indices, by plain
    loops over the entries."""
    d = T_oct.ndim
    N = T_oct.shape[0] - 1
    shape = (N,) * d
    out = np.empty((len(rows), len(cols)), dtype=np.complex128)
    for i, r in enumerate(rows):
        p = np.unravel_index(int(r), shape)
        for j, c in enumerate(cols):
            q = np.unravel_index(int(c), shape)
            n = [int(a) - int(b) for a, b in zip(p, q)]
            v = complex(T_oct[tuple(abs(x) for x in n)])
            if odd_axis is not None:
                v *= np.sign(n[odd_axis])
            out[i, j] = v
    return out
