"""Per-axis grid sizes (N_0, N_1[, N_2]), oracle side, float64.  TEST
INFRASTRUCTURE ONLY.

The box stays [-1/2, 1/2]^d and axis j has N_j points, h_j = 1/N_j.  Section 4's
construction carries over axis by axis: the spectrum is sampled at
s_m = (pi/2) m on the per-axis 4N_j grids (the frequency step 2 pi/(4 N_j h_j)
is pi/2 on every axis), so

    T(n) = prod_j (4 N_j)^{-1} sum_m G^L(|s_m|) exp(2 pi i sum_j m_j n_j/(4 N_j)),

m_j in [-2N_j, 2N_j), n_j in [-N_j, N_j]; the multiplier is the prod_j (2N_j)
point DFT of T cropped to (-N_j, N_j] per axis.  Each routine reuses the
isotropic one-axis factors of ``oracle.kernel`` with that axis's N_j.
"""
from __future__ import annotations

import numpy as np

from . import fft as offt
from . import kernel as K
from .spectrum import G_truncated


def spectrum_4n(Ns, kernel: str, k: float, L: float) -> np.ndarray:
    """G^L(|s_m|) on the full prod (4 N_j) grid in DFT storage order."""
    d = len(Ns)
    m2 = np.zeros(tuple(4 * N for N in Ns))
    for j, N in enumerate(Ns):
        shape = [1] * d
        shape[j] = 4 * N
        m2 = m2 + (K.signed_freq(4 * N).astype(np.float64) ** 2).reshape(shape)
    return G_truncated(d, kernel, k, L, (0.5 * np.pi * np.sqrt(m2)).ravel()).reshape(m2.shape)


def T_by_fft(Ns, kernel: str, k: float, L: float, deriv_axis=None) -> np.ndarray:
    """T (or T_j) on offsets prod [-N_j, N_j], index n + N_j, by the inverse DFT."""
    d = len(Ns)
    G4 = spectrum_4n(Ns, kernel, k, L)
    if deriv_axis is not None:
        N = Ns[deriv_axis]
        m = K.signed_freq(4 * N).astype(np.float64)
        m[m == -2 * N] = 0.0
        shape = [1] * d
        shape[deriv_axis] = 4 * N
        G4 = G4 * (1j * 0.5 * np.pi * m).reshape(shape)
    t = offt.ifftn(G4)
    return t[np.ix_(*[np.arange(-N, N + 1) % (4 * N) for N in Ns])]


def ghat_by_fft(T_full: np.ndarray, Ns, odd_axis=None) -> np.ndarray:
    """prod (2 N_j) multiplier: the DFT of T cropped to (-N_j, N_j] per axis."""
    idx = []
    for N in Ns:
        off = K.signed_freq(2 * N)
        off[N] = N
        idx.append(off + N)
    t = T_full[np.ix_(*idx)].copy()
    if odd_axis is not None:
        sl = [slice(None)] * len(Ns)
        sl[odd_axis] = Ns[odd_axis]
        t[tuple(sl)] = 0.0
    return offt.fftn(t)


def spectrum_octant(Ns, kernel: str, k: float, L: float) -> np.ndarray:
    """G^L(|s_m|) for m in prod [0, 2N_j]."""
    d = len(Ns)
    msq = np.zeros(tuple(2 * N + 1 for N in Ns), dtype=np.int64)
    for j, N in enumerate(Ns):
        shape = [1] * d
        shape[j] = 2 * N + 1
        msq = msq + (np.arange(2 * N + 1, dtype=np.int64) ** 2).reshape(shape)
    vals, inv = np.unique(msq, return_inverse=True)
    return G_truncated(d, kernel, k, L, 0.5 * np.pi * np.sqrt(vals.astype(np.float64)))[inv].reshape(msq.shape)


def T_octant_by_sums(Ns, kernel: str, k: float, L: float, deriv_axis=None) -> np.ndarray:
    """T (or T_j) for n in prod [0, N_j] by separable cosine (sine on axis j) sums."""
    x = spectrum_octant(Ns, kernel, k, L)
    for ax, N in enumerate(Ns):
        x = K._apply_axis(K.sin_matrix_4n(N) if ax == deriv_axis else K.cos_matrix_4n(N), x, ax)
    return x


def ghat_octant_by_sums(T_oct: np.ndarray, odd_axis=None) -> np.ndarray:
    """Multiplier at m in prod [0, N_j] from the kernel octant (per-axis factors
    of ``oracle.kernel.ghat_octant_by_sums``)."""
    x = T_oct.astype(np.complex128)
    for ax in range(T_oct.ndim):
        N = T_oct.shape[ax] - 1
        n = np.arange(N + 1)[None, :]
        m = np.arange(N + 1)[:, None]
        if ax == odd_axis:
            M = 2.0 * np.sin(np.pi * np.mod(m * n, 2 * N) / N)
            M[:, 0] = 0.0
            M[:, N] = 0.0
        else:
            M = np.where((n == 0) | (n == N), 1.0, 2.0) * np.cos(np.pi * np.mod(m * n, 2 * N) / N)
        x = K._apply_axis(M, x, ax)
    if odd_axis is not None:
        x = -1j * x
    return x


def ghat_full_from_octant(G_oct: np.ndarray, odd_axis=None) -> np.ndarray:
    """prod (2 N_j) multiplier in natural storage order from its octant."""
    idx = []
    for ax in range(G_oct.ndim):
        N = G_oct.shape[ax] - 1
        q = np.arange(2 * N)
        idx.append(np.minimum(q, 2 * N - q))
    out = G_oct[np.ix_(*idx)].astype(np.complex128)
    if odd_axis is not None:
        N = G_oct.shape[odd_axis] - 1
        q = np.arange(2 * N)
        sgn = np.where(q < N, 1.0, -1.0)
        sgn[0] = 0.0
        sgn[N] = 0.0
        shape = [1] * G_oct.ndim
        shape[odd_axis] = 2 * N
        out = out * sgn.reshape(shape)
    return out


def apply_fft2n(G_full: np.ndarray, f: np.ndarray) -> np.ndarray:
    """phi = crop(IDFT(G * DFT(zero-pad f))) on the per-axis 2N_j grid."""
    pad = np.zeros(G_full.shape, dtype=np.complex128)
    pad[tuple(slice(0, n) for n in f.shape)] = f
    out = offt.ifftn(G_full * offt.fftn(pad))
    return out[tuple(slice(0, n) for n in f.shape)]


def apply_direct(T_full: np.ndarray, f: np.ndarray) -> np.ndarray:
    """phi_p = sum_{p'} T(p - p') f_{p'} by brute force (T_full indexed n + N_j)."""
    phi = np.zeros(f.shape, dtype=np.complex128)
    for src in np.ndindex(*f.shape):
        fv = f[src]
        if fv == 0:
            continue
        sl = tuple(slice(N - s, 2 * N - s) for s, N in zip(src, f.shape))
        phi += T_full[sl] * fv
    return phi


def grid(Ns):
    """The per-axis coordinates x_p = (p - N/2 + 1)/N as an open meshgrid."""
    from paper_1604_03155_gb300 import inputs as I
    return np.meshgrid(*[I.grid_coords(N) for N in Ns], indexing="ij")
