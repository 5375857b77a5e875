"""Pins of the discrete kernel T, derivative kernels T_j and the (2N)^d
multipliers of Section 4 (no GPU)."""
import itertools

import numpy as np
import pytest

from oracle import kernel as K
from oracle import spectrum as S

CASES = [(3, "laplace", 0.0, 1.8, 4), (3, "helmholtz", 9.0, 1.8, 6), (2, "laplace", 0.0, 1.5, 8),
         (2, "helmholtz", 20.0, 1.5, 10)]


def _T_literal(d, N, kernel, k, L, n, deriv_axis=None):
    """T(n) by the triple/double sum over m in [-2N, 2N)^d exactly as written."""
    M = 4 * N
    acc = 0j
    for m in itertools.product(range(-2 * N, 2 * N), repeat=d):
        s = 0.5 * np.pi * np.sqrt(sum(mi * mi for mi in m))
        g = S.G_truncated(d, kernel, k, L, np.array([s]))[0]
        if deriv_axis is not None:
            mj = m[deriv_axis]
            g = g * (0 if mj == -2 * N else 1j * 0.5 * np.pi * mj)
        acc += g * np.exp(2j * np.pi * sum(a * b for a, b in zip(m, n)) / M)
    return acc / M ** d


@pytest.mark.parametrize("d,kernel,k,L", [(3, "laplace", 0.0, 1.8), (3, "helmholtz", 5.0, 1.8),
                                          (2, "laplace", 0.0, 1.5), (2, "helmholtz", 7.0, 1.5)])
def test_T_against_literal_sum(d, kernel, k, L):
    N = 2
    Tf = K.T_by_fft(d, N, kernel, k, L)
    To = K.T_full_from_octant(K.T_octant_by_sums(d, N, kernel, k, L))
    for n in [(0,) * d, (1,) + (0,) * (d - 1), (2,) * d, (-1, 2) + (0,) * (d - 2)]:
        ref = _T_literal(d, N, kernel, k, L, n)
        idx = tuple(x + N for x in n)
        assert abs(Tf[idx] - ref) < 1e-14 * abs(Tf).max()
        assert abs(To[idx] - ref) < 1e-14 * abs(Tf).max()
    for j in range(d):
        Tjf = K.T_by_fft(d, N, kernel, k, L, deriv_axis=j)
        n = (1, -2) + (1,) * (d - 2)
        ref = _T_literal(d, N, kernel, k, L, n, deriv_axis=j)
        assert abs(Tjf[tuple(x + N for x in n)] - ref) < 1e-14 * abs(Tjf).max()


@pytest.mark.parametrize("d,kernel,k,L,N", CASES)
def test_two_routes_agree_and_symmetries(d, kernel, k, L, N):
    Tf = K.T_by_fft(d, N, kernel, k, L)
    To = K.T_octant_by_sums(d, N, kernel, k, L)
    scale = np.abs(Tf).max()
    assert np.abs(Tf - K.T_full_from_octant(To)).max() < 1e-14 * scale
    # even in every axis and invariant under axis permutations
    for ax in range(d):
        assert np.abs(Tf - np.flip(Tf, ax)).max() < 1e-15 * scale
    assert np.abs(Tf - np.swapaxes(Tf, 0, 1)).max() < 1e-15 * scale
    if kernel == "laplace":
        assert np.abs(Tf.imag).max() < 1e-14 * scale
    G = K.ghat_by_fft(Tf, N)
    Go = K.ghat_octant_by_sums(To, N)
    assert np.abs(G - K.ghat_full_from_octant(Go)).max() < 1e-14 * np.abs(G).max()
    for j in range(d):
        Tj = K.T_by_fft(d, N, kernel, k, L, deriv_axis=j)
        Tjo = K.T_octant_by_sums(d, N, kernel, k, L, deriv_axis=j)
        sj = np.abs(Tj).max()
        assert np.abs(Tj - K.T_full_from_octant(Tjo, odd_axis=j)).max() < 1e-14 * sj
        assert np.abs(Tj + np.flip(Tj, j)).max() < 1e-15 * sj  # odd in n_j
        other = (j + 1) % d
        assert np.abs(Tj - np.flip(Tj, other)).max() < 1e-15 * sj  # even elsewhere
        Gj = K.ghat_by_fft(Tj, N, odd_axis=j)
        Gjo = K.ghat_octant_by_sums(Tjo, N, odd_axis=j)
        assert np.abs(Gj - K.ghat_full_from_octant(Gjo, odd_axis=j)).max() < 1e-14 * np.abs(Gj).max()


def test_T_approximates_green_function_away_from_origin():
    """Section 4 (Fig. 2): T is a mollified Green's function; away from the
    origin T(n) ~ h^d g(|n| h) for a smooth density's quadrature weight."""
    N = 32
    To = K.T_octant_by_sums(3, N, "laplace", 0.0, 1.8)
    h = 1.0 / N
    for n in (8, 12, 16):
        g = 1.0 / (4 * np.pi * n * h)
        assert abs(To[n, 0, 0].real / h ** 3 - g) < 2e-2 * g
    # the on-diagonal entry stays finite (the naive rule would blow up)
    assert np.isfinite(To[0, 0, 0]) and 0 < To[0, 0, 0].real / h ** 3 < 10 / (4 * np.pi * h)


def test_multiplier_sum_rule():
    """sum over the (2N)^d multiplier equals (2N)^d T(0) (inverse DFT at offset 0)."""
    N = 6
    Tf = K.T_by_fft(2, N, "helmholtz", 11.0, 1.5)
    G = K.ghat_by_fft(Tf, N)
    assert abs(G.sum() / (2 * N) ** 2 - Tf[N, N]) < 1e-15 * abs(G).max()
