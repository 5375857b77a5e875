"""Pins of the per-axis grid oracle (no GPU): the cubic case equals the
isotropic oracle, the two routes to T and the multiplier agree, brute force
equals the FFT apply, and a Gaussian source converges to its closed-form
potential on an anisotropic grid."""
import math

import numpy as np
import pytest

from oracle import aniso as AN
from oracle import apply as A
from oracle import closed_forms as CF
from oracle import kernel as K
from paper_1604_03155_gb300 import inputs as I


def test_cubic_case_equals_the_isotropic_oracle():
    for d, N, kernel, k, L in [(3, 6, "helmholtz", 9.0, 1.8), (2, 8, "laplace", 0.0, 1.5)]:
        Ns = (N,) * d
        assert np.array_equal(AN.T_octant_by_sums(Ns, kernel, k, L), K.T_octant_by_sums(d, N, kernel, k, L))
        T = K.T_octant_by_sums(d, N, kernel, k, L)
        assert np.allclose(AN.ghat_octant_by_sums(T), K.ghat_octant_by_sums(T, N), rtol=0, atol=1e-15)


@pytest.mark.parametrize("Ns,kernel,k,L", [((4, 6, 8), "helmholtz", 7.0, 1.8), ((6, 4), "laplace", 0.0, 1.5),
                                           ((4, 8, 6), "laplace", 0.0, 1.8)])
def test_two_routes_and_brute_force(Ns, kernel, k, L):
    d = len(Ns)
    Tf = AN.T_by_fft(Ns, kernel, k, L)
    To = AN.T_octant_by_sums(Ns, kernel, k, L)
    assert np.abs(Tf[tuple(slice(N, None) for N in Ns)] - To).max() < 1e-14 * np.abs(To).max()
    G = AN.ghat_octant_by_sums(To)
    Gfull = AN.ghat_full_from_octant(G)
    assert np.abs(AN.ghat_by_fft(Tf, Ns) - Gfull).max() < 1e-13 * np.abs(Gfull).max()
    f = I.random_complex_field(31, Ns)
    ref = AN.apply_direct(Tf, f)
    assert A.rel_l2(AN.apply_fft2n(Gfull, f), ref) < 1e-14
    # derivative kernel along the last axis
    j = d - 1
    Tjf = AN.T_by_fft(Ns, kernel, k, L, deriv_axis=j)
    Tjo = AN.T_octant_by_sums(Ns, kernel, k, L, deriv_axis=j)
    assert np.abs(Tjf[tuple(slice(N, None) for N in Ns)] - Tjo).max() < 1e-14 * np.abs(Tjo).max()
    Gj = AN.ghat_full_from_octant(AN.ghat_octant_by_sums(Tjo, odd_axis=j), odd_axis=j)
    assert A.rel_l2(AN.apply_fft2n(Gj, f), AN.apply_direct(Tjf, f)) < 1e-13


def test_gaussian_closed_form_on_an_anisotropic_grid():
    """3D Laplace, unit-mass Gaussian sigma = 0.05 on 20 x 24 x 32 and
    40 x 48 x 64: spectral convergence to erf(r/(sqrt 2 s))/(4 pi r)."""
    s = 0.05
    errs = []
    for Ns in [(20, 24, 32), (40, 48, 64)]:
        X = AN.grid(Ns)
        r = np.sqrt(sum(x * x for x in X))
        rho = (2 * math.pi * s * s) ** -1.5 * np.exp(-r * r / (2 * s * s))
        G = AN.ghat_full_from_octant(AN.ghat_octant_by_sums(AN.T_octant_by_sums(Ns, "laplace", 0.0, 1.8)))
        errs.append(A.rel_l2(AN.apply_fft2n(G, rho), CF.laplace3(r, s)))
    assert errs[1] < 1e-10 and errs[0] > 100 * errs[1]
