"""Pins of the oracle's volume potential (Section 4) and gradients: brute force
against both FFT forms, operator invariants, and superalgebraic convergence to
the Gaussian closed forms of Section 5.1 (no GPU)."""
import math

import numpy as np
import pytest

from oracle import apply as A
from oracle import closed_forms as CF
from oracle import kernel as K
from paper_1604_03155_gb300 import inputs as I

CASES = [(3, "laplace", 0.0, 1.8, 6), (3, "helmholtz", 13.0, 1.8, 8), (2, "laplace", 0.0, 1.5, 12),
         (2, "helmholtz", 30.0, 1.5, 16), (3, "biharmonic", 0.0, 1.8, 6), (2, "biharmonic", 0.0, 1.5, 12)]


def _setup(d, kernel, k, L, N):
    Tf = K.T_by_fft(d, N, kernel, k, L)
    return Tf, K.ghat_by_fft(Tf, N)


@pytest.mark.parametrize("d,kernel,k,L,N", CASES)
def test_three_forms_agree(d, kernel, k, L, N):
    Tf, G = _setup(d, kernel, k, L, N)
    f = I.random_complex_field(11, (N,) * d)
    ref = A.apply_direct(Tf, f)
    assert A.rel_l2(A.apply_fft2n(G, f), ref) < 1e-14
    G4 = K.spectrum_4n(d, N, kernel, k, L)
    assert A.rel_l2(A.apply_fft4n(G4, f), ref) < 1e-14
    pts = [(0,) * d, (N - 1,) * d, tuple(range(d))]
    assert np.abs(A.apply_direct_at(Tf, f, pts) - np.array([ref[p] for p in pts])).max() < 1e-14 * np.abs(ref).max()
    # the pointwise sum from the octant (the full-size sampled form): every node
    allp = list(np.ndindex(*f.shape))
    Toct = Tf[(slice(N, None),) * d]
    assert np.abs(A.apply_direct_at_octant(Toct, f, allp) - ref.ravel()).max() < 1e-14 * np.abs(ref).max()
    for j in range(d):
        Tj = K.T_by_fft(d, N, kernel, k, L, deriv_axis=j)
        gref = A.apply_direct(Tj, f)
        got = A.apply_direct_at_octant(Tj[(slice(N, None),) * d], f, allp, odd_axis=j)
        assert np.abs(got - gref.ravel()).max() < 1e-14 * np.abs(gref).max()
        assert A.rel_l2(A.apply_fft2n(K.ghat_by_fft(Tj, N, odd_axis=j), f), gref) < 1e-14
        assert A.rel_l2(A.apply_fft4n(G4, f, deriv_axis=j), gref) < 1e-14


@pytest.mark.parametrize("d,kernel,k,L,N", CASES)
def test_operator_invariants(d, kernel, k, L, N):
    Tf, G = _setup(d, kernel, k, L, N)
    f = I.random_complex_field(12, (N,) * d)
    g = I.random_complex_field(13, (N,) * d)
    Af, Ag = A.apply_fft2n(G, f), A.apply_fft2n(G, g)
    # linearity
    assert A.rel_l2(A.apply_fft2n(G, 2.5 * f - 1j * g), 2.5 * Af - 1j * Ag) < 1e-14
    # complex symmetry of the convolution with an even kernel: <g, A f> = <f, A g> (bilinear)
    assert abs(np.sum(g * Af) - np.sum(f * Ag)) < 1e-13 * np.abs(Af).sum()
    # reflection covariance in every axis and axis permutation
    for ax in range(d):
        assert A.rel_l2(A.apply_fft2n(G, np.flip(f, ax)), np.flip(Af, ax)) < 1e-14
    assert A.rel_l2(A.apply_fft2n(G, np.swapaxes(f, 0, 1)), np.swapaxes(Af, 0, 1)) < 1e-14
    # translation covariance on the overlap (shift by one node along axis 0)
    fs = np.zeros_like(f)
    f0 = f.copy()
    f0[-1] = 0
    fs[1:] = f0[:-1]
    A0, As = A.apply_fft2n(G, f0), A.apply_fft2n(G, fs)
    assert np.abs(As[1:] - A0[:-1]).max() < 1e-14 * np.abs(A0).max()


def test_laplace_real_and_positive_semidefinite():
    N = 8
    Tf, G = _setup(3, "laplace", 0.0, 1.8, N)
    f = I.random_complex_field(14, (N,) * 3).real
    phi = A.apply_fft2n(G, f)
    assert np.abs(phi.imag).max() < 1e-14 * np.abs(phi).max()
    assert np.sum(f * phi.real) > 0
    # principal block of a PSD circulant: smallest eigenvalue of the explicit matrix >= 0
    n = 4
    Tf4 = K.T_by_fft(3, n, "laplace", 0.0, 1.8)
    idx = list(np.ndindex(n, n, n))
    M = np.array([[Tf4[tuple(np.array(p) - np.array(q) + n)].real for q in idx] for p in idx])
    assert np.allclose(M, M.T)
    assert np.linalg.eigvalsh(M).min() > -1e-15 * np.abs(M).max()


def test_2n_gradient_mode_agrees_with_exact_for_centred_source():
    """Both gradient modes approximate the same derivative when the source is
    negligible at the box edge (Section 3, spectral differentiation)."""
    N = 32
    Tf, G = _setup(3, "laplace", 0.0, 1.8, N)
    f = I.workload("laplace3d_single_gaussian").density(N)
    g2 = A.grad_spectral2n(G, f)
    for j in range(3):
        Tj = K.T_by_fft(3, N, "laplace", 0.0, 1.8, deriv_axis=j)
        ge = A.apply_fft2n(K.ghat_by_fft(Tj, N, odd_axis=j), f)
        assert A.rel_l2(g2[j], ge) < 1e-7


def _grid_r(N, d):
    x = I.grid_coords(N)
    X = np.meshgrid(*([x] * d), indexing="ij")
    return X, np.sqrt(sum(a * a for a in X))


def test_superalgebraic_convergence_laplace3d_erf():
    """The 3D Laplace Gaussian (sigma = 0.08, unnormalised exp(-r^2/sigma^2)):
    error vs the erf closed form falls faster than any power of h (Section 5.1)."""
    errs = {}
    for N in (8, 16, 24, 32):
        To = K.T_octant_by_sums(3, N, "laplace", 0.0, 1.8)
        G = K.ghat_full_from_octant(K.ghat_octant_by_sums(To, N))
        f = I.workload("laplace3d_single_gaussian").density(N)
        _, r = _grid_r(N, 3)
        ex = I.gaussian_amplitude(0.08, 3) * CF.laplace3(r, 0.08 / math.sqrt(2))
        errs[N] = A.rel_l2(A.apply_fft2n(G, f), ex)
    assert errs[32] < 1e-10
    assert errs[16] / errs[32] > 1e5  # far steeper than any fixed low order
    assert errs[8] > errs[16] > errs[24] > errs[32]


def test_laplace3d_exact_gradient_vs_analytic():
    N = 32
    sig = 0.08 / math.sqrt(2)
    Q = I.gaussian_amplitude(0.08, 3)
    f = I.workload("laplace3d_single_gaussian").density(N)
    X, r = _grid_r(N, 3)
    rs = np.where(r == 0, 1.0, r)
    dr = np.where(r == 0, 0.0, Q * CF.laplace3_dr(rs, sig))
    for j in range(3):
        Tj = K.T_by_fft(3, N, "laplace", 0.0, 1.8, deriv_axis=j)
        gj = A.apply_fft2n(K.ghat_by_fft(Tj, N, odd_axis=j), f)
        ex = dr * X[j] / rs
        assert A.rel_l2(gj, ex) < 1e-7


@pytest.mark.parametrize("d,kernel,k,N,tol", [(3, "helmholtz", 2.0, 40, 1e-9), (2, "laplace", 0.0, 64, 1e-9),
                                              (2, "helmholtz", 2.0, 64, 1e-9), (3, "biharmonic", 0.0, 40, 1e-9),
                                              (2, "biharmonic", 0.0, 64, 1e-9)])
def test_convergence_to_corrected_closed_forms(d, kernel, k, N, tol):
    """Fig. 3's test (sigma = 0.05, k = 2) with the corrected closed forms; a
    sign, a missing i or a wrong special function would fail at O(1)."""
    sig = 0.05
    L = 1.8 if d == 3 else 1.5
    To = K.T_octant_by_sums(d, N, kernel, k, L)
    G = K.ghat_full_from_octant(K.ghat_octant_by_sums(To, N))
    X, r = _grid_r(N, d)
    rho = (2 * math.pi * sig * sig) ** (-d / 2) * np.exp(-r * r / (2 * sig * sig))
    phi = A.apply_fft2n(G, rho)
    if kernel == "biharmonic":
        ex = CF.biharmonic3(r, sig) if d == 3 else CF.biharmonic2(r, sig)
    elif d == 3:
        ex = CF.helmholtz3(r, sig, k)
    elif kernel == "laplace":
        ex = CF.laplace2(r, sig)
    else:
        # quadrature closed form on the distinct radii only
        ru, inv = np.unique(np.round(r, 14), return_inverse=True)
        ex = CF.helmholtz2(ru, sig, k)[inv].reshape(r.shape)
    assert A.rel_l2(phi, ex) < tol
