"""Pins of the oracle's variable-coefficient Poisson operator (Section 5.2,
eq. pbeq) and of the synthetic molecule inputs (no GPU)."""
import math

import numpy as np
import pytest

from oracle import closed_forms as CF
from oracle import ls as LS
from oracle import pb as PB
from paper_1604_03155_gb300 import inputs as I


def _manufactured(N, s=0.08):
    """sigma = the unit-mass Gaussian (width s) at the origin, whose potential
    phi = erf(r/(sqrt 2 s))/(4 pi r) is known in closed form; eps = 2 + a
    Gaussian bump; rho = -eps sigma + grad(eps) . grad(phi), all analytic."""
    x = I.grid_coords(N)
    X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt(sum(a * a for a in X))
    sig = (2 * math.pi * s * s) ** -1.5 * np.exp(-r * r / (2 * s * s))
    rs = np.where(r == 0, 1.0, r)
    dphi = np.where(r == 0, 0.0, CF.laplace3_dr(rs, s))
    c, w = np.array([0.1, -0.05, 0.08]), 0.15
    g = np.exp(-sum((X[j] - c[j]) ** 2 for j in range(3)) / w ** 2)
    eps = 2.0 + g
    ge = np.stack([-2 * (X[j] - c[j]) / w ** 2 * g for j in range(3)])
    rho = -eps * sig + sum(ge[j] * dphi * X[j] / rs for j in range(3))
    return eps, ge, rho, sig


@pytest.mark.parametrize("N,bar", [(16, 1e-5), (24, 1e-9)])
def test_manufactured_closed_form_solution(N, bar):
    """The solve recovers the analytic sigma to spectral accuracy (2.2e-6 at
    N = 16, 3.6e-11 at N = 24): the operator's -eps sigma, its grad(eps) term
    and the exact gradient kernels are checked against closed forms only."""
    eps, ge, rho, sig = _manufactured(N)
    prob = PB.PBProblem(N, eps, ge)
    x, its, mv, h = LS.bicgstab(prob.op, rho.astype(np.complex128), tol=1e-13)
    assert np.linalg.norm((x - sig).ravel()) / np.linalg.norm(sig.ravel()) < bar


def test_constant_eps_and_dense_solve():
    N = 8
    mol = I.pb_molecule()
    eps, ge, rho = (t.numpy() for t in I.pb_fields(mol, N))
    # constant eps: grad(eps) = 0 and sigma = -rho/eps exactly, at the first half step
    const = PB.PBProblem(N, np.full((N,) * 3, 3.0), np.zeros((3,) + (N,) * 3))
    b = I.random_complex_field(5, (N,) * 3)
    x, its, mv, h = LS.bicgstab(const.op, b, tol=1e-14)
    assert its == 1 and mv == 1 and np.allclose(x, -b / 3.0, rtol=1e-15, atol=0)
    # the molecule's operator: Bi-CGStab and GMRES reach the dense solution
    prob = PB.PBProblem(N, eps, ge)
    xd = PB.dense_solve(prob, rho)
    xb, its, mv, h = LS.bicgstab(prob.op, rho.astype(np.complex128), tol=1e-13)
    xg, itg, hg = LS.gmres(prob.op, rho.astype(np.complex128), tol=1e-13, restart=40)
    assert np.linalg.norm((xb - xd).ravel()) / np.linalg.norm(xd.ravel()) < 1e-11
    assert np.linalg.norm((xg - xd).ravel()) / np.linalg.norm(xd.ravel()) < 1e-11


def test_molecule_inputs():
    """The dielectric lies between eps_in and eps_out and equals eps_out far
    from the atoms; for one and two atoms eps, its gradient (product rule) and
    rho equal the closed forms of the recipe."""
    mol = I.pb_molecule()
    centres, charges = mol
    assert centres.shape == (I.PB_ATOMS, 3) and np.linalg.norm(centres, axis=1).max() < I.PB_BALL
    assert charges.min() >= -1 and charges.max() <= 1
    N = 48
    eps, ge, rho = (t.numpy() for t in I.pb_fields(mol, N))
    assert eps.min() >= I.PB_EPS_IN - 1e-12 and eps.max() <= I.PB_EPS_OUT + 1e-12
    assert eps[0, 0, 0] == I.PB_EPS_OUT and eps[-1, -1, -1] == I.PB_EPS_OUT
    # one atom alone: eps = eps_out + (eps_in - eps_out) alpha, rho = c alpha
    one = (np.array([[0.0, 0.0, 0.0]]), np.array([0.5]))
    e1, g1, r1 = (t.numpy() for t in I.pb_fields(one, 16))
    x = I.grid_coords(16)
    X = np.meshgrid(x, x, x, indexing="ij")
    a = np.exp(-sum(v * v for v in X) / (I.PB_MU2 * I.PB_RADIUS ** 2))
    a = np.where(np.sqrt(sum(v * v for v in X)) <= I.PB_CUTOFF * math.sqrt(I.PB_MU2) * I.PB_RADIUS, a, 0.0)
    assert np.allclose(e1, I.PB_EPS_OUT + (I.PB_EPS_IN - I.PB_EPS_OUT) * a, rtol=0, atol=1e-14)
    assert np.allclose(r1, 0.5 * a, rtol=0, atol=1e-15)
    # two overlapping atoms: q = 1 - (1 - a1)(1 - a2), grad q by the product rule
    two = (np.array([[0.0, 0.0, 0.0], [0.03, -0.02, 0.01]]), np.array([1.0, -1.0]))
    e2, g2, r2 = (t.numpy() for t in I.pb_fields(two, 32))
    x = I.grid_coords(32)
    X = np.meshgrid(x, x, x, indexing="ij")
    w2 = I.PB_MU2 * I.PB_RADIUS ** 2
    al, gal = [], []
    for c in two[0]:
        d = [X[j] - c[j] for j in range(3)]
        r2c = sum(v * v for v in d)
        ai = np.where(np.sqrt(r2c) <= I.PB_CUTOFF * math.sqrt(w2), np.exp(-r2c / w2), 0.0)
        al.append(ai)
        gal.append([-2 * d[j] / w2 * ai for j in range(3)])
    q = 1 - (1 - al[0]) * (1 - al[1])
    assert np.allclose(e2, q * I.PB_EPS_IN + (1 - q) * I.PB_EPS_OUT, rtol=0, atol=1e-14)
    for j in range(3):
        gq = gal[0][j] * (1 - al[1]) + gal[1][j] * (1 - al[0])
        assert np.allclose(g2[j], (I.PB_EPS_IN - I.PB_EPS_OUT) * gq, rtol=0, atol=1e-12 * np.abs(gq).max())
    assert np.allclose(r2, al[0] - al[1], rtol=0, atol=1e-15)


def _manufactured_2d(N, s=0.08):
    """2D: sigma = the unit-mass Gaussian, phi = -(E_1(r^2/2s^2) + log r^2)/(4 pi)
    (the corrected Section 5.1 form), grad phi = -(1 - e^{-r^2/2s^2})/(2 pi r) x/r
    (Gauss's law); eps = 2 + a Gaussian bump."""
    x = I.grid_coords(N)
    X = np.meshgrid(x, x, indexing="ij")
    r = np.sqrt(X[0] ** 2 + X[1] ** 2)
    sig = np.exp(-r * r / (2 * s * s)) / (2 * math.pi * s * s)
    rs = np.where(r == 0, 1.0, r)
    dphi = np.where(r == 0, 0.0, -(1 - np.exp(-rs * rs / (2 * s * s))) / (2 * math.pi * rs))
    c, w = np.array([0.1, -0.05]), 0.15
    g = np.exp(-((X[0] - c[0]) ** 2 + (X[1] - c[1]) ** 2) / w ** 2)
    eps = 2.0 + g
    ge = np.stack([-2 * (X[j] - c[j]) / w ** 2 * g for j in range(2)])
    rho = -eps * sig + sum(ge[j] * dphi * X[j] / rs for j in range(2))
    return eps, ge, rho, sig


def test_manufactured_closed_form_solution_2d():
    """The 2D operator recovers the analytic sigma to spectral accuracy, and
    the gradient closed form is the derivative of the Section 5.1 potential."""
    s = 0.08
    r = np.array([0.05, 0.1, 0.3])
    hstep = 1e-6
    fd = (CF.laplace2(r + hstep, s) - CF.laplace2(r - hstep, s)) / (2 * hstep)
    assert np.allclose(fd, -(1 - np.exp(-r * r / (2 * s * s))) / (2 * math.pi * r), rtol=1e-7)
    for N, bar in [(32, 1e-5), (64, 1e-10)]:
        eps, ge, rho, sig = _manufactured_2d(N, s)
        prob = PB.PBProblem(N, eps, ge)
        x, its, mv, h = LS.bicgstab(prob.op, rho.astype(np.complex128), tol=1e-13)
        assert np.linalg.norm((x - sig).ravel()) / np.linalg.norm(sig.ravel()) < bar, N
