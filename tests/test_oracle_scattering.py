"""Pins of the oracle's scattering pieces of Section 5.3 (no GPU): the paper's
contrasts, textbook Bi-CGStab, and the field and density forms of the
Lippmann-Schwinger equation."""
import numpy as np
import pytest

from oracle import ls as LS
from paper_1604_03155_gb300 import inputs as I


def test_paper_contrasts_closed_forms():
    N = 40
    x = I.grid_coords(N)
    disk, lens = I.filtered_disk(N), I.luneburg_lens(N)
    assert disk.shape == lens.shape == (N, N)
    c = N // 2 - 1  # x = 0
    assert x[c] == 0.0
    assert disk[c, c] == 1.0 and lens[c, c] == 1.0
    # the filtered disk at |x| = 0.25 (grid point x = 0.25 on the axis): exp(-1/2)
    j = int(np.argmin(np.abs(x - 0.25)))
    assert x[j] == 0.25
    assert disk[j, c] == pytest.approx(np.exp(-0.5), rel=1e-15)
    # the lens: 1 - (r/0.45)^2 inside, zero at and beyond r = 0.45
    r = np.sqrt(x[:, None] ** 2 + x[None, :] ** 2)
    inside = r < 0.45
    assert np.allclose(lens[inside], 1 - (r[inside] / 0.45) ** 2, rtol=0, atol=1e-15)
    assert np.all(lens[~inside] == 0.0) and lens.min() >= 0.0
    # radial symmetry under the grid's reflections about x = 0 (grid points -x exist for |x| < 1/2)
    assert np.array_equal(disk[c - 5, c + 3], disk[c + 5, c - 3])
    # the smoothed cube of the 3D example and the 2D plane wave
    cube = I.cube_bump(8)
    assert cube.shape == (8, 8, 8) and cube.max() <= 1.0
    pw = I.plane_wave(N, 7.0, d=2)
    assert pw.shape == (N, N) and np.allclose(pw[:, 3], np.exp(1j * 7.0 * x))


def test_bicgstab_scalar_multiple_of_identity_stops_at_the_first_half_step():
    b = np.arange(1, 7) + 1j * np.arange(6)
    c = 2.5 - 0.5j
    x, its, mv, hist = LS.bicgstab(lambda v: c * v, b, tol=1e-14)
    assert its == 1 and mv == 1 and len(hist) == 2
    assert np.allclose(x, b / c, rtol=1e-15, atol=0)


def test_bicgstab_terminates_in_as_many_steps_as_distinct_eigenvalues():
    """Bi-CGStab's residual is psi_j(A) phi_j(A) r_0 with phi_j the Bi-CG
    polynomial, which vanishes on r_0 after m steps when A has m distinct
    eigenvalues (exact arithmetic): a wrong alpha, omega or beta breaks it."""
    rng = np.random.default_rng(7)
    n = 12
    S = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    lam = np.repeat([1.0 + 0.5j, 2.0 - 1.0j, 0.5 + 0.2j], n // 3)
    M = S @ np.diag(lam) @ np.linalg.inv(S)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, its, mv, hist = LS.bicgstab(lambda v: M @ v, b, tol=1e-10)
    assert its <= 3
    assert np.linalg.norm(M @ x - b) / np.linalg.norm(b) < 1e-9
    # a generic matrix needs many more
    G = np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    x, its, mv, hist = LS.bicgstab(lambda v: G @ v, b, tol=1e-12)
    assert its > 3 and np.linalg.norm(G @ x - b) / np.linalg.norm(b) < 1e-11
    assert mv in (2 * its, 2 * its - 1)


@pytest.fixture(scope="module")
def problems():
    out = {}
    for name, d, N, size in [("disk", 2, 16, 2.0), ("lens", 2, 16, 2.0), ("cube", 3, 8, 1.0)]:
        q = {"disk": I.filtered_disk, "lens": I.luneburg_lens, "cube": I.cube_bump}[name](N)
        k = 2 * np.pi * size
        out[name] = (LS.LSProblem(N, k, q), I.plane_wave(N, k, d))
    return out


@pytest.mark.parametrize("name", ["disk", "lens", "cube"])
def test_field_and_density_forms_give_the_same_scattered_field(problems, name):
    """u solves A u = k^2 V[q u_inc] and s solves B s = k^2 q u_inc; then
    u = V[s] (s = k^2 q (u + u_inc) is the density of the scattered field)."""
    prob, uinc = problems[name]
    u = LS.dense_solve(prob, prob.rhs(uinc))
    s = LS.dense_solve(prob, prob.rhs_density(uinc), form="density")
    assert np.linalg.norm((prob.V(s) - u).ravel()) / np.linalg.norm(u.ravel()) < 1e-12
    assert np.allclose(s, prob.k ** 2 * prob.q * (u + uinc), rtol=0, atol=1e-11 * np.abs(s).max())


@pytest.mark.parametrize("name", ["disk", "lens", "cube"])
@pytest.mark.parametrize("form", ["field", "density"])
def test_bicgstab_reaches_the_dense_solution(problems, name, form):
    prob, uinc = problems[name]
    op = prob.op if form == "field" else prob.op_density
    b = prob.rhs(uinc) if form == "field" else prob.rhs_density(uinc)
    xd = LS.dense_solve(prob, b, form=form)
    x, its, mv, hist = LS.bicgstab(op, b, tol=1e-13)
    assert hist[-1] < 1e-13 and mv in (2 * its, 2 * its - 1)
    assert np.linalg.norm((x - xd).ravel()) / np.linalg.norm(xd.ravel()) < 1e-11
