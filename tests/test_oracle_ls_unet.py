"""Pins of the oracle's Lippmann-Schwinger operator and solvers, and of the
FP64 U-Net reference used to check the GPU network (no GPU)."""
import itertools

import numpy as np
import pytest

from oracle import ls as LS
from oracle import unet as U
from paper_1604_03155_gb300 import inputs as I


@pytest.fixture(scope="module")
def small_problem():
    N, k = 8, 6.0
    q = I.ls_contrast(I.LS_TRAIN_SEED, N)
    return LS.LSProblem(N, k, q), I.plane_wave(N, k)


def test_dense_solve_and_gmres_agree(small_problem):
    prob, uinc = small_problem
    b = prob.rhs(uinc)
    ud = LS.dense_solve(prob, b)
    assert prob.residual(ud, b) < 1e-13
    ug, its, hist = LS.gmres(prob.op, b, tol=1e-12, restart=30)
    assert prob.residual(ug, b) < 1e-11
    assert np.linalg.norm((ug - ud).ravel()) / np.linalg.norm(ud.ravel()) < 1e-10
    assert hist[-1] < 1e-12 and its < 200


def test_gmres_estimates_are_the_minimal_krylov_residuals():
    """GMRES's defining property (Saad & Schultz 1986): after k steps from x = 0
    the residual is the smallest ||b - A x|| over x in span{b, A b, ..., A^{k-1} b},
    computed here by least squares on an orthonormalised Krylov matrix.  With a
    restart after m steps, the next cycle begins from the explicit residual,
    which equals the last estimate, and the minimisation restarts from there."""
    rng = np.random.default_rng(7)
    n = 40
    A = np.eye(n) + 0.4 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    mv = lambda x: A @ x
    bn = np.linalg.norm(b)

    def minres(r0, k):
        K = np.empty((n, k), dtype=np.complex128)
        v = r0.copy()
        for j in range(k):
            K[:, j] = v
            v = A @ v
        Q, _ = np.linalg.qr(K)
        y = np.linalg.lstsq(A @ Q, r0, rcond=None)[0]
        return np.linalg.norm(r0 - A @ Q @ y), Q @ y

    _, its, hist = LS.gmres(mv, b, tol=1e-14, restart=60, maxit=12)
    assert its == 12 and hist[0] == 1.0
    for k in range(1, 13):
        assert abs(hist[k] - minres(b, k)[0] / bn) <= 1e-9 * hist[k], k
    x, _, hist = LS.gmres(mv, b, tol=1e-14, restart=3, maxit=6)
    r3, x3 = minres(b, 3)
    assert abs(hist[3] - r3 / bn) <= 1e-9 * hist[3]
    assert abs(hist[4] - hist[3]) <= 1e-9 * hist[3]  # the explicit residual of the restart
    r6, e3 = minres(b - A @ x3, 3)
    assert abs(hist[-1] - r6 / bn) <= 1e-9 * hist[-1]
    assert np.linalg.norm(x - (x3 + e3)) <= 1e-9 * np.linalg.norm(x)


def test_arnoldi_basis_pinned_by_qr_of_the_krylov_matrix(small_problem):
    """The Arnoldi vectors are the Q factor of [b, A b, ..., A^m b] (unique up to
    a unit phase per column, fixed by h_{j+1,j} > 0) and satisfy A V_m = V_{m+1} H."""
    prob, uinc = small_problem
    b = prob.rhs(uinc)
    m = 6
    V, H = LS.arnoldi(prob.op, b, m)
    n = b.size
    K = np.empty((n, m + 1), dtype=np.complex128)
    x = b.copy()
    for j in range(m + 1):
        K[:, j] = x.ravel()
        x = prob.op(x)
    Q, R = np.linalg.qr(K)  # Householder QR (LAPACK), an independent route
    Vm = V.reshape(m + 1, n).T
    phase = np.diag(Q.conj().T @ Vm)
    assert np.allclose(np.abs(phase), 1.0, atol=1e-6)
    # the monomial basis is ill-conditioned (the QR route loses ~30x per column),
    # so the bound is loose; a wrong sign, index or projection gives O(1) errors
    assert np.abs(Vm - Q * phase).max() < 1e-5
    assert np.abs(Vm.conj().T @ Vm - np.eye(m + 1)).max() < 1e-12
    AV = np.stack([prob.op(V[j]).ravel() for j in range(m)], axis=1)
    assert np.abs(AV - Vm @ H).max() < 1e-12 * np.abs(AV).max()
    assert np.all(np.diag(H, -1).real > 0) and np.all(np.diag(H, -1).imag == 0)
    assert np.all(np.tril(H, -2) == 0)


def test_lippmann_schwinger_limits(small_problem):
    prob, uinc = small_problem
    # no contrast: no scattered field
    zero = LS.LSProblem(prob.N, prob.k, np.zeros_like(prob.q))
    b0 = zero.rhs(uinc)
    assert np.abs(b0).max() == 0.0
    # weak contrast: Born approximation u ~ b, error O(q^2)
    for eps in (1e-3, 1e-4):
        weak = LS.LSProblem(prob.N, prob.k, eps * prob.q)
        bw = weak.rhs(uinc)
        uw = LS.dense_solve(weak, bw)
        born_err = np.linalg.norm((uw - bw).ravel()) / np.linalg.norm(uw.ravel())
        assert born_err < 50 * eps  # first-order correction relative to the O(eps) field
    # the operator is I - k^2 V q: applying it to the solution reproduces b
    b = prob.rhs(uinc)
    u = LS.dense_solve(prob, b)
    assert np.allclose(u - prob.k ** 2 * prob.V(prob.q * u), b, atol=1e-13 * np.abs(b).max())


def test_contrast_and_incident_field():
    q = I.ls_contrast(I.LS_TRAIN_SEED + 3, 32)
    assert q.shape == (32, 32, 32) and abs(q.max() - 0.5) < 0.3 and q.min() > -0.3
    b = I.cube_bump(32)
    assert abs(b[15, 15, 15] - 1.0) < 1e-15 and b[0, 0, 0] < 1e-6
    u = I.plane_wave(16, 30.0)
    x = I.grid_coords(16)
    assert np.allclose(u[:, 3, 7], np.exp(30j * x)) and np.allclose(np.abs(u), 1.0)


# ---------------------------------------------------------------------------
# U-Net reference
# ---------------------------------------------------------------------------

def _conv_literal(x, w, b):
    Ci, S = x.shape[0], x.shape[1]
    y = np.zeros((w.shape[0], S, S, S))
    for co in range(w.shape[0]):
        for z, yy, xx in itertools.product(range(S), repeat=3):
            acc = b[co]
            for ci in range(Ci):
                for o, (kz, ky, kx) in enumerate(U.OFFSETS):
                    pz, py, px = z + kz - 1, yy + ky - 1, xx + kx - 1
                    if 0 <= pz < S and 0 <= py < S and 0 <= px < S:
                        acc += w[co, ci, o] * x[ci, pz, py, px]
            y[co, z, yy, xx] = acc
    return y


def test_conv_matches_literal_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 4, 4, 4))
    w = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    assert np.abs(U.conv3d(x, w, b) - _conv_literal(x, w, b)).max() < 1e-12


def test_adjoint_pairs():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 8, 8, 8))
    y4 = rng.standard_normal((2, 4, 4, 4))
    assert np.isclose(np.sum(U.pool(x) * y4), np.sum(x * U.pool_back(y4)))
    y8 = rng.standard_normal((2, 8, 8, 8))
    assert np.isclose(np.sum(U.up(y4) * y8), np.sum(y4 * U.up_back(y8)))
    w = rng.standard_normal((3, 2, 27))
    dy = rng.standard_normal((3, 8, 8, 8))
    dx, dw, db = U.conv3d_backward(x, w, dy)
    assert np.isclose(np.sum(U.conv3d(x, w, np.zeros(3)) * dy), np.sum(x * dx))


def test_backward_against_finite_differences():
    C, S = 4, 8
    params = U.init_params(I.BASE_SEED + 77, C=C)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, S, S, S))
    target = rng.standard_normal((2, S, S, S))
    L, grads = U.loss_and_grads(params, x, target)
    for layer in range(10):
        dw = grads[layer][0].ravel()
        for idx in (0, 7, dw.size - 1):
            fd = U.grad_fd(params, x, target, layer, idx)
            assert abs(fd - dw[idx]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (layer, idx, fd, dw[idx])
    # input gradient
    out, cache = U.forward(params, x)
    _, dout = U.mse(out, target)
    _, dx = U.backward(params, cache, dout)
    h = 1e-6
    for idx in [(0, 1, 2, 3), (2, 7, 0, 5)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (U.mse(U.forward(params, xp)[0], target)[0] - U.mse(U.forward(params, xm)[0], target)[0]) / (2 * h)
        assert abs(fd - dx[idx]) <= 1e-6 * max(1e-3, abs(fd))


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 3.14159265, -2.5e-3], dtype=np.float32)
    r = I.bf16_round(x)
    assert r[0] == 1.0 and r[2] == 1.0  # ties to even
    assert r[1] == np.float32(1.0 + 2 ** -7) or r[1] == 1.0
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8)
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)
