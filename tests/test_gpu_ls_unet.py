"""Lippmann-Schwinger solve (flexible GMRES on the FP32 apply) and the learned
preconditioner network (the project's own conv3d forward/backward kernels)
against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import ls as OLS
from oracle import unet as OU
from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300 import vp
from paper_1604_03155_gb300.vp import Plan, UNet

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _weights(seed, C=16, bias_seed=None):
    layers = I.unet_init_weights(seed, C)
    out = []
    for i, (w, b) in enumerate(layers):
        if bias_seed is not None:
            b = (0.05 * I.normal(bias_seed + i, b.size)).astype(np.float32)
        out.append((I.bf16_round(w), I.bf16_round(b)))
    return out


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("S,slope", [(8, 0.1), (16, 0.1), (8, 1.0)])
def test_unet_forward_loss_and_gradients_match_oracle(S, slope):
    layers = _weights(I.BASE_SEED + 300, bias_seed=I.BASE_SEED + 400)
    net = UNet(S, 16, weights=layers, slope=slope)
    x = I.random_complex_field(I.BASE_SEED + 301, (3, S, S, S)).real.astype(np.float32)
    t = I.random_complex_field(I.BASE_SEED + 302, (2, S, S, S)).real.astype(np.float32)
    xd, td = torch.from_numpy(x).to(DEV), torch.from_numpy(t).to(DEV)
    out = net.forward(xd).cpu().numpy()
    params = [(w.astype(np.float64), b.astype(np.float64)) for w, b in layers]
    ref, _ = OU.forward(params, x.astype(np.float64), slope)
    assert _rel(out, ref) < 1e-5
    loss = net.loss_grad(xd, td)
    L, grads = OU.loss_and_grads(params, x.astype(np.float64), t.astype(np.float64), slope)
    assert abs(loss - L) < 1e-5 * L
    g = net.get(2)
    off = 0
    for i, (w, b) in enumerate(layers):
        gw = g[off:off + w.size].reshape(w.shape)
        off += w.size
        gb = g[off:off + b.size]
        off += b.size
        assert _rel(gw, grads[i][0]) < 1e-4, i
        assert _rel(gb, grads[i][1]) < 1e-4, i
    net.close()


def test_unet_training_reduces_loss():
    S = 16
    net = UNet(S, 16, weights=_weights(I.BASE_SEED + 310))
    xh = I.random_complex_field(I.BASE_SEED + 311, (3, S, S, S)).real.astype(np.float32)
    x = torch.from_numpy(xh).to(DEV)
    # a target the network can represent (half of the first two input channels);
    # the FP64 oracle with the same Adam steps ends near 0.12 x the first loss
    t = torch.from_numpy(0.5 * xh[:2]).to(DEV)
    first = net.loss_grad(x, t)
    for _ in range(60):
        net.loss_grad(x, t)
        net.adam_step(3e-3)
    last = net.loss_grad(x, t)
    assert last < 0.3 * first
    w, wq = net.get(0), net.get(1)
    assert np.array_equal(wq, I.bf16_round(w))  # BF16 copies of the FP32 master weights
    net.close()


def _ls_setup(N, k, seed):
    plan = Plan(3, N, "helmholtz", k, 1.8, precision="fp32")
    q = torch.from_numpy(I.ls_contrast(seed, N).astype(np.float32)).to(DEV)
    uinc = torch.from_numpy(I.plane_wave(N, k).astype(np.complex64)).to(DEV)
    b = vp.ls_rhs(plan, q, uinc)
    return plan, q, uinc, b


def test_ls_solve_matches_oracle_dense_solve():
    N, k = 12, 6.0
    plan, q, uinc, b = _ls_setup(N, k, I.LS_TRAIN_SEED)
    u = torch.zeros_like(uinc)
    st = vp.ls_solve(plan, q, b, u, u_inc=uinc, tol=1e-7, maxit=500, restart=30)
    assert st["true_residual"] < 1e-6 and st["used_fallback"] == 0
    prob = OLS.LSProblem(N, k, I.ls_contrast(I.LS_TRAIN_SEED, N).astype(np.float32).astype(np.float64))
    ref = OLS.dense_solve(prob, prob.rhs(I.plane_wave(N, k).astype(np.complex64).astype(np.complex128)))
    got = u.cpu().numpy()
    assert np.linalg.norm((got - ref).ravel()) / np.linalg.norm(ref.ravel()) < 1e-5
    # the operator entry point agrees with the oracle operator
    Au = vp.ls_operator(plan, q, u).cpu().numpy()
    assert np.linalg.norm((Au - prob.op(got.astype(np.complex128))).ravel()) / np.linalg.norm(Au.ravel()) < 1e-5


def test_krylov_basis_matches_oracle_arnoldi():
    N, k, m = 12, 6.0, 8
    plan, q, uinc, b = _ls_setup(N, k, I.LS_TRAIN_SEED)
    V = vp.ls_krylov_basis(plan, q, b, m).cpu().numpy().astype(np.complex128)
    assert V.shape == (m + 1, N, N, N)
    prob = OLS.LSProblem(N, k, I.ls_contrast(I.LS_TRAIN_SEED, N).astype(np.float32).astype(np.float64))
    Vr, _ = OLS.arnoldi(prob.op, b.cpu().numpy().astype(np.complex128), m)
    G = V.reshape(m + 1, -1).conj() @ V.reshape(m + 1, -1).T
    assert np.abs(G - np.eye(m + 1)).max() < 1e-5
    for j in range(m + 1):
        assert np.linalg.norm((V[j] - Vr[j]).ravel()) < 1e-4, j


def test_flexible_basis_with_identity_network_is_the_arnoldi_basis():
    """A network with all-zero weights makes the preconditioner the identity
    (z = r exactly), so the flexible directions are the plain Arnoldi vectors."""
    N, k, m = 16, 8.0, 6
    plan, q, uinc, b = _ls_setup(N, k, I.LS_TRAIN_SEED + 2)
    net = UNet(N, 16)
    net.set_weights(np.zeros(net.nparams, np.float32))
    net.bind(q)
    Z = vp.ls_flexible_basis(plan, q, b, m, net)
    V = vp.ls_krylov_basis(plan, q, b, m)
    assert Z.shape[0] == m
    assert torch.equal(Z, V[:m])
    net.close()


def test_ls_solve_full_size_true_residual():
    """N = 128, k = 30, q = smoothed cube + perturbations, plane wave: plain
    GMRES reaches a true FP64 residual below 1e-6."""
    plan, q, uinc, b = _ls_setup(128, 30.0, I.LS_HELDOUT_SEED)
    u = torch.zeros_like(uinc)
    st = vp.ls_solve(plan, q, b, u, u_inc=uinc, tol=3e-7, maxit=2000, restart=40)
    assert st["true_residual"] < 1e-6, st
    assert st["iterations"] < 2000


def test_untrained_preconditioner_falls_back_and_still_converges():
    N, k = 32, 10.0
    plan, q, uinc, b = _ls_setup(N, k, I.LS_TRAIN_SEED + 1)
    net = UNet(N, 16, weights=_weights(I.BASE_SEED + 320))
    net.bind(q)
    u = torch.zeros_like(uinc)
    st = vp.ls_solve(plan, q, b, u, u_inc=uinc, tol=3e-7, maxit=800, restart=20, precond=net)
    assert st["true_residual"] < 1e-6, st
    net.close()


@pytest.mark.parametrize("tag", ["c300", "c2000"])
def test_trained_preconditioner_against_plain_gmres(tag):
    """Held-out contrasts (N = 128, k = 30, plane wave): plain flexible GMRES
    against the trained network as right preconditioner, same restart length,
    both measured by the true FP64 residual.  The committed reports
    (weights/unet_ls_k30_n128_<tag>.json, 50 held-out contrasts) measured 20.2
    plain iterations against 30.6 (trained on 300 contrasts, no fallback) and
    66.4 (2000 contrasts, every solve fell back): on this well-conditioned
    problem the network does not reduce the iteration count.  The test pins
    what holds: the preconditioned solve reaches the same true residual and
    stays within 4x the plain iterations."""
    import os

    from paper_1604_03155_gb300 import precond as P
    wdir = os.path.join(os.path.dirname(vp.__file__), "weights")
    N, k = 128, 30.0
    plan = Plan(3, N, "helmholtz", k, 1.8, precision="fp32")
    net = UNet(N, 16, slope=0.1)
    P.load_weights(net, os.path.join(wdir, f"unet_ls_k30_n128_{tag}.npy"))
    ev = P.evaluate(plan, net, N, k, [I.LS_HELDOUT_SEED + i for i in range(3)], tol=1e-6, restart=20)
    s = ev["summary"]
    print(tag, s)
    assert s["plain_true_residual_max"] < 1e-6 and s["precond_true_residual_max"] < 1e-6
    assert s["precond_iterations"] <= 4 * s["plain_iterations"]
    net.close()
    plan.close()


def test_bounded_wait_timeout_is_reported_and_recoverable():
    """The tensor-core convolutions and weight gradients bound their waits for
    the MMAs: with the MMAs withheld (a completion nothing signals) the waits
    run out after a short budget, the kernels finish, the status reports
    VP_ERR_TIMEOUT once, and the network runs correctly afterwards."""
    S = 8
    net = UNet(S, 16, weights=_weights(5))
    x = torch.from_numpy(I.normal(91, 3 * S ** 3).astype(np.float32).reshape(3, S, S, S)).to(DEV)
    tgt = torch.zeros((2, S, S, S), dtype=torch.float32, device=DEV)
    ref = net.forward(x).cpu().numpy()
    net.status()
    net.set_timeout(0.001)
    net.withhold(True)
    net.forward(x)
    with pytest.raises(vp.VPError) as ei:
        net.status()
    assert ei.value.status == vp.VP_ERR_TIMEOUT
    with pytest.raises(vp.VPError) as ei:
        net.loss_grad(x, tgt)  # the weight gradients' waits run out too
    assert ei.value.status == vp.VP_ERR_TIMEOUT
    net.withhold(False)
    net.set_timeout(2.0)
    net.status()  # cleared
    out = net.forward(x).cpu().numpy()
    net.status()
    assert np.array_equal(out, ref)
    net.close()


def test_training_resumes_from_a_checkpoint(tmp_path):
    """Weights and Adam state saved after 5 steps and restored into a fresh
    network give, after 5 more steps, the same weights bit for bit as the run
    that never stopped; restoring the weights alone (Adam state reset) does not."""
    from paper_1604_03155_gb300 import precond as P
    S = 16
    xh = I.random_complex_field(I.BASE_SEED + 321, (3, S, S, S)).real.astype(np.float32)
    x = torch.from_numpy(xh).to(DEV)
    t = torch.from_numpy(0.5 * xh[:2]).to(DEV)

    def steps(net, n):
        for _ in range(n):
            net.loss_grad(x, t)
            net.adam_step(3e-3)

    a = UNet(S, 16, weights=_weights(I.BASE_SEED + 320))
    steps(a, 5)
    ck = str(tmp_path / "ck.npz")
    P.save_checkpoint(a, ck, next_contrast=5)
    m, v, step = a.get_adam()
    assert step == 5 and np.abs(m).max() > 0 and v.min() >= 0
    steps(a, 5)
    ref = a.get(0)

    b = UNet(S, 16)
    extra = P.load_checkpoint(b, ck)
    assert extra == {"next_contrast": 5} and b.get_adam()[2] == 5
    steps(b, 5)
    assert np.array_equal(b.get(0), ref)

    c = UNet(S, 16)
    c.set_weights(np.load(ck)["weights"])
    assert c.get_adam()[2] == 0
    steps(c, 5)
    assert not np.array_equal(c.get(0), ref)
    with pytest.raises(vp.VPError):
        c.set_adam(m[:-1], v, 1)
    with pytest.raises(vp.VPError):
        c.set_adam(m, v, -1)
    for net in (a, b, c):
        net.close()


def test_wait_budget_from_the_environment(monkeypatch):
    """VP_TIMEOUT_MS sets the bounded waits' budget at vp_unet_create: with the
    MMAs withheld a forward reports VP_ERR_TIMEOUT after about 1 ms per
    convolution, not after the built-in 2 s."""
    import time
    monkeypatch.setenv("VP_TIMEOUT_MS", "1")
    S = 8
    net = UNet(S, 16, weights=_weights(5))
    x = torch.from_numpy(I.normal(92, 3 * S ** 3).astype(np.float32).reshape(3, S, S, S)).to(DEV)
    ref = net.forward(x).cpu().numpy()
    net.withhold(True)
    t0 = time.perf_counter()
    net.forward(x)
    with pytest.raises(vp.VPError) as ei:
        net.status()
    elapsed = time.perf_counter() - t0
    assert ei.value.status == vp.VP_ERR_TIMEOUT
    assert elapsed < 1.0, elapsed
    net.withhold(False)
    net.status()
    assert np.array_equal(net.forward(x).cpu().numpy(), ref)
    net.close()
