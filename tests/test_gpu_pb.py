"""The variable-coefficient Poisson solve of Section 5.2 on the GPU (Bi-CGStab
over the exact-gradient apply; FP64, FP32 and mixed precision) against the
oracle and a closed-form manufactured solution."""
import math

import numpy as np
import pytest
import torch

from oracle import closed_forms as CF
from oracle import ls as OLS
from oracle import pb as OPB
from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300 import vp
from paper_1604_03155_gb300.vp import Plan

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _manufactured(N, s=0.08):
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


def _solve(N, eps, ge, rho, precision, tol, mixed=False, history=False):
    plan = Plan(3, N, "laplace", 0.0, 0.0, precision="fp32" if mixed else precision)
    rdt, cdt = (torch.float32, torch.complex64) if precision == "fp32" else (torch.float64, torch.complex128)
    e = torch.as_tensor(np.asarray(eps)).to(DEV, rdt).contiguous()
    g = torch.as_tensor(np.asarray(ge)).to(DEV, rdt).contiguous()
    b = torch.as_tensor(np.asarray(rho)).to(DEV, cdt).contiguous()
    out = vp.pb_solve(plan, e, g, b, tol=tol, mixed=mixed, history=history)
    plan.close()
    return (out[0].cpu().numpy(),) + tuple(out[1:])


def _rel2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_molecule_fp64_against_oracle():
    N = 16
    eps, ge, rho = (t.numpy() for t in I.pb_fields(I.pb_molecule(), N))
    prob = OPB.PBProblem(N, eps, ge)
    x, its, mv, ohist = OLS.bicgstab(prob.op, rho.astype(np.complex128), tol=1e-13)
    sig, st, hist = _solve(N, eps, ge, rho, "fp64", 1e-13, history=True)
    assert st["true_residual"] < 1e-12 and abs(st["iterations"] - its) <= 1
    assert _rel2(sig, x) < 1e-10
    m = min(len(hist), len(ohist))
    big = np.asarray(ohist[:m]) > 1e-9
    assert np.all(np.abs(np.asarray(hist[:m])[big] - np.asarray(ohist[:m])[big]) <= 1e-2 * np.asarray(ohist[:m])[big])


@pytest.mark.parametrize("mixed", [False, True])
def test_manufactured_solution_fp64_accuracy(mixed):
    """N = 64: the analytic sigma to 1e-10 (FP64, and mixed precision)."""
    N = 64
    eps, ge, rho, sig = _manufactured(N)
    got, st = _solve(N, eps, ge, rho, "fp64", 1e-13, mixed=mixed)
    assert _rel2(got, sig) < 1e-10
    assert st["true_residual"] < 1e-12 and st["used_fallback"] == 0


def test_mixed_fallback_continues_from_mixed_iterate():
    """An FP32 phase cut off by maxit hands over to FP64 Bi-CGStab on the
    correction equation from the mixed iterate: the analytic sigma to 1e-10."""
    N = 48
    eps, ge, rho, sig = _manufactured(N)
    _, st64 = _solve(N, eps, ge, rho, "fp64", 1e-13)
    plan = Plan(3, N, "laplace", 0.0, 0.0, precision="fp32")
    e = torch.as_tensor(eps).to(DEV).contiguous()
    g = torch.as_tensor(ge).to(DEV).contiguous()
    b = torch.as_tensor(rho).to(DEV, torch.complex128).contiguous()
    maxit = max(2, (2 * st64["iterations"]) // 3)
    got, st = vp.pb_solve(plan, e, g, b, tol=1e-13, maxit=maxit, mixed=True)
    plan.close()
    assert st["used_fallback"] == 1 and st["true_residual"] < 1e-12
    assert _rel2(got.cpu().numpy(), sig) < 1e-10


def test_fp32_against_oracle():
    N = 24
    eps, ge, rho, sig = _manufactured(N)
    got, st = _solve(N, eps, ge, rho, "fp32", 1e-6)
    assert st["true_residual"] < 1e-5
    assert _rel2(got, sig) < 1e-5  # the N = 24 discretisation error is 3.6e-11


def test_full_size_molecule_mixed_matches_fp64():
    """N = 128 with the 1235-atom molecule: the mixed solve equals the FP64 one."""
    N = 128
    eps, ge, rho = I.pb_fields(I.pb_molecule(), N, device=DEV)
    plan = Plan(3, N, "laplace", 0.0, 0.0, precision="fp64")
    b = rho.to(torch.complex128)
    s64, st64 = vp.pb_solve(plan, eps, ge.contiguous(), b, tol=1e-12)
    sm, stm = vp.pb_solve(plan, eps, ge.contiguous(), b, tol=1e-12, mixed=True)
    assert st64["true_residual"] < 1e-12 and stm["true_residual"] < 1e-12
    assert float((sm - s64).norm() / s64.norm()) < 1e-10
    assert st64["iterations"] < 40
    plan.close()


def test_pb_edge_cases():
    N = 8
    plan = Plan(3, N, "laplace", 0.0, 0.0, precision="fp64")
    eps = torch.full((N, N, N), 2.0, dtype=torch.float64, device=DEV)
    ge = torch.zeros((3, N, N, N), dtype=torch.float64, device=DEV)
    z = torch.zeros((N, N, N), dtype=torch.complex128, device=DEV)
    s, st = vp.pb_solve(plan, eps, ge, z)
    assert st["iterations"] == 0 and torch.count_nonzero(s) == 0
    with pytest.raises(vp.VPError):
        vp.pb_solve(plan, eps, ge, z, sigma=z)
    plan.close()
    hel = Plan(3, N, "helmholtz", 3.0, 0.0, precision="fp64")
    with pytest.raises(vp.VPError):
        vp.pb_solve(hel, eps, ge, z)
    hel.close()


def _manufactured_2d(N, s=0.08):
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


def test_manufactured_solution_2d():
    """2D Laplace plan, N = 256: the analytic sigma (Gauss's-law gradient) to
    1e-10 in FP64 and mixed precision."""
    N = 256
    eps, ge, rho, sig = _manufactured_2d(N)
    for mixed in (False, True):
        plan = Plan(2, N, "laplace", 0.0, 0.0, precision="fp32" if mixed else "fp64")
        e = torch.from_numpy(eps).to(DEV)
        gg = torch.from_numpy(ge).to(DEV).contiguous()
        b = torch.from_numpy(rho).to(DEV, torch.complex128)
        got, st = vp.pb_solve(plan, e, gg, b, tol=1e-13, mixed=mixed)
        assert _rel2(got.cpu().numpy(), sig) < 1e-10, mixed
        plan.close()


def _gmres(d, N, eps, ge, rho, tol, restart=40, maxit=1000, history=False):
    plan = Plan(d, N, "laplace", 0.0, 0.0, precision="fp64")
    e = torch.as_tensor(np.asarray(eps)).to(DEV, torch.float64).contiguous()
    g = torch.as_tensor(np.asarray(ge)).to(DEV, torch.float64).contiguous()
    b = torch.as_tensor(np.asarray(rho)).to(DEV, torch.complex128).contiguous()
    out = vp.pb_gmres(plan, e, g, b, tol=tol, restart=restart, maxit=maxit, history=history)
    plan.close()
    return (out[0].cpu().numpy(),) + tuple(out[1:])


def test_gmres_follows_the_oracle_gmres():
    """GMRES(40) on the molecule at N = 16 (no restart): the oracle's GMRES
    residual estimates step by step (within 1% while above 1e-9), its step count
    within one, and its solution to 1e-10."""
    N = 16
    eps, ge, rho = (t.numpy() for t in I.pb_fields(I.pb_molecule(), N))
    prob = OPB.PBProblem(N, eps, ge)
    x, its, ohist = OLS.gmres(prob.op, rho.astype(np.complex128), tol=1e-13, restart=40)
    assert its < 40
    sig, st, hist = _gmres(3, N, eps, ge, rho, 1e-13, history=True)
    assert abs(st["iterations"] - its) <= 1 and st["restarts"] == 0
    assert st["matvecs"] == st["iterations"]
    assert st["true_residual"] < 1e-12
    assert _rel2(sig, x) < 1e-10
    m = min(len(hist), len(ohist))
    big = np.asarray(ohist[:m]) > 1e-9
    assert np.all(np.abs(np.asarray(hist[:m])[big] - np.asarray(ohist[:m])[big]) <= 1e-2 * np.asarray(ohist[:m])[big])


def test_gmres_restarted_matches_the_oracle():
    """GMRES(4) with restarts from the explicit residual: the oracle's GMRES(4)
    solution to 1e-10 and its step count within two."""
    N = 16
    eps, ge, rho = (t.numpy() for t in I.pb_fields(I.pb_molecule(), N))
    prob = OPB.PBProblem(N, eps, ge)
    x, its, _ = OLS.gmres(prob.op, rho.astype(np.complex128), tol=1e-13, restart=4)
    sig, st = _gmres(3, N, eps, ge, rho, 1e-13, restart=4)
    assert st["restarts"] >= 1 and st["matvecs"] == st["iterations"] + st["restarts"]
    assert abs(st["iterations"] - its) <= 2
    assert st["true_residual"] < 1e-12
    assert _rel2(sig, x) < 1e-10


def test_gmres_manufactured_solutions():
    """The analytic sigma to 1e-10: 3D N = 64 and 2D N = 256."""
    eps, ge, rho, sig = _manufactured(64)
    got, st = _gmres(3, 64, eps, ge, rho, 1e-13)
    assert _rel2(got, sig) < 1e-10 and st["true_residual"] < 1e-12
    eps, ge, rho, sig = _manufactured_2d(256)
    got, st = _gmres(2, 256, eps, ge, rho, 1e-13)
    assert _rel2(got, sig) < 1e-10 and st["true_residual"] < 1e-12


def test_gmres_full_size_molecule_matches_bicgstab():
    """N = 128, the 1235-atom molecule: GMRES and Bi-CGStab give the same sigma
    to 1e-10; repeated GMRES solves are bit-identical."""
    N = 128
    eps, ge, rho = I.pb_fields(I.pb_molecule(), N, device=DEV)
    plan = Plan(3, N, "laplace", 0.0, 0.0, precision="fp64")
    b = rho.to(torch.complex128)
    g = ge.contiguous()
    s1, st1 = vp.pb_gmres(plan, eps, g, b, tol=1e-12)
    s2, _ = vp.pb_gmres(plan, eps, g, b, tol=1e-12)
    sb, stb = vp.pb_solve(plan, eps, g, b, tol=1e-12)
    plan.close()
    assert st1["true_residual"] < 1e-12 and st1["iterations"] < 40
    assert torch.equal(s1, s2)
    assert float((s1 - sb).norm() / sb.norm()) < 1e-10


def test_gmres_edge_cases():
    N = 8
    plan = Plan(3, N, "laplace", 0.0, 0.0, precision="fp64")
    eps = torch.full((N, N, N), 2.0, dtype=torch.float64, device=DEV)
    ge = torch.zeros((3, N, N, N), dtype=torch.float64, device=DEV)
    z = torch.zeros((N, N, N), dtype=torch.complex128, device=DEV)
    s, st = vp.pb_gmres(plan, eps, ge, z)
    assert st["iterations"] == 0 and torch.count_nonzero(s) == 0
    # constant eps, grad eps = 0: P = -2 I, one step solves it
    rho = torch.randn((N, N, N), dtype=torch.float64, device=DEV).to(torch.complex128)
    s, st = vp.pb_gmres(plan, eps, ge, rho)
    assert st["iterations"] == 1 and torch.allclose(s, -rho / 2, rtol=1e-14, atol=0)
    for bad in (0, 513):
        with pytest.raises(vp.VPError):
            vp.pb_gmres(plan, eps, ge, rho, restart=bad)
    with pytest.raises(vp.VPError):
        vp.pb_gmres(plan, eps, ge, rho, sigma=rho)
    # the step budget: VP_OK with the residual reached so far
    e2 = eps + 0.5 * torch.rand_like(eps)
    g2 = 0.3 * torch.randn_like(ge)
    s, st = vp.pb_gmres(plan, e2, g2, rho, tol=1e-14, maxit=2)
    assert st["iterations"] == 2 and st["true_residual"] > 1e-14
    # GMRES(1) still converges on this near-identity operator
    s1, st1 = vp.pb_gmres(plan, e2, g2, rho, tol=1e-12, restart=1, maxit=500)
    assert st1["true_residual"] < 1e-12 and st1["restarts"] >= 1
    plan.set_precision("fp32")
    with pytest.raises(vp.VPError):
        vp.pb_gmres(plan, eps, ge, rho)
    plan.close()
