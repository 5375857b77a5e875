"""The paper's scattering solver on the GPU (Section 5.3): Bi-CGStab over the
FP64 and FP32 applies, field and density forms, against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import ls as OLS
from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300 import vp
from paper_1604_03155_gb300.vp import Plan

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
CONTRAST = {"disk": I.filtered_disk, "lens": I.luneburg_lens, "cube": I.cube_bump}


def _case(name, N, size):
    q = CONTRAST[name](N)
    k = 2 * np.pi * size
    return q, k, I.plane_wave(N, k, q.ndim)


def _gpu_solve(q, k, uinc, form, precision, tol, maxit=4000, history=False):
    d, N = q.ndim, q.shape[0]
    plan = Plan(d, N, "helmholtz", k, 0.0, precision=precision)
    rdt, cdt = (torch.float64, torch.complex128) if precision == "fp64" else (torch.float32, torch.complex64)
    qd = torch.from_numpy(q).to(DEV, rdt)
    ud = torch.from_numpy(uinc).to(DEV, cdt)
    out = vp.ls_bicgstab(plan, qd, ud, form=form, tol=tol, maxit=maxit, history=history)
    plan.close()
    return (out[0].cpu().numpy(),) + tuple(out[1:])


def _rel2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


_ORACLE = {}


def _oracle(name, N, size, form):
    """The oracle's problem and its Bi-CGStab solve at tol 1e-13 (cached):
    (problem, u_inc, iterations, history, scattered field)."""
    key = (name, N, size, form)
    if key not in _ORACLE:
        q, k, uinc = _case(name, N, size)
        prob = OLS.LSProblem(N, k, q)
        op = prob.op if form == "field" else prob.op_density
        b = prob.rhs(uinc) if form == "field" else prob.rhs_density(uinc)
        x, its, mv, hist = OLS.bicgstab(op, b, tol=1e-13)
        _ORACLE[key] = (prob, uinc, its, hist, x if form == "field" else prob.V(x))
    return _ORACLE[key]


@pytest.mark.parametrize("name,N,size", [("disk", 48, 2.0), ("lens", 48, 2.0), ("cube", 12, 1.0)])
@pytest.mark.parametrize("form", ["field", "density"])
def test_fp64_bicgstab_matches_oracle(name, N, size, form):
    """FP64: the oracle's iterates (recurrence residuals equal until the stop,
    iteration counts equal up to the last step) and its solution to 1e-10."""
    q, k, uinc = _case(name, N, size)
    prob, _, its, ohist, u_ref = _oracle(name, N, size, form)
    u_gpu, st, hist = _gpu_solve(q, k, uinc, form, "fp64", 1e-13, history=True)
    assert st["estimated_residual"] < 1e-13 and st["true_residual"] < 1e-12
    assert abs(st["iterations"] - its) <= 1 and st["matvecs"] in (2 * st["iterations"], 2 * st["iterations"] - 1)
    assert _rel2(u_gpu, u_ref) < 1e-10
    # the same iterates: the recurrence residuals agree while they stay well above
    # the rounding level (different summation orders; Bi-CGStab amplifies the
    # difference as the residual falls)
    m = min(len(hist), len(ohist))
    h, oh = np.asarray(hist[:m]), np.asarray(ohist[:m])
    big = oh > 1e-9
    assert big.sum() >= 5
    assert np.all(np.abs(h[big] - oh[big]) <= 1e-2 * oh[big])


@pytest.mark.parametrize("name,N,size", [("disk", 16, 2.0), ("lens", 16, 2.0), ("cube", 8, 1.0)])
def test_fp64_bicgstab_matches_dense_solve(name, N, size):
    """Small grids: both forms against the oracle's dense direct solve."""
    q, k, uinc = _case(name, N, size)
    prob = OLS.LSProblem(N, k, q)
    u_dense = OLS.dense_solve(prob, prob.rhs(uinc))
    for form in ("field", "density"):
        u_gpu, st = _gpu_solve(q, k, uinc, form, "fp64", 1e-13)
        assert _rel2(u_gpu, u_dense) < 1e-10, form


@pytest.mark.parametrize("name,N,size", [("disk", 48, 2.0), ("cube", 12, 1.0)])
@pytest.mark.parametrize("form", ["field", "density"])
def test_fp32_bicgstab_matches_oracle(name, N, size, form):
    q, k, uinc = _case(name, N, size)
    u_ref = _oracle(name, N, size, "field")[4]
    u_gpu, st = _gpu_solve(q, k, uinc, form, "fp32", 1e-5)
    assert st["estimated_residual"] < 1e-5
    # FP32 applies carry ~1e-6 relative error per product
    assert st["true_residual"] < 3e-5
    assert _rel2(u_gpu, u_ref) < 1e-4


def test_forms_agree_and_residual_at_full_size():
    """2D N = 1024 (2N = 2048) filtered disk, 20 wavelengths, FP64: both forms
    converge to 1e-12 with a true residual below 1e-11 and give the same field."""
    q, k, uinc = _case("disk", 1024, 20.0)
    u_f, st_f = _gpu_solve(q, k, uinc, "field", "fp64", 1e-12)
    u_d, st_d = _gpu_solve(q, k, uinc, "density", "fp64", 1e-12)
    for st in (st_f, st_d):
        assert st["estimated_residual"] < 1e-12 and st["true_residual"] < 1e-11
        assert 100 < st["matvecs"] < 2000
    assert _rel2(u_d, u_f) < 1e-10


def test_3d_full_size_fp64_residual():
    """3D N = 128 (2N = 256) smoothed cube, 10 wavelengths, FP64."""
    q, k, uinc = _case("cube", 128, 10.0)
    u, st = _gpu_solve(q, k, uinc, "density", "fp64", 1e-12)
    assert st["estimated_residual"] < 1e-12 and st["true_residual"] < 1e-11


def test_deterministic_and_history():
    q, k, uinc = _case("lens", 64, 4.0)
    u1, st1, h1 = _gpu_solve(q, k, uinc, "density", "fp64", 1e-12, history=True)
    u2, st2, h2 = _gpu_solve(q, k, uinc, "density", "fp64", 1e-12, history=True)
    assert np.array_equal(u1, u2) and np.array_equal(h1, h2) and st1["matvecs"] == st2["matvecs"]
    assert h1[0] == 1.0 and h1[-1] < 1e-12 and len(h1) == st1["iterations"] + 1


def test_edge_cases():
    N, k = 16, 2 * np.pi
    plan = Plan(2, N, "helmholtz", k, 0.0, precision="fp64")
    q = torch.from_numpy(I.filtered_disk(N)).to(DEV)
    # zero incident field: u = 0 without iterations
    z = torch.zeros((N, N), dtype=torch.complex128, device=DEV)
    u, st = vp.ls_bicgstab(plan, q, z, form="field")
    assert st["iterations"] == 0 and st["matvecs"] == 0 and torch.count_nonzero(u) == 0
    # zero contrast: b = 0 as well
    u, st = vp.ls_bicgstab(plan, torch.zeros_like(q), torch.from_numpy(I.plane_wave(N, k, 2)).to(DEV), form="density")
    assert st["iterations"] == 0 and torch.count_nonzero(u) == 0
    # maxit reached: VP_OK, residual above tol, exactly maxit iterations
    ui = torch.from_numpy(I.plane_wave(N, k, 2)).to(DEV)
    u, st = vp.ls_bicgstab(plan, q, ui, form="field", tol=1e-14, maxit=2)
    assert st["iterations"] == 2 and st["matvecs"] == 4 and st["estimated_residual"] > 1e-14
    # dtype and precision mismatches, aliasing, a Laplace plan
    with pytest.raises(vp.VPError):
        vp.ls_bicgstab(plan, q.float(), ui.to(torch.complex64))
    with pytest.raises(vp.VPError):
        vp.ls_bicgstab(plan, q, ui, u=ui)
    with pytest.raises(vp.VPError):
        vp.ls_bicgstab(plan, q, ui, form="other")
    plan.close()
    lap = Plan(2, N, "laplace", 0.0, 0.0, precision="fp64")
    with pytest.raises(vp.VPError):
        vp.ls_bicgstab(lap, q, ui)
    lap.close()
    tc = Plan(3, 128, "helmholtz", 10.0, 0.0, precision="tc_bf16x2")
    q3 = torch.zeros((128,) * 3, dtype=torch.float32, device=DEV)
    with pytest.raises(vp.VPError):
        vp.ls_bicgstab(tc, q3, torch.zeros((128,) * 3, dtype=torch.complex64, device=DEV))
    tc.close()


def _gpu_mixed(q, k, uinc, form, tol=1e-12, delta=1e-2, history=False):
    d, N = q.ndim, q.shape[0]
    plan = Plan(d, N, "helmholtz", k, 0.0, precision="fp32")
    qd = torch.from_numpy(q).to(DEV, torch.float64)
    ud = torch.from_numpy(uinc).to(DEV, torch.complex128)
    out = vp.ls_bicgstab_mixed(plan, qd, ud, form=form, tol=tol, delta=delta, history=history)
    plan.close()
    return (out[0].cpu().numpy(),) + tuple(out[1:])


@pytest.mark.parametrize("name,N,size", [("disk", 48, 2.0), ("lens", 48, 2.0), ("cube", 12, 1.0)])
@pytest.mark.parametrize("form", ["field", "density"])
def test_mixed_precision_reaches_fp64_accuracy(name, N, size, form):
    """FP32 iterations with FP64 reliable updates reach the oracle's FP64
    solution to 1e-10 with a true FP64 residual below 1e-12."""
    q, k, uinc = _case(name, N, size)
    u_ref = _oracle(name, N, size, "field")[4]
    u, st, hist = _gpu_mixed(q, k, uinc, form, history=True)
    assert st["estimated_residual"] < 1e-12 and st["true_residual"] < 1e-12
    assert st["restarts"] >= 2  # FP64 updates happened
    assert _rel2(u, u_ref) < 1e-10
    assert hist[0] == 1.0 and len(hist) == st["iterations"] + 1


def test_mixed_precision_full_size_matches_fp64_solver():
    """2D N = 1024 filtered disk, 20 wavelengths: the mixed solve agrees with the
    FP64 solve to 1e-10 in both forms."""
    q, k, uinc = _case("disk", 1024, 20.0)
    u64, st64 = _gpu_solve(q, k, uinc, "density", "fp64", 1e-12)
    for form in ("density", "field"):
        u, st = _gpu_mixed(q, k, uinc, form)
        assert st["true_residual"] < 1e-12, form
        assert _rel2(u, u64) < 1e-10, form
        assert st["matvecs"] < 3 * st64["matvecs"], form


def test_mixed_precision_edge_cases():
    N, k = 16, 2 * np.pi
    plan = Plan(2, N, "helmholtz", k, 0.0, precision="fp64")
    q = torch.from_numpy(I.filtered_disk(N)).to(DEV)
    z = torch.zeros((N, N), dtype=torch.complex128, device=DEV)
    u, st = vp.ls_bicgstab_mixed(plan, q, z)
    assert st["iterations"] == 0 and torch.count_nonzero(u) == 0
    ui = torch.from_numpy(I.plane_wave(N, k, 2)).to(DEV)
    for bad in (0.0, 1.0, -0.5):
        with pytest.raises(vp.VPError):
            vp.ls_bicgstab_mixed(plan, q, ui, delta=bad)
    # the plan's precision is restored
    u, st = vp.ls_bicgstab_mixed(plan, q, ui)
    phi = plan.apply(ui)  # complex128 input works only if the plan is back in FP64
    assert phi.dtype == torch.complex128 and st["true_residual"] < 1e-12
    plan.close()


def test_mixed_precision_fallback_mechanics():
    """An FP32 phase that cannot finish within maxit hands over to the FP64 solve:
    used_fallback is set and the products of both phases are counted."""
    q, k, uinc = _case("disk", 48, 2.0)
    plan = Plan(2, 48, "helmholtz", k, 0.0, precision="fp32")
    qd = torch.from_numpy(q).to(DEV)
    ud = torch.from_numpy(uinc).to(DEV)
    u, st = vp.ls_bicgstab_mixed(plan, qd, ud, tol=1e-12, maxit=3)
    assert st["used_fallback"] == 1
    assert st["iterations"] == 6 and st["matvecs"] == 12
    # an update after every iteration that gains little stalls the FP32 phase
    # early; the FP64 solve that continues from the mixed iterate converges
    u, st = vp.ls_bicgstab_mixed(plan, qd, ud, tol=1e-12, maxit=60, delta=0.999999)
    assert st["true_residual"] < 1e-12
    plan.close()


@pytest.mark.parametrize("form", ["field", "density"])
def test_mixed_precision_fallback_continues_from_mixed_iterate(form):
    """An FP32 phase cut off by maxit = the FP64 solve's iteration count (the
    FP32 phase needs about 1.5x that, with one idle launch per update) hands
    over to an FP64 solve of the correction equation M e = b - M x from the
    mixed iterate x: u = x + e (field) or V[s + e] (density) is the oracle's
    solution to 1e-10, and that FP64 phase takes fewer products than the FP64
    solve from zero."""
    q, k, uinc = _case("disk", 48, 2.0)
    u_ref = _oracle("disk", 48, 2.0, "field")[4]
    _, st64 = _gpu_solve(q, k, uinc, form, "fp64", 1e-12)
    maxit = st64["iterations"]
    plan = Plan(2, 48, "helmholtz", k, 0.0, precision="fp32")
    qd = torch.from_numpy(q).to(DEV)
    ud = torch.from_numpy(uinc).to(DEV)
    u, st = vp.ls_bicgstab_mixed(plan, qd, ud, form=form, tol=1e-12, maxit=maxit)
    plan.close()
    assert st["used_fallback"] == 1, (st, st64)
    assert st["true_residual"] < 1e-12, (st, st64)
    assert _rel2(u.cpu().numpy(), u_ref) < 1e-10
    # the FP32 phase ran maxit graph launches, each an iteration of two products
    # except the one idle launch after each update
    mixed_products = 2 * (maxit - st["restarts"])
    assert st["matvecs"] - mixed_products < st64["matvecs"], (st, st64)


@pytest.mark.parametrize("form", ["field", "density"])
def test_mixed_precision_nonfinite_fp32_phase_restarts_in_fp64(form):
    """An incident field of amplitude 1e37 overflows the FP32 products (the
    transforms sum thousands of such values) but not FP64: the FP32 phase ends
    non-finite and the FP64 phase starts again from zero.  The solution is
    linear in the incident field, so it is 1e37 times the oracle's."""
    name, N, size = "disk", 48, 2.0
    q, k, uinc = _case(name, N, size)
    u_ref = _oracle(name, N, size, "field")[4]
    scale = 1e37
    u, st = _gpu_mixed(q, k, uinc * scale, form)
    assert np.all(np.isfinite(u))
    assert st["used_fallback"] == 1
    assert st["true_residual"] < 1e-12
    assert _rel2(u / scale, u_ref) < 1e-10
