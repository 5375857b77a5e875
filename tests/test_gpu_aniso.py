"""Per-axis grid sizes on the GPU (an N_0 x N_1 [x N_2] grid on the unit box):
the FP64 precompute, the apply and exact gradients against the per-axis
oracle, a Gaussian against its closed form, the cubic case against the cubic
plan, and the features that take cubic plans only."""
import math

import numpy as np
import pytest
import torch

from oracle import aniso as AN
from oracle import apply as A
from oracle import closed_forms as CF
from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300 import vp
from paper_1604_03155_gb300.vp import Plan, VPError

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
CASES = [((8, 12, 16), "helmholtz", 9.0, 1.8), ((16, 12, 8), "laplace", 0.0, 1.8), ((24, 16, 12), "biharmonic", 0.0, 1.8),
         ((12, 8), "helmholtz", 20.0, 1.5), ((16, 48), "laplace", 0.0, 1.5)]


def _relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("Ns,kernel,k,L", CASES)
def test_octants_against_oracle(Ns, kernel, k, L):
    plan = Plan(len(Ns), Ns, kernel, k, L)
    To = AN.T_octant_by_sums(Ns, kernel, k, L)
    assert plan.get_array("T").shape == To.shape
    assert _relmax(plan.get_array("T"), To) < 1e-13
    assert _relmax(plan.get_array("ghat"), AN.ghat_octant_by_sums(To)) < 1e-13
    j = len(Ns) - 1
    Tj = AN.T_octant_by_sums(Ns, kernel, k, L, deriv_axis=j)
    assert _relmax(plan.get_array("Tj", j), Tj) < 1e-13
    assert _relmax(plan.get_array("ghatj", j), AN.ghat_octant_by_sums(Tj, odd_axis=j)) < 1e-13
    plan.close()


@pytest.mark.parametrize("Ns,kernel,k,L", CASES)
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_apply_and_gradient_against_oracle(Ns, kernel, k, L, prec):
    d = len(Ns)
    plan = Plan(d, Ns, kernel, k, L, precision=prec)
    cdt = np.complex64 if prec == "fp32" else np.complex128
    f = I.random_complex_field(700 + sum(Ns), Ns).astype(cdt)
    phi, g = plan.apply_grad(torch.from_numpy(f).to(DEV))
    phi, g = phi.cpu().numpy(), g.cpu().numpy()
    To = AN.T_octant_by_sums(Ns, kernel, k, L)
    ref = AN.apply_fft2n(AN.ghat_full_from_octant(AN.ghat_octant_by_sums(To)), f.astype(np.complex128))
    bar = 1e-5 if prec == "fp32" else 1e-12
    kappa = 10.0 if kernel == "helmholtz" else 1.0  # random data: cancellation in the oscillatory convolution
    assert A.rel_l2(phi, ref) < bar * kappa
    for j in range(d):
        Tj = AN.T_octant_by_sums(Ns, kernel, k, L, deriv_axis=j)
        Gj = AN.ghat_full_from_octant(AN.ghat_octant_by_sums(Tj, odd_axis=j), odd_axis=j)
        gref = AN.apply_fft2n(Gj, f.astype(np.complex128))
        assert A.rel_l2(g[j], gref) < 10 * bar * kappa, j
    plan.close()


def test_gaussian_closed_form_64x96x128():
    """3D Laplace, unit-mass Gaussian sigma = 0.05 on a 64 x 96 x 128 grid
    (FP64): the erf closed form to spectral accuracy."""
    Ns, s = (64, 96, 128), 0.05
    X = AN.grid(Ns)
    r = np.sqrt(sum(x * x for x in X))
    rho = (2 * math.pi * s * s) ** -1.5 * np.exp(-r * r / (2 * s * s))
    plan = Plan(3, Ns, "laplace", 0.0, 0.0, precision="fp64")
    phi = plan.apply(torch.from_numpy(rho).to(DEV)).cpu().numpy()
    assert A.rel_l2(phi, CF.laplace3(r, s)) < 1e-10
    plan.close()


def test_cubic_case_and_cubic_only_features():
    N = 16
    cube = Plan(3, N, "helmholtz", 9.0, 0.0)
    aniso = Plan(3, (N, N, N), "helmholtz", 9.0, 0.0)
    f = torch.from_numpy(I.random_complex_field(5, (N,) * 3).astype(np.complex64)).to(DEV)
    assert torch.equal(cube.apply(f), aniso.apply(f))
    cube.close()
    aniso.close()
    p = Plan(3, (128, 128, 64), "helmholtz", 9.0, 0.0)
    with pytest.raises(VPError):
        p.set_precision("tc_bf16x2")
    q = torch.zeros((128, 128, 64), dtype=torch.float32, device=DEV)
    u = torch.zeros((128, 128, 64), dtype=torch.complex64, device=DEV)
    with pytest.raises(VPError):
        vp.ls_solve(p, q, u, torch.empty_like(u))
    # the Nystrom entries and Bi-CGStab take the per-axis grid
    off = torch.tensor([[0, 0, 0], [128, -128, 64], [-3, 5, -64]], dtype=torch.int32, device=DEV)
    got = p.kernel_entries(off).cpu().numpy()
    own = p.get_array("T")
    assert np.array_equal(got, own[tuple(np.abs(off.cpu().numpy()).T)])
    p.close()
    with pytest.raises(VPError):
        Plan(3, (16, 12), "laplace", 0.0, 0.0)
    with pytest.raises(VPError):
        Plan(3, (16, 10, 12), "laplace", 0.0, 0.0)  # 2N = 20 is not built


def test_scattering_on_a_per_axis_grid():
    """Bi-CGStab (FP64) on a 24 x 32 x 16 grid against the oracle's Bi-CGStab."""
    from oracle import ls as OLS
    Ns, k = (24, 32, 16), 2 * np.pi
    X = AN.grid(Ns)
    q = np.exp(-0.5 * sum((x / 0.25) ** 8 for x in X))
    uinc = np.exp(1j * k * X[0]) * np.ones(Ns)
    To = AN.T_octant_by_sums(Ns, "helmholtz", k, 1.8)
    G = AN.ghat_full_from_octant(AN.ghat_octant_by_sums(To))
    op = lambda s: s - k * k * q * AN.apply_fft2n(G, s)
    x, its, mv, h = OLS.bicgstab(op, k * k * q * uinc, tol=1e-13)
    plan = Plan(3, Ns, "helmholtz", k, 0.0, precision="fp64")
    u, st = vp.ls_bicgstab(plan, torch.from_numpy(q).to(DEV), torch.from_numpy(uinc).to(DEV), form="density",
                           tol=1e-13)
    ref = AN.apply_fft2n(G, x)
    assert A.rel_l2(u.cpu().numpy(), ref) < 1e-10
    plan.close()


@pytest.mark.parametrize("strategy", [vp.VP_BATCH_PERSISTENT, vp.VP_BATCH_GRAPH_STREAMS])
def test_batch_of_per_axis_grids(strategy):
    """The batch configuration's other reading: per-axis sizes drawn from
    {48, 64, 96, 128} (here smaller, for the oracle); every density of a mixed
    batch against the per-axis oracle."""
    specs = [((8, 12, 16), "helmholtz", 9.0), ((16, 8, 12), "laplace", 0.0), ((12, 16), "helmholtz", 20.0),
             ((24, 16, 8), "helmholtz", 15.0), ((8, 8, 8), "laplace", 0.0)]
    plans, fs, hs = [], [], []
    for i, (Ns, kern, k) in enumerate(specs):
        plans.append(Plan(len(Ns), Ns, kern, k, 0.0, precision="fp32"))
        h = I.random_complex_field(900 + i, Ns).astype(np.complex64)
        hs.append(h)
        fs.append(torch.from_numpy(h).to(DEV))
    b = vp.Batch(plans)
    b.set_strategy(strategy)
    outs = b.apply(fs)
    b.status()
    for (Ns, kern, k), h, o in zip(specs, hs, outs):
        L = 1.8 if len(Ns) == 3 else 1.5
        G = AN.ghat_full_from_octant(AN.ghat_octant_by_sums(AN.T_octant_by_sums(Ns, kern, k, L)))
        ref = AN.apply_fft2n(G, h.astype(np.complex128))
        assert A.rel_l2(o.cpu().numpy(), ref) < 1e-4, Ns
    b.close()
    for p in plans:
        p.close()
