"""GPU apply (pruned pencil FFT passes, fused multiply, gradients) against the
FP64 CPU oracle on identical seeded inputs.  Bars: relative L2 <= 1e-12 for
the FP64 form and <= 1e-5 for FP32, gradients stacked over the d components
held to the same bars."""
import math

import numpy as np
import pytest
import torch

from oracle import apply as A
from oracle import closed_forms as CF
from oracle import kernel as K
from oracle_cases import check, condition, potential
from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300.vp import Plan, VPError

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}
CDT = {"fp32": torch.complex64, "fp64": torch.complex128}
NPC = {"fp32": np.complex64, "fp64": np.complex128}
DEV = "cuda:0"


def _density(d, N, seed, prec, n_gauss=6):
    src = I.random_gaussians(seed, n_gauss, d)
    return I.sample_gaussians(src, N).astype(NPC[prec])


def _run(plan, f, grad_mode=None):
    ft = torch.from_numpy(f).to(DEV)
    if grad_mode is None:
        phi = plan.apply(ft)
        torch.cuda.synchronize()
        return phi.cpu().numpy(), None
    plan.set_grad_mode(grad_mode)
    phi, g = plan.apply_grad(ft)
    torch.cuda.synchronize()
    return phi.cpu().numpy(), g.cpu().numpy()


SIZES3 = [4, 6, 8, 12, 16, 24, 32]
SIZES2 = [4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 256, 512]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("N", SIZES3)
@pytest.mark.parametrize("kernel,k", [("laplace", 0.0), ("helmholtz", 17.0)])
def test_apply_3d(prec, N, kernel, k):
    plan = Plan(3, N, kernel, k, 0.0, precision=prec)
    f = _density(3, N, 1000 + N, prec)
    phi, _ = _run(plan, f)
    ref, _ = potential(3, N, kernel, k, 1.8, f)
    assert check(f"3d {kernel} k={k} N={N} {prec}", A.rel_l2(phi, ref), TOL[prec], condition(3, N, kernel, k, 1.8, f))
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("N", SIZES2)
@pytest.mark.parametrize("kernel,k", [("laplace", 0.0), ("helmholtz", 40.0)])
def test_apply_2d(prec, N, kernel, k):
    plan = Plan(2, N, kernel, k, 0.0, precision=prec)
    f = _density(2, N, 2000 + N, prec)
    phi, _ = _run(plan, f)
    ref, _ = potential(2, N, kernel, k, 1.5, f)
    assert check(f"2d {kernel} k={k} N={N} {prec}", A.rel_l2(phi, ref), TOL[prec], condition(2, N, kernel, k, 1.5, f))
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mode", ["exact", "spectral2n"])
@pytest.mark.parametrize("d,N,kernel,k", [(3, 8, "helmholtz", 9.0), (3, 12, "laplace", 0.0), (3, 16, "helmholtz", 30.0),
                                          (2, 6, "laplace", 0.0), (2, 32, "helmholtz", 40.0), (2, 96, "helmholtz", 25.0),
                                          (2, 128, "laplace", 0.0)])
def test_apply_grad(prec, mode, d, N, kernel, k):
    plan = Plan(d, N, kernel, k, 0.0, precision=prec)
    f = _density(d, N, 3000 + N, prec)
    phi, g = _run(plan, f, mode)
    L = 1.8 if d == 3 else 1.5
    ref_phi, ref_g = potential(d, N, kernel, k, L, f, mode)
    kap = condition(d, N, kernel, k, L, f)
    kap_g = max([kap] + [condition(d, N, kernel, k, L, f, j) for j in range(d)]) if mode == "exact" else kap
    name = f"grad {mode} {d}d {kernel} k={k} N={N} {prec}"
    assert check(name + " phi", A.rel_l2(phi, ref_phi), TOL[prec], kap)
    assert check(name + " grad", A.rel_l2(g, ref_g), TOL[prec], kap_g)
    # grad without phi
    plan.set_grad_mode(mode)
    _, g2 = plan.apply_grad(torch.from_numpy(f).to(DEV), with_phi=False)
    torch.cuda.synchronize()
    assert check(name + " grad only", A.rel_l2(g2.cpu().numpy(), ref_g), TOL[prec], kap_g)
    plan.close()


@pytest.mark.parametrize("prec,rdt", [("fp32", np.float32), ("fp64", np.float64)])
@pytest.mark.parametrize("d,N", [(3, 16), (2, 64)])
def test_laplace_real_path(prec, rdt, d, N):
    plan = Plan(d, N, "laplace", 0.0, 0.0, precision=prec)
    f = _density(d, N, 4000 + N, prec).real.astype(rdt)
    phi = plan.apply(torch.from_numpy(f).to(DEV)).cpu().numpy()
    ref, _ = potential(d, N, "laplace", 0.0, 1.8 if d == 3 else 1.5, f)
    assert phi.dtype == rdt
    assert A.rel_l2(phi, ref.real) < TOL[prec]
    with pytest.raises(VPError):
        Plan(d, N, "helmholtz", 3.0, 0.0, precision=prec).apply(torch.from_numpy(f).to(DEV))
    plan.close()


def test_delta_response_is_the_kernel():
    """Section 4: T is the response to a unit source at a node."""
    N = 12
    plan = Plan(3, N, "helmholtz", 11.0, 0.0, precision="fp64")
    f = np.zeros((N, N, N), np.complex128)
    p0 = (N // 2 - 1,) * 3  # the origin node
    f[p0] = 1.0
    phi = plan.apply(torch.from_numpy(f).to(DEV)).cpu().numpy()
    T = plan.get_array("T")  # GPU precompute, octant
    Tf = K.T_full_from_octant(T)
    idx = np.arange(N) - p0[0] + N  # offset p - p0 -> index + N
    assert np.abs(phi - Tf[np.ix_(idx, idx, idx)]).max() < 1e-15 * np.abs(T).max()
    plan.close()


def test_zero_input_and_repeated_calls():
    plan = Plan(2, 32, "helmholtz", 10.0, 0.0)
    z = torch.zeros((32, 32), dtype=torch.complex64, device=DEV)
    assert torch.count_nonzero(plan.apply(z)).item() == 0
    f = _density(2, 32, 77, "fp32")
    ft = torch.from_numpy(f).to(DEV)
    a = plan.apply(ft).cpu().numpy()
    plan.apply_grad(ft)
    b = plan.apply(ft).cpu().numpy()
    assert np.array_equal(a, b)  # deterministic, workspace reuse is clean
    plan.close()


def test_host_pointer_path_matches_device_path():
    N = 16
    plan = Plan(3, N, "helmholtz", 20.0, 0.0)
    f = _density(3, N, 55, "fp32")
    dev = plan.apply(torch.from_numpy(f).to(DEV)).cpu().numpy()
    host = plan.apply(f)  # numpy in, numpy out, staged by the library
    assert isinstance(host, np.ndarray) and np.array_equal(host, dev)
    phi_h, g_h = plan.apply_grad(f)
    phi_d, g_d = plan.apply_grad(torch.from_numpy(f).to(DEV))
    assert np.array_equal(g_h, g_d.cpu().numpy())
    plan.close()


def test_dtype_precision_mismatch_rejected():
    plan = Plan(2, 16, "laplace", 0.0, 0.0, precision="fp32")
    with pytest.raises(VPError):
        plan.apply(torch.zeros((16, 16), dtype=torch.complex128, device=DEV))
    plan.close()


def test_workload_laplace3d_fp64_against_erf():
    """The N=32 3D Laplace Gaussian (sigma = 0.08) in FP64: <= 1e-12 vs the
    oracle and spectral accuracy (~3e-11) vs the erf closed form."""
    w = I.workload("laplace3d_single_gaussian")
    f = w.density()
    plan = Plan(3, 32, "laplace", 0.0, 1.8, precision="fp64")
    phi = plan.apply(torch.from_numpy(f).to(DEV)).cpu().numpy()
    ref, _ = potential(3, 32, "laplace", 0.0, 1.8, f)
    assert A.rel_l2(phi, ref) < 1e-12
    x = I.grid_coords(32)
    X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt(sum(a * a for a in X))
    ex = I.gaussian_amplitude(0.08, 3) * CF.laplace3(r, 0.08 / math.sqrt(2))
    assert A.rel_l2(phi, ex) < 5e-11
    plan.close()


def test_workload_helmholtz2d_n1024_grad_full():
    """2D Helmholtz k = 40, N = 1024, 8 Gaussians, FP32 apply with exact
    gradients: every element against the FP64 oracle (2N FFT form)."""
    w = I.workload("helmholtz2d_k40_n1024_grad")
    f = I.to_device_dtype(w.density(), "fp32")
    plan = Plan(2, 1024, "helmholtz", 40.0, 1.5, precision="fp32")
    phi, g = _run(plan, f, "exact")
    ref_phi, ref_g = potential(2, 1024, "helmholtz", 40.0, 1.5, f, "exact")
    assert A.rel_l2(phi, ref_phi) < 1e-5
    assert A.rel_l2(g, ref_g) < 1e-5
    plan.close()


@pytest.mark.parametrize("d,N,prec", [(2, 64, "fp32"), (3, 32, "fp64")])
def test_pinned_host_buffers_in_place_and_staged_match_device_path(d, N, prec):
    """Pinned host buffers are read and written in place by the first and last
    pass (or staged with host_access off): both give the device path's bits."""
    plan = Plan(d, N, "helmholtz", 11.0, 0.0, precision=prec)
    plan.set_grad_mode("exact")
    f = _density(d, N, 6000 + N, prec)
    phi_d, g_d = plan.apply_grad(torch.from_numpy(f).to(DEV))
    torch.cuda.synchronize()
    fp = torch.from_numpy(f).pin_memory()
    for direct in (True, False):
        plan.set_host_access(direct)
        phi_h = torch.empty_like(fp).pin_memory()
        g_h = torch.empty((d,) + fp.shape, dtype=fp.dtype).pin_memory()
        plan.apply_grad(fp, phi_h, g_h)
        assert torch.equal(phi_h, phi_d.cpu()) and torch.equal(g_h, g_d.cpu()), direct
    plan.close()
