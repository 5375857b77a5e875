"""vp_apply_pipeline: the apply of vp_apply / vp_apply_grad on a list of
host densities, with the copies of one density overlapping the transforms of
the next.  Each output must equal the single-density call on the same density
bit for bit (the same kernels on the same workspace, only the copies are
scheduled differently), and the potential is held to the FP64 oracle at the
flat FP32 bar (relative L2 <= 1e-5, Section 4's apply)."""
import numpy as np
import pytest
import torch

from oracle import apply as A
from oracle_cases import check, condition, potential
from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300.vp import Plan, VPError

pytestmark = pytest.mark.gpu


def _densities(d, N, count, seed, dtype=np.complex64):
    out = []
    for i in range(count):
        src = I.random_gaussians(seed + i, 6, d)
        out.append(torch.from_numpy(I.sample_gaussians(src, N).astype(dtype)).pin_memory())
    return out


@pytest.mark.parametrize("d,N,kernel,k,count", [(3, 32, "helmholtz", 17.0, 1), (3, 32, "helmholtz", 17.0, 5),
                                                (3, 64, "laplace", 0.0, 7), (2, 128, "helmholtz", 40.0, 4)])
def test_pipeline_equals_single_applies_and_oracle(d, N, kernel, k, count):
    plan = Plan(d, N, kernel, k, 0.0, precision="fp32")
    plan.set_host_access(False)
    fs = _densities(d, N, count, 8100 + N)
    phis, grads = plan.apply_pipeline(fs)
    assert grads is None and len(phis) == count
    for f, phi in zip(fs, phis):
        one = plan.apply(f)
        assert torch.equal(phi, one), "pipelined and single apply differ"
    # a second call reuses the slots
    phis2, _ = plan.apply_pipeline(fs[::-1])
    for a, b in zip(phis2, phis[::-1]):
        assert torch.equal(a, b)
    L = 1.8 if d == 3 else 1.5
    f0 = fs[-1].numpy()
    ref, _ = potential(d, N, kernel, k, L, f0)
    assert check(f"pipeline {d}d N={N} {kernel} x{count}", A.rel_l2(phis[-1].numpy(), ref), 1e-5,
                 condition(d, N, kernel, k, L, f0))
    plan.close()


@pytest.mark.parametrize("with_phi", [True, False])
def test_pipeline_gradients_equal_apply_grad(with_phi):
    d, N, count = 2, 64, 5
    plan = Plan(d, N, "helmholtz", 30.0, 0.0, precision="fp32")
    fs = _densities(d, N, count, 8300)
    phis, grads = plan.apply_pipeline(fs, with_phi=with_phi, with_grad=True)
    for i, f in enumerate(fs):
        phi1, g1 = plan.apply_grad(f, with_phi=with_phi)
        assert torch.equal(grads[i], g1)
        if with_phi:
            assert torch.equal(phis[i], phi1)
        else:
            assert phis is None
    plan.close()


def test_pipeline_real_laplace_fp64_and_pageable():
    d, N, count = 3, 32, 4
    plan = Plan(d, N, "laplace", 0.0, 0.0, precision="fp64")
    fs = [f.real.to(torch.float64).contiguous() for f in _densities(d, N, count, 8400)]  # pageable
    phis, _ = plan.apply_pipeline(fs)
    for f, phi in zip(fs, phis):
        assert phi.dtype == torch.float64
        assert torch.equal(phi, plan.apply(f))
    plan.close()


def test_pipeline_device_tensors_and_large_count():
    d, N, count = 3, 32, 12
    plan = Plan(d, N, "helmholtz", 10.0, 0.0, precision="fp32")
    fs = [f.to("cuda:0") for f in _densities(d, N, count, 8500)]
    phis, _ = plan.apply_pipeline(fs)
    torch.cuda.synchronize()
    for f, phi in zip(fs, phis):
        assert torch.equal(phi, plan.apply(f))
    torch.cuda.synchronize()
    plan.close()


def test_pipeline_rejects_bad_arguments():
    plan = Plan(3, 32, "helmholtz", 10.0, 0.0, precision="fp32")
    f = _densities(3, 32, 2, 8600)
    assert plan.apply_pipeline([]) == ([], [])
    with pytest.raises(VPError):  # both outputs off
        plan.apply_pipeline(f, with_phi=False, with_grad=False)
    with pytest.raises(VPError):  # phi aliases f
        plan.apply_pipeline(f, phis=f)
    with pytest.raises(VPError):  # mixed shapes
        plan.apply_pipeline([f[0], torch.zeros(16, 16, 16, dtype=torch.complex64)])
    with pytest.raises(VPError):  # dtype does not match the FP32 plan
        plan.apply_pipeline([x.to(torch.complex128) for x in f])
    plan.close()


def test_pipeline_tensor_core_precision():
    plan = Plan(3, 128, "helmholtz", 30.0, 0.0, precision="tc_bf16x2")
    fs = _densities(3, 128, 3, 8700)
    phis, _ = plan.apply_pipeline(fs)
    for f, phi in zip(fs, phis):
        assert torch.equal(phi, plan.apply(f))
    with pytest.raises(VPError):  # the tensor-core precisions serve the potential only
        plan.apply_pipeline(fs, with_grad=True)
    plan.close()


def test_pipeline_full_size_3d_n256():
    """The bench workload's grid (3D Helmholtz k = 60, N = 256: 2N = 512, the
    TMA fused pass): four densities through three slots, each output equal to
    the device-resident apply bit for bit."""
    N = 256
    plan = Plan(3, N, "helmholtz", 60.0, 1.8, precision="fp32")
    fs = _densities(3, N, 4, 8800)
    phis, _ = plan.apply_pipeline(fs)
    for f, phi in zip(fs, phis):
        dev = plan.apply(f.to("cuda:0"))
        torch.cuda.synchronize()
        assert torch.equal(phi, dev.cpu())
    plan.close()
