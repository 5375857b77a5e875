"""Saved plans on the device: a plan loaded from vp_plan_save's file holds the
same FP64 arrays bit for bit and every apply (FP32, FP64, gradients) equals the
saved plan's bit for bit; a loaded plan without gradient kernels builds them
on first use exactly as a fresh plan does.  Timing of save / load against the
precompute is printed for the 3D N = 256 plan."""
import time

import numpy as np
import pytest
import torch

from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300.vp import Plan, VPError

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _density(dims, seed):
    src = I.random_gaussians(seed, 6, len(dims))
    f = I.sample_gaussians(src, dims[0]) if len(set(dims)) == 1 else I.sample_gaussians_grid(src, dims)
    return torch.from_numpy(np.ascontiguousarray(f).astype(np.complex64)).to(DEV)


def _arrays(plan, grad):
    out = {"T": plan.get_array("T"), "ghat": plan.get_array("ghat")}
    if grad:
        for j in range(plan.d):
            out[f"Tj{j}"] = plan.get_array("Tj", j)
            out[f"ghatj{j}"] = plan.get_array("ghatj", j)
    return out


def test_save_load_3d_with_gradients(tmp_path):
    N = 32
    plan = Plan(3, N, "helmholtz", 17.0, 0.0, precision="fp32")
    f = _density((N,) * 3, 9500)
    phi0, g0 = plan.apply_grad(f)
    torch.cuda.synchronize()
    path = tmp_path / "h3.vpplan"
    plan.save(path)
    q = Plan.load(path)
    assert q.d == 3 and q.dims == (N,) * 3 and q.kernel == "helmholtz"
    a0, a1 = _arrays(plan, True), _arrays(q, True)
    for name in a0:
        assert np.array_equal(a0[name], a1[name]), name
    phi1, g1 = q.apply_grad(f)
    torch.cuda.synchronize()
    assert torch.equal(phi0, phi1) and torch.equal(g0, g1)
    assert torch.equal(plan.apply(f), q.apply(f))
    for p in (plan, q):
        p.set_precision("fp64")
    f64 = f.to(torch.complex128)
    assert torch.equal(plan.apply(f64), q.apply(f64))
    plan.close()
    q.close()


def test_save_load_per_axis_grid_builds_gradients_later(tmp_path):
    dims = (32, 48)
    plan = Plan(2, dims, "laplace", 0.0, 0.0, precision="fp32")
    f = _density(dims, 9600)
    phi0 = plan.apply(f)
    path = tmp_path / "l2.vpplan"
    plan.save(path)  # no gradient kernels yet
    q = Plan.load(path)
    assert q.dims == dims and q.N == dims and q.kernel == "laplace"
    assert torch.equal(phi0, q.apply(f))
    _, g0 = plan.apply_grad(f)
    _, g1 = q.apply_grad(f)
    torch.cuda.synchronize()
    assert torch.equal(g0, g1)
    fr = f.real.contiguous()
    assert torch.equal(plan.apply(fr), q.apply(fr))
    plan.close()
    q.close()


def test_corrupted_file_is_refused(tmp_path):
    plan = Plan(3, 16, "biharmonic", 0.0, 0.0)
    path = tmp_path / "b.vpplan"
    plan.save(path)
    data = bytearray(path.read_bytes())
    data[200] ^= 1
    path.write_bytes(bytes(data))
    with pytest.raises(VPError, match="checksum"):
        Plan.load(path)
    plan.close()


def test_save_load_time_3d_n256(tmp_path):
    t0 = time.perf_counter()
    plan = Plan(3, 256, "helmholtz", 60.0, 1.8)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    path = tmp_path / "h256.vpplan"
    t0 = time.perf_counter()
    plan.save(path)
    t_save = time.perf_counter() - t0
    t0 = time.perf_counter()
    q = Plan.load(path)
    torch.cuda.synchronize()
    t_load = time.perf_counter() - t0
    print(f"PLANFILE 3d N=256: create {t_create:.3f} s, save {t_save:.3f} s, load {t_load:.3f} s, "
          f"{path.stat().st_size / 1e6:.0f} MB")
    f = _density((256,) * 3, 9700)
    assert torch.equal(plan.apply(f), q.apply(f))
    plan.close()
    q.close()
