"""Tile-shape autotuner of the FP32 four-step passes (vp_plan_autotune,
vp_plan_pass_config, vp_plan_set_pass_config): every candidate shape of every
pass computes the same potential.  Small grids are held to the FP64 oracle at
the flat FP32 bar (relative L2 <= 1e-5); on larger 3D grids each candidate is
compared with candidate 0, the measured default that the full-size tests hold
to the oracle, at relative L2 <= 1e-6 (two FP32 summation orders)."""
import os

import numpy as np
import pytest
import torch

from oracle import apply as A
from oracle_cases import check, condition, potential
from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300.vp import Plan, VPError

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
NPASS = 5


def _density(d, N, seed):
    src = I.random_gaussians(seed, 6, d)
    return I.sample_gaussians(src, N).astype(np.complex64)


def _apply(plan, f):
    phi = plan.apply(torch.from_numpy(f).to(DEV))
    torch.cuda.synchronize()
    return phi.cpu().numpy()


def _candidates(plan):
    """(pass, candidate) pairs of the four-step passes, candidate 0 excluded."""
    out = []
    for p in range(NPASS):
        cfg, count, name = plan.pass_config(p)
        assert cfg == 0
        out += [(p, c) for c in range(1, count)]
    return out


def _set(plan, p, c):
    try:
        plan.set_pass_config(p, c)
        return True
    except VPError:  # the shape exceeds a CTA's shared memory
        return False


@pytest.mark.parametrize("d,N,kernel,k", [(3, 32, "helmholtz", 17.0), (2, 64, "helmholtz", 40.0),
                                          (2, 128, "laplace", 0.0), (2, 256, "helmholtz", 40.0),
                                          (2, 512, "helmholtz", 40.0)])
def test_every_shape_against_oracle(d, N, kernel, k):
    plan = Plan(d, N, kernel, k, 0.0, precision="fp32")
    L = 1.8 if d == 3 else 1.5
    f = _density(d, N, 7000 + N)
    ref, _ = potential(d, N, kernel, k, L, f)
    kappa = condition(d, N, kernel, k, L, f)
    cands = _candidates(plan)
    assert cands, "the four-step passes have candidate shapes"
    assert check(f"shapes {d}d N={N} default", A.rel_l2(_apply(plan, f), ref), 1e-5, kappa)
    for p, c in cands:
        if not _set(plan, p, c):
            continue
        name = plan.pass_config(p)[2]
        assert check(f"shapes {d}d N={N} {plan.PASS_NAMES[p]} {name}", A.rel_l2(_apply(plan, f), ref), 1e-5, kappa)
        plan.set_pass_config(p, 0)
    plan.close()


@pytest.mark.parametrize("N", [64, 128, 256])
def test_every_shape_3d_against_default(N):
    plan = Plan(3, N, "helmholtz", 30.0, 0.0, precision="fp32")
    f = _density(3, N, 7100 + N)
    base = _apply(plan, f)
    assert np.isfinite(base).all()
    for p, c in _candidates(plan):
        if not _set(plan, p, c):
            continue
        err = A.rel_l2(_apply(plan, f), base)
        print(f"PARITY shapes 3d N={N} {plan.PASS_NAMES[p]} {plan.pass_config(p)[2]} rel_l2_vs_default={err:.2e}")
        assert err < 1e-6, (N, p, c, err)
        plan.set_pass_config(p, 0)
    plan.close()


def test_set_pass_config_rejects_bad_indices():
    plan = Plan(3, 32, "helmholtz", 10.0, 0.0, precision="fp32")
    with pytest.raises(VPError):
        plan.set_pass_config(2, 7)
    with pytest.raises(VPError):
        plan.set_pass_config(5, 0)
    plan2 = Plan(2, 64, "helmholtz", 10.0, 0.0, precision="fp32")
    assert plan2.pass_config(1)[2] == "absent"  # no axis-1 passes in 2D
    plan.close()
    plan2.close()


def test_autotune_choices_and_cache(tmp_path, monkeypatch):
    cache = tmp_path / "vp_autotune.txt"
    monkeypatch.setenv("VP_AUTOTUNE_CACHE", str(cache))
    N, k = 32, 17.0
    plan = Plan(3, N, "helmholtz", k, 0.0, precision="fp32")
    chosen = plan.autotune(force=True)
    print("autotune 3d N=32:", chosen)
    assert set(chosen) == set(plan.PASS_NAMES)
    text = cache.read_text()
    assert "|passes|3d32x32x32 " in text
    f = _density(3, N, 7200)
    ref, _ = potential(3, N, "helmholtz", k, 1.8, f)
    kappa = condition(3, N, "helmholtz", k, 1.8, f)
    assert check("autotuned 3d N=32", A.rel_l2(_apply(plan, f), ref), 1e-5, kappa)
    # a cached choice is reused: candidate 1 for the fused pass, 0 elsewhere
    key = text.strip().splitlines()[-1].rsplit(" ", 1)[0]
    with open(cache, "a") as fh:
        fh.write(f"{key} {(1 << 6) + 1}\n")
    plan2 = Plan(3, N, "helmholtz", k, 0.0, precision="fp32")
    plan2.autotune()
    assert [plan2.pass_config(p)[0] for p in range(NPASS)] == [0, 0, 1, 0, 0]
    assert check("cached choice 3d N=32", A.rel_l2(_apply(plan2, f), ref), 1e-5, kappa)
    plan.close()
    plan2.close()
