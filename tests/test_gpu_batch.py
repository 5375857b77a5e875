"""Batched persistent apply (vp_batch_*): many densities of uneven size, kernel
and wavenumber in one launch, against the FP64 oracle and the single-plan
apply; strategies, graph replays with new pointers, the bounded-wait timeout
path and the autotuner cache."""
import os

import numpy as np
import pytest
import torch

from oracle import apply as A
from oracle_cases import check, condition, potential
from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300 import vp
from paper_1604_03155_gb300.vp import Batch, Plan, VPError

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

MIXED = [(3, 8, "laplace", 0.0), (3, 12, "helmholtz", 7.0), (3, 16, "helmholtz", 25.0), (3, 24, "laplace", 0.0),
         (2, 16, "helmholtz", 30.0), (2, 32, "laplace", 0.0), (3, 32, "helmholtz", 12.0), (2, 48, "helmholtz", 9.0)]


def _make(specs, seed=0):
    plans, fs, hs = [], [], []
    for i, (d, N, kern, k) in enumerate(specs):
        plans.append(Plan(d, N, kern, k, 0.0, precision="fp32"))
        src = I.random_gaussians(I.BASE_SEED + 700 + 31 * i + seed, 4, d)
        h = I.sample_gaussians(src, N).astype(np.complex64)
        hs.append(h)
        fs.append(torch.from_numpy(h).to(DEV))
    return plans, fs, hs


@pytest.mark.parametrize("strategy", [vp.VP_BATCH_PERSISTENT, vp.VP_BATCH_PERSISTENT_ONE_PER_SM,
                                      vp.VP_BATCH_PER_DENSITY, vp.VP_BATCH_GRAPH_STREAMS])
def test_mixed_batch_against_oracle(strategy):
    plans, fs, hs = _make(MIXED)
    b = Batch(plans)
    b.set_strategy(strategy)
    outs = b.apply(fs)
    b.status()
    torch.cuda.synchronize()
    for (d, N, kern, k), h, o in zip(MIXED, hs, outs):
        L = 1.8 if d == 3 else 1.5
        ref, _ = potential(d, N, kern, k, L, h)
        assert check(f"batch {d}d {kern} k={k} N={N}", A.rel_l2(o.cpu().numpy(), ref), 1e-5,
                     condition(d, N, kern, k, L, h))
    b.close()


def test_replays_with_new_pointers_match_single_plan_apply():
    plans, fs, hs = _make(MIXED)
    b = Batch(plans)
    b.set_strategy(vp.VP_BATCH_PERSISTENT)
    for rep in range(3):
        fs2 = [f * (1.0 + 0.5j * rep) for f in fs]
        outs = [torch.full_like(f, float("nan")) for f in fs2]
        b.apply(fs2, outs)
        b.status()
        for p, f, o in zip(plans, fs2, outs):
            ref = p.apply(f)
            torch.cuda.synchronize()
            assert A.rel_l2(o.cpu().numpy(), ref.cpu().numpy()) < 2e-6
    b.close()


def test_bounded_wait_timeout_is_reported_and_recoverable():
    """A withheld dependency makes the dependent tiles give up after the
    timeout; the kernel finishes, the status reports VP_ERR_TIMEOUT and the
    batch works again once the dependency is restored."""
    plans, fs, hs = _make(MIXED[:3])
    b = Batch(plans)
    b.set_strategy(vp.VP_BATCH_PERSISTENT)
    b.set_timeout(0.002)
    b.withhold(1, 2)
    b.apply(fs)
    with pytest.raises(VPError) as ei:
        b.status()
    assert ei.value.status == vp.VP_ERR_TIMEOUT
    b.withhold(0, 0)  # restore
    b.set_timeout(2.0)
    outs = b.apply(fs)
    b.status()
    for p, f, o in zip(plans, fs, outs):
        ref = p.apply(f)
        torch.cuda.synchronize()
        assert A.rel_l2(o.cpu().numpy(), ref.cpu().numpy()) < 2e-6
    b.close()


def test_autotuner_chooses_and_caches(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("VP_AUTOTUNE_CACHE", str(cache))
    plans, fs, hs = _make(MIXED[:4])
    b = Batch(plans)
    assert b.strategy() == 0
    b.apply(fs)
    b.status()
    s, c = b.strategy(), b.chunk()
    assert s in (1, 2, 3, 4) and c in (4, 8, 16, 32)
    text = cache.read_text()
    assert "3d8x8x8" in text  # the key names every axis's size
    assert int(text.strip().split()[-1]) == s + 100 * c  # cached as strategy + 100 x chunk
    b.close()
    b2 = Batch(plans)  # a new batch of the same sizes reads the cached choice
    assert b2.strategy() == s and b2.chunk() == c
    b2.close()


@pytest.mark.parametrize("chunk", [1, 4, 32])
def test_persistent_chunk_sizes_against_oracle(chunk):
    """The persistent launch with work items of 1, 4 and 32 tiles gives the
    oracle's potentials (the chunk only changes how tiles are scheduled)."""
    plans, fs, hs = _make(MIXED)
    b = Batch(plans)
    b.set_strategy(vp.VP_BATCH_PERSISTENT)
    b.set_chunk(chunk)
    assert b.chunk() == chunk
    outs = b.apply(fs)
    b.status()
    for (d, N, kern, k), h, o in zip(MIXED, hs, outs):
        L = 1.8 if d == 3 else 1.5
        ref, _ = potential(d, N, kern, k, L, h)
        assert check(f"batch chunk {chunk} {d}d {kern} k={k} N={N}", A.rel_l2(o.cpu().numpy(), ref), 1e-5, 1.0)
    b.close()


def test_invalid_batches_rejected():
    p64 = Plan(3, 8, "laplace", 0.0, 0.0, precision="fp64")
    with pytest.raises(VPError):
        Batch([p64])
    p = Plan(3, 256, "laplace", 0.0, 0.0, precision="fp32")  # 2N = 512 not in the batch kernel
    with pytest.raises(VPError):
        Batch([p])


def test_workload_batch64_against_single_plan_and_oracle():
    """The 64-density recipe (N in {48, 64, 96, 128}, half Laplace, half
    Helmholtz k in [5, 40], four Gaussians each): every density against its own
    plan's apply, two of them against the oracle."""
    recipe = I.batch_recipe()
    plans = [Plan(3, w.N, w.kernel, w.k, 1.8, precision="fp32") for w in recipe]
    hs = [w.density().astype(np.complex64) for w in recipe]
    fs = [torch.from_numpy(h).to(DEV) for h in hs]
    b = Batch(plans)
    b.set_strategy(vp.VP_BATCH_PERSISTENT)
    outs = b.apply(fs)
    b.status()
    for p, f, o in zip(plans, fs, outs):
        ref = p.apply(f)
        torch.cuda.synchronize()
        assert A.rel_l2(o.cpu().numpy(), ref.cpu().numpy()) < 2e-6
    for i in (0, 40):
        w = recipe[i]
        if w.N > 64:
            continue
        ref, _ = potential(3, w.N, w.kernel, w.k, 1.8, hs[i])
        assert A.rel_l2(outs[i].cpu().numpy(), ref) < 1e-5
    b.close()
