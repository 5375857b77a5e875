"""Host logic of bench.py's multi-rank path, on CPU with the gloo backend:
the max-over-ranks reduction of the timed region, the per-rank densities, and
the reference arm's silent non-zero ranks."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"max": got}, fh)
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks(tmp_path):
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    for r in range(2):
        with open(tmp_path / f"r{r}.json") as fh:
            assert json.load(fh)["max"] == 15.0


def test_max_over_ranks_single_process_is_identity():
    assert bench.max_over_ranks(3.25, "cpu") == 3.25


def test_each_rank_gets_its_own_density_of_the_same_recipe():
    wl = bench.WORKLOADS["helmholtz2d_k40_n1024_grad"]
    from paper_1604_03155_gb300 import inputs as I
    f0 = bench.density_for("helmholtz2d_k40_n1024_grad", wl, 0)
    f1 = bench.density_for("helmholtz2d_k40_n1024_grad", wl, 1)
    assert f0.shape == f1.shape == (1024, 1024)
    assert np.array_equal(f0, I.workload("helmholtz2d_k40_n1024_grad").density())
    assert not np.allclose(f0, f1)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
