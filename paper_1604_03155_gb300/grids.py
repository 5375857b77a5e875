"""Times the FP32 apply on cubic and per-axis grids (vp_plan_create_aniso),
16 Gaussian sources, with CUDA events on the plan's stream and a 256 MB L2
flush before every timed apply.  Reports ms per apply, grid points per second
and the per-pass times.

    python -m paper_1604_03155_gb300.grids --grids 128x128x128,128x128x64,64x96x128
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import inputs as I
from . import vp


def time_grid(Ns, kernel: str, k: float, reps: int):
    import torch
    dev = torch.device("cuda", 0)
    d = len(Ns)
    plan = vp.Plan(d, tuple(Ns), kernel, k, 0.0, precision="fp32")
    stream = torch.cuda.Stream(device=dev)
    plan.set_stream(stream)
    src = I.random_gaussians(I.BASE_SEED + 11, 16, d)
    X = np.meshgrid(*[I.grid_coords(N) for N in Ns], indexing="ij")
    f = np.zeros(Ns, dtype=np.complex128)
    for c, s, a in zip(src.centres, src.sigmas, src.amps):
        f += a * np.exp(-sum((X[j] - c[j]) ** 2 for j in range(d)) / s ** 2)
    ft = torch.from_numpy(f.astype(np.complex64)).to(dev)
    phi = torch.empty_like(ft)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(3):
            plan.apply(ft, phi)
        plan.set_timing(True)
        s_ = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        e_ = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        for i in range(reps):
            flush.fill_(float(i))
            s_[i].record(stream)
            plan.apply(ft, phi)
            e_[i].record(stream)
    torch.cuda.synchronize(dev)
    plan.set_timing(False)
    passes = {k: v[1] / v[0] for k, v in plan.get_timing().items() if v[0]}
    ms = sum(a.elapsed_time(b) for a, b in zip(s_, e_)) / reps
    plan.close()
    pts = int(np.prod(Ns))
    return dict(grid="x".join(str(n) for n in Ns), points=pts, ms=ms, pts_per_s=pts / (ms * 1e-3),
                passes_ms=passes)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--grids", default="128x128x128,128x128x64,64x96x128,96x128x128")
    ap.add_argument("--kernel", default="helmholtz")
    ap.add_argument("--k", type=float, default=30.0)
    ap.add_argument("--reps", type=int, default=50)
    a = ap.parse_args(argv)
    for g in a.grids.split(","):
        Ns = [int(v) for v in g.split("x")]
        print(json.dumps(time_grid(Ns, a.kernel, a.k if a.kernel == "helmholtz" else 0.0, a.reps)), flush=True)


if __name__ == "__main__":
    main()
