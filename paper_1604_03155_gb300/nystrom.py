"""Times the Nystrom entry kernels (Section 4, the remark after the discrete
convolution): dense blocks T(p_i - p'_j) of the discretised volume-integral
matrix for random target and source nodes, and batches of kernel entries at
random offsets, with CUDA events after warm-up.  Reports entries per second and
the output bandwidth (the blocks are written once; the FP64 octant they gather
from stays in L2 for N <= 128 in 3D).

    python -m paper_1604_03155_gb300.nystrom --d 3 --N 128 --rows 8192 --cols 8192
"""
from __future__ import annotations

import argparse
import json

from . import vp


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--d", type=int, default=3)
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--kernel", default="helmholtz")
    ap.add_argument("--k", type=float, default=30.0)
    ap.add_argument("--rows", type=int, default=8192)
    ap.add_argument("--cols", type=int, default=8192)
    ap.add_argument("--dtype", default="c128", choices=["c64", "c128"])
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--boxes", action="store_true",
                    help="rows and columns are the nodes of two sub-boxes of the grid (the index sets of a "
                         "hierarchical solver) instead of random nodes")
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    dt = torch.complex128 if a.dtype == "c128" else torch.complex64
    plan = vp.Plan(a.d, a.N, a.kernel, a.k if a.kernel == "helmholtz" else 0.0, 0.0)
    U = a.N ** a.d
    g = torch.Generator(device="cpu").manual_seed(1)
    if a.boxes:
        def box(count, corner):
            # the first `count` nodes of a sub-box whose last axis spans 32 nodes, in C order
            side = int(round((count / 32) ** (1.0 / (a.d - 1))))
            shape = [side] * (a.d - 1) + [32]
            idx = torch.stack(torch.meshgrid(*[torch.arange(n) for n in shape], indexing="ij"), -1).reshape(-1, a.d)
            idx = idx + torch.tensor(corner)
            flat = torch.zeros(idx.shape[0], dtype=torch.int64)
            for j in range(a.d):
                flat = flat * a.N + idx[:, j]
            return flat[:count].to(dev)
        rows = box(a.rows, [a.N // 8] * a.d)
        cols = box(a.cols, [a.N // 2] * a.d)
    else:
        rows = torch.randint(0, U, (a.rows,), generator=g).to(dev)
        cols = torch.randint(0, U, (a.cols,), generator=g).to(dev)
    off = torch.randint(-a.N + 1, a.N, (a.rows * 64, a.d), generator=g, dtype=torch.int32).to(dev)
    out = {}
    for name, fn, count in [("matrix_block", lambda: plan.matrix_block(rows, cols, dtype=dt), a.rows * a.cols),
                            ("kernel_entries", lambda: plan.kernel_entries(off, dtype=dt), off.shape[0])]:
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(a.reps):
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ms += s.elapsed_time(e)
        ms /= a.reps
        esize = 16 if dt == torch.complex128 else 8
        out[name] = {"entries": count, "ms": ms, "entries_per_s": count / (ms * 1e-3),
                     "output_GBps": count * esize / (ms * 1e-3) / 1e9}
    print(json.dumps({"d": a.d, "N": a.N, "kernel": a.kernel, "dtype": a.dtype, "boxes": a.boxes, **out}))
    plan.close()


if __name__ == "__main__":
    main()
