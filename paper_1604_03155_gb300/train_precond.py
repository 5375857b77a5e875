"""Trains the learned Lippmann-Schwinger preconditioner and evaluates it.

    python -m paper_1604_03155_gb300.train_precond --N 128 --k 30 --contrasts 2000 \
        --heldout 50 --out paper_1604_03155_gb300/weights/unet_ls_k30_n128

Writes <out>.npy (the FP32 master weights, layer order of vp_unet),
<out>.ckpt.npz (weights, Adam state and the next contrast index, for --resume)
and <out>.json (training loss, and plain vs preconditioned flexible GMRES on the
held-out contrasts: iterations, seconds, true FP64 residual).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1604_03155_gb300 import inputs as I  # noqa: E402
from paper_1604_03155_gb300 import precond as P  # noqa: E402
from paper_1604_03155_gb300 import vp  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--k", type=float, default=30.0)
    ap.add_argument("--contrasts", type=int, default=2000)
    ap.add_argument("--heldout", type=int, default=50)
    ap.add_argument("--krylov", type=int, default=12)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--restart", type=int, default=20)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--slope", type=float, default=0.1, help="leaky-ReLU slope (1: linear network)")
    ap.add_argument("--init", default=None, help="start from these weights (.npy) instead of the seeded init")
    ap.add_argument("--first", type=int, default=0, help="index of the first training contrast")
    ap.add_argument("--onpolicy", action="store_true", help="add pairs from the network's own FGMRES directions")
    ap.add_argument("--resume", default=None,
                    help="continue from a checkpoint (.npz: weights, Adam state, next contrast index)")
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_1604_03155_gb300", "weights", "unet_ls_k30_n128"))
    a = ap.parse_args()
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    plan = vp.Plan(3, a.N, "helmholtz", a.k, 1.8, precision="fp32")
    net = vp.UNet(a.N, 16, weights=I.unet_init_weights(I.BASE_SEED + 901), slope=a.slope)
    if a.init:
        P.load_weights(net, a.init)
    if a.resume:
        a.first = int(P.load_checkpoint(net, a.resume).get("next_contrast", a.first))
    seeds = [I.LS_TRAIN_SEED + a.first + i for i in range(a.contrasts)]
    tr = P.train(plan, net, a.N, a.k, seeds, krylov=a.krylov, lr=a.lr, restart=a.restart, onpolicy=a.onpolicy,
                 log=lambda m: print(m, flush=True))
    P.save_weights(net, a.out + ".npy")
    P.save_checkpoint(net, a.out + ".ckpt.npz", next_contrast=a.first + a.contrasts)
    ev = P.evaluate(plan, net, a.N, a.k, [I.LS_HELDOUT_SEED + i for i in range(a.heldout)], tol=a.tol,
                    restart=a.restart)
    report = {"N": a.N, "k": a.k, "slope": a.slope, "contrasts": a.contrasts, "first": a.first, "init": a.init,
              "onpolicy": a.onpolicy, "krylov_pairs": a.krylov, "lr": a.lr,
              "restart": a.restart, "tol": a.tol, "train": tr, "heldout": ev["summary"]}
    with open(a.out + ".json", "w") as fh:
        json.dump(report, fh, indent=1)
    print(json.dumps(report), flush=True)


if __name__ == "__main__":
    main()
