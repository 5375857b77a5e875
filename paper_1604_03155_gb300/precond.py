"""Training and evaluation of the learned Lippmann-Schwinger preconditioner.

Any field x gives an exact pair (r, e) = (A x, x).  The fields used are the
ones the plain solver produces on seeded contrasts: the orthonormal Krylov
basis v_0 = b/||b||, ..., v_m of its first GMRES cycle (the kind of vector the
flexible iteration later hands the preconditioner) and the converged field u*
(r = b).  With s = sqrt(n)/||r|| the network learns (s r, q) -> s (e - r),
i.e. A^-1 - I, and the preconditioner is z = r + net(s r, q)/s.  Pairs are
generated on the fly (one contrast at a time) and the network is updated with
Adam after each pair; all arithmetic runs in the library's kernels (vp_ls_*,
vp_unet_*).
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs as I
from . import vp


def problem(plan, N: int, k: float, seed: int, dev):
    import torch
    q = torch.from_numpy(I.ls_contrast(seed, N).astype(np.float32)).to(dev)
    uinc = torch.from_numpy(I.plane_wave(N, k).astype(np.complex64)).to(dev)
    b = vp.ls_rhs(plan, q, uinc)
    return q, uinc, b


def train(plan, net, N: int, k: float, seeds, krylov: int = 12, lr: float = 1e-3, steps_per_pair: int = 1,
          restart: int = 20, onpolicy: bool = False, dev="cuda:0", log=None) -> dict:
    """Online training on the pairs (A v_j, v_j), j = 0..krylov, and (b, u*)
    of each contrast in ``seeds``.  With ``onpolicy`` also on (A z_j, z_j) for
    the directions z_j = M(v_j) of one flexible GMRES cycle preconditioned by
    the network itself: when M is close to A^-1, A z_j is close to the v_j the
    network is applied to inside the solver."""
    import torch
    x = torch.empty((3, N, N, N), dtype=torch.float32, device=dev)
    t = torch.empty((2, N, N, N), dtype=torch.float32, device=dev)
    losses = []
    t0 = time.perf_counter()
    per = None
    for ci, seed in enumerate(seeds):
        q, uinc, b = problem(plan, N, k, seed, dev)
        ustar = torch.zeros_like(b)
        vp.ls_solve(plan, q, b, ustar, tol=1e-7, maxit=3000, restart=restart)
        pairs = [(b, ustar)]
        for v in vp.ls_krylov_basis(plan, q, b, krylov):
            pairs.append((vp.ls_operator(plan, q, v), v))
        if onpolicy:
            net.bind(q)
            for z in vp.ls_flexible_basis(plan, q, b, krylov, net):
                pairs.append((vp.ls_operator(plan, q, z), z))
        per = len(pairs)
        for r, e in pairs:
            vp.ls_training_pair(plan, q, r, None, e, x, t)
            for _ in range(steps_per_pair):
                losses.append(net.loss_grad(x, t))
                net.adam_step(lr)
        if log and (ci + 1) % 25 == 0:
            log(f"contrast {ci + 1}/{len(seeds)} loss {np.mean(losses[-25 * per:]):.4e}")
    per = per or 1
    return {"pairs": len(losses), "first_loss": float(np.mean(losses[:per * 2])),
            "last_loss": float(np.mean(losses[-per * 2:])), "seconds": time.perf_counter() - t0}


def evaluate(plan, net, N: int, k: float, seeds, tol: float = 1e-6, restart: int = 20, dev="cuda:0") -> dict:
    """Plain vs preconditioned solves on held-out contrasts (true FP64 residual)."""
    import torch
    rows = []
    for seed in seeds:
        q, uinc, b = problem(plan, N, k, seed, dev)
        u = torch.zeros_like(b)
        plain = vp.ls_solve(plan, q, b, u, u_inc=uinc, tol=tol * 0.3, maxit=4000, restart=restart)
        torch.cuda.synchronize()
        u2 = torch.zeros_like(b)
        net.bind(q)
        pre = vp.ls_solve(plan, q, b, u2, u_inc=uinc, tol=tol * 0.3, maxit=4000, restart=restart, precond=net)
        torch.cuda.synchronize()
        rows.append({"seed": seed, "plain": plain, "precond": pre})
    agg = {
        "plain_iterations": float(np.mean([r["plain"]["iterations"] for r in rows])),
        "precond_iterations": float(np.mean([r["precond"]["iterations"] for r in rows])),
        "plain_seconds": float(np.mean([r["plain"]["seconds"] for r in rows])),
        "precond_seconds": float(np.mean([r["precond"]["seconds"] for r in rows])),
        "plain_true_residual_max": float(max(r["plain"]["true_residual"] for r in rows)),
        "precond_true_residual_max": float(max(r["precond"]["true_residual"] for r in rows)),
        "fallbacks": int(sum(r["precond"]["used_fallback"] for r in rows)),
        "contrasts": len(rows),
    }
    return {"summary": agg, "rows": rows}


def save_weights(net, path: str):
    np.save(path, net.get(0))


def load_weights(net, path: str):
    net.set_weights(np.load(path))


def save_checkpoint(net, path: str, **extra):
    """Weights, Adam state and any extra scalars (e.g. the next contrast index)
    in one .npz file."""
    m, v, step = net.get_adam()
    np.savez(path, weights=net.get(0), adam_m=m, adam_v=v, adam_step=np.int64(step),
             **{k: np.asarray(val) for k, val in extra.items()})


def load_checkpoint(net, path: str) -> dict:
    """Restores weights and Adam state; returns the extra scalars."""
    z = np.load(path)
    net.set_weights(z["weights"])
    net.set_adam(z["adam_m"], z["adam_v"], int(z["adam_step"]))
    return {k: z[k].item() for k in z.files if k not in ("weights", "adam_m", "adam_v", "adam_step")}
