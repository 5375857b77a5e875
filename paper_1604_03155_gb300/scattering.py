"""Scattering experiments of Section 5.3 on the GPU (the paper's Tables 4, 5
and 7): the smoothly filtered disk and the Luneburg lens in 2D and the smoothed
cube in 3D, a plane wave incident along the first axis, solved with the
library's Bi-CGStab (vp_ls_bicgstab) at tolerance 1e-12.

For each box size (in free-space wavelengths, k = 2 pi size) the scattered
field is solved on a fine reference grid and on coarser grids nested in it
(N_ref / N an integer: with x_p = (p - N/2 + 1)/N, coarse point p is fine
point m (p + 1) - 1), and

    E2   = ||u_N - u_ref||_2 / ||u_ref||_2     over the coarse points
    Einf = max |u_N - u_ref| / max |u_ref|

with N_matvec (operator products of the iteration), T_solve (right-hand side,
iteration and final apply, seconds) and T_precomp (plan creation: the FP64
multiplier and FFT tables, seconds).

    python -m paper_1604_03155_gb300.scattering --tables disk,lens,cube --out results.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs as I
from . import vp

# (d, contrast, [(size in wavelengths, reference N, [grid N ...]), ...]); every
# grid N divides its reference N, and 2N is a built FFT length
TABLES = {
    "disk": (2, I.filtered_disk, [(1, 768, [16, 24, 32, 48]), (20, 768, [64, 96, 128, 192]),
                                  (80, 2048, [256, 512, 1024])]),
    "lens": (2, I.luneburg_lens, [(1, 2048, [256, 512, 1024]), (20, 2048, [256, 512, 1024]),
                                  (40, 2048, [256, 512, 1024]), (60, 2048, [512, 1024])]),
    "cube": (3, I.cube_bump, [(1, 384, [32, 48, 64]), (20, 384, [64, 96, 128]), (40, 384, [128, 192])]),
}
DELTA = 1e-2  # reliable-update threshold of the mixed-precision solver
REF_PRECISION = "fp64"  # precision of the reference solves
MIXED_MAXIT = 3000  # FP32 iteration budget of a mixed solve before its FP64 phase

QUICK = {
    "disk": (2, I.filtered_disk, [(1, 256, [16, 32]), (20, 256, [64, 128])]),
    "lens": (2, I.luneburg_lens, [(1, 512, [128, 256])]),
    "cube": (3, I.cube_bump, [(1, 96, [24, 32, 48])]),
}


def solve(d: int, contrast, N: int, size: float, precision: str, form: str, tol: float, maxit: int):
    """One solve on the N^d grid; returns (u on the device, stats, T_precomp)."""
    import torch
    k = 2 * np.pi * size
    dev = torch.device("cuda", torch.cuda.current_device())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = vp.Plan(d, N, "helmholtz", k, 0.0, precision="fp32" if precision == "mixed" else precision)
    torch.cuda.synchronize()
    t_pre = time.perf_counter() - t0
    rdt, cdt = (torch.float32, torch.complex64) if precision == "fp32" else (torch.float64, torch.complex128)
    q = torch.from_numpy(contrast(N)).to(dev, rdt)
    uinc = torch.from_numpy(I.plane_wave(N, k, d)).to(dev, cdt)
    if precision == "mixed":  # FP32 iterations, FP64 reliable updates (an FP64 phase after MIXED_MAXIT)
        u, stats = vp.ls_bicgstab_mixed(plan, q, uinc, form=form, tol=tol, delta=DELTA, maxit=min(maxit, MIXED_MAXIT))
    else:
        u, stats = vp.ls_bicgstab(plan, q, uinc, form=form, tol=tol, maxit=maxit)
    plan.close()
    return u, stats, t_pre


def nested(u_ref, N: int):
    """The reference field at the points of the nested N grid."""
    m = u_ref.shape[0] // N
    sl = slice(m - 1, None, m)
    return u_ref[(sl,) * u_ref.dim()]


def errors(u, u_ref_coarse):
    import torch
    diff = u.to(torch.complex128) - u_ref_coarse
    e2 = float(torch.linalg.vector_norm(diff) / torch.linalg.vector_norm(u_ref_coarse))
    einf = float(diff.abs().max() / u_ref_coarse.abs().max())
    return e2, einf


def run_table(name: str, spec, precision: str, form: str, tol: float, maxit: int, log=print):
    d, contrast, rows = spec
    out = []
    for size, n_ref, grids in rows:
        u_ref, st_ref, pre_ref = solve(d, contrast, n_ref, size, REF_PRECISION, form, 1e-12, maxit)
        rec = dict(table=name, size=size, N=n_ref, N_tot=n_ref ** d, reference=True, precision=REF_PRECISION, form=form,
                   matvecs=st_ref["matvecs"], updates=st_ref["restarts"], fallback=st_ref["used_fallback"],
                   T_solve=st_ref["seconds"], T_precomp=pre_ref,
                   residual=st_ref["estimated_residual"], true_residual=st_ref["true_residual"])
        out.append(rec)
        log(json.dumps(rec))
        for N in grids:
            assert n_ref % N == 0
            u, st, pre = solve(d, contrast, N, size, precision, form, tol, maxit)
            e2, einf = errors(u, nested(u_ref, N))
            rec = dict(table=name, size=size, N=N, N_tot=N ** d, reference=False, precision=precision, form=form,
                       E2=e2, Einf=einf, matvecs=st["matvecs"], updates=st["restarts"],
                       fallback=st["used_fallback"], T_solve=st["seconds"], T_precomp=pre,
                       residual=st["estimated_residual"], true_residual=st["true_residual"])
            out.append(rec)
            log(json.dumps(rec))
            del u
        del u_ref
    return out


def markdown(rows) -> str:
    lines = ["| table | size (wavelengths) | N_tot | N | E2 | Einf | N_matvec | T_solve (s) | T_precomp (s) |",
             "|---|---|---|---|---|---|---|---|---|"]
    for r in rows:
        e2 = "-" if r["reference"] else f"{r['E2']:.2e}"
        ei = "-" if r["reference"] else f"{r['Einf']:.2e}"
        lines.append(f"| {r['table']} ({r['precision']}) | {r['size']} | {r['N_tot']} | {r['N']} | {e2} | {ei} | "
                     f"{r['matvecs']} | {r['T_solve']:.3f} | {r['T_precomp']:.3f} |")
    return "\n".join(lines)


def main(argv=None):
    global DELTA, REF_PRECISION, MIXED_MAXIT
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--tables", default="disk,lens,cube")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "mixed"],
                    help="mixed: FP32 iterations with FP64 reliable updates (FP64 accuracy)")
    ap.add_argument("--delta", type=float, default=None, help="reliable-update threshold (mixed), default 1e-2")
    ap.add_argument("--reference-precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--mixed-maxit", type=int, default=None,
                    help=f"FP32 iteration budget of a mixed solve, default {MIXED_MAXIT}")
    ap.add_argument("--form", default="density", choices=["density", "field"])
    ap.add_argument("--tol", type=float, default=None, help="default 1e-12 (fp64), 1e-6 (fp32)")
    ap.add_argument("--maxit", type=int, default=20000)
    ap.add_argument("--quick", action="store_true", help="small grids only")
    ap.add_argument("--single", default=None, metavar="TABLE:SIZE:N",
                    help="one solve (no reference), e.g. disk:20:512; prints its stats")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    DELTA = DELTA if a.delta is None else a.delta
    MIXED_MAXIT = MIXED_MAXIT if a.mixed_maxit is None else a.mixed_maxit
    REF_PRECISION = a.reference_precision
    tol = a.tol if a.tol is not None else (1e-6 if a.precision == "fp32" else 1e-12)
    if a.single:
        name, size, N = a.single.split(":")
        d, contrast, _ = TABLES[name]
        u, st, pre = solve(d, contrast, int(N), float(size), a.precision, a.form, tol, a.maxit)
        print(json.dumps(dict(table=name, size=float(size), N=int(N), precision=a.precision, form=a.form,
                              T_precomp=pre, **st)))
        return
    specs = QUICK if a.quick else TABLES
    rows = []
    for name in a.tables.split(","):
        rows += run_table(name, specs[name], a.precision, a.form, tol, a.maxit)
    print(markdown(rows))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
