"""The variable-coefficient Poisson experiment of Section 5.2 (the paper's
Table 3) on the GPU, with a seeded synthetic 1235-atom molecule standing in for
the paper's protein: -eps sigma + grad(eps) . grad V[sigma] = rho solved with
restarted GMRES, the paper's solver (vp_pb_gmres, FP64), or with Bi-CGStab
(vp_pb_solve, FP64 or mixed precision), over the exact-gradient apply at
tolerance 1e-12; the potential phi = V[sigma] compared with a reference solve
on a finer grid that contains the coarse nodes (N_ref / N an integer).

    E2   = ||phi_N - phi_ref||_2 / ||phi_ref||_2 over the coarse nodes
    Einf = max |phi_N - phi_ref| / max |phi_ref|

with the iteration count, the operator products, T_solve (seconds) and
T_precomp (plan creation with the derivative multipliers, seconds).

    python -m paper_1604_03155_gb300.pb --solver gmres --out pb.json
"""
from __future__ import annotations

import argparse
import json
import time

from . import inputs as I
from . import vp

GRIDS = [64, 96, 128, 192]
N_REF = 384


def solve(N: int, mol, precision: str, tol: float, maxit: int, solver: str = "gmres", restart: int = 40):
    """One solve on the N^3 grid: (phi on the device, stats, T_precomp)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    eps, ge, rho = I.pb_fields(mol, N, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = vp.Plan(3, N, "laplace", 0.0, 0.0, precision="fp32" if precision == "mixed" else "fp64")
    plan.get_array("ghatj", 0)  # builds the derivative multipliers
    torch.cuda.synchronize()
    t_pre = time.perf_counter() - t0
    if solver == "gmres":
        sigma, st = vp.pb_gmres(plan, eps, ge.contiguous(), rho.to(torch.complex128), tol=tol, restart=restart,
                                maxit=maxit)
    else:
        sigma, st = vp.pb_solve(plan, eps, ge.contiguous(), rho.to(torch.complex128), tol=tol, maxit=maxit,
                                mixed=precision == "mixed")
    plan.set_precision("fp64")
    phi = plan.apply(sigma)
    plan.close()
    return phi, st, t_pre


def errors(phi, ref):
    import torch
    m = ref.shape[0] // phi.shape[0]
    sl = slice(m - 1, None, m)
    r = ref[sl, sl, sl]
    diff = phi - r
    return (float(torch.linalg.vector_norm(diff) / torch.linalg.vector_norm(r)),
            float(diff.abs().max() / r.abs().max()))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--solver", default="gmres", choices=["gmres", "bicgstab"])
    ap.add_argument("--restart", type=int, default=40, help="GMRES restart length")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"], help="mixed: Bi-CGStab only")
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--maxit", type=int, default=2000)
    ap.add_argument("--grids", default=",".join(str(n) for n in GRIDS))
    ap.add_argument("--ref", type=int, default=N_REF)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    if a.solver == "gmres" and a.precision != "fp64":
        ap.error("GMRES runs in FP64")
    mol = I.pb_molecule()
    rows = []
    ref, st, pre = solve(a.ref, mol, a.precision, a.tol, a.maxit, a.solver, a.restart)
    rows.append(dict(N=a.ref, N_tot=a.ref ** 3, reference=True, solver=a.solver, precision=a.precision,
                     iterations=st["iterations"],
                     matvecs=st["matvecs"], T_solve=st["seconds"], T_precomp=pre, residual=st["true_residual"]))
    print(json.dumps(rows[-1]), flush=True)
    for N in [int(v) for v in a.grids.split(",")]:
        assert a.ref % N == 0
        phi, st, pre = solve(N, mol, a.precision, a.tol, a.maxit, a.solver, a.restart)
        e2, einf = errors(phi, ref)
        rows.append(dict(N=N, N_tot=N ** 3, reference=False, solver=a.solver, precision=a.precision, E2=e2,
                         Einf=einf,
                         iterations=st["iterations"], matvecs=st["matvecs"], T_solve=st["seconds"], T_precomp=pre,
                         residual=st["true_residual"]))
        print(json.dumps(rows[-1]), flush=True)
    print("| N_tot | N | E2 | Einf | iterations | products | T_solve (s) | T_precomp (s) |")
    print("|---|---|---|---|---|---|---|---|")
    for r in rows:
        e2 = "-" if r["reference"] else f"{r['E2']:.2e}"
        ei = "-" if r["reference"] else f"{r['Einf']:.2e}"
        print(f"| {r['N_tot']} | {r['N']} | {e2} | {ei} | {r['iterations']} | {r['matvecs']} | {r['T_solve']:.3f} | "
              f"{r['T_precomp']:.3f} |")
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
