"""Benchmark of the volume-potential apply on GB300.

Default workload: 3D Helmholtz, k = 60, N = 256 (the apply runs on 512^3
complex64), sixteen random Gaussian sources, FP32 complex apply, FP64
precompute done once before timing.  The FP64 form, the three split-operand
tensor-core forms and cuFFT are timed beside it on the same plan and input,
each with its relative L2 error against the FP64 oracle at sampled nodes.
--workload selects the others (e.g. helmholtz2d_k40_n1024_grad: 2D Helmholtz,
k = 40, N = 1024, phi + 2 exact gradient fields).

One step = one vp_apply (vp_apply_grad) on inputs resident in HBM; L2 (129 MB)
is flushed by writing a 256 MB buffer before every timed step, outside the
timed events.  The metric is grid points per second per potential, N^d / t_step
(a gradient call counts once).  Printed as one JSON line on rank 0.

--impl reference times the CPU oracle (float64, its own FFT) on the host cores
instead: one worker process per core, each running one apply of the workload's
sources on a smaller grid per step; it is a deliberately slow correctness
reference.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "helmholtz2d_k40_n1024_grad": dict(d=2, N=1024, kernel="helmholtz", k=40.0, L=1.5, grad=True),
    "helmholtz3d_k60_n256": dict(d=3, N=256, kernel="helmholtz", k=60.0, L=1.8, grad=False),
    "laplace3d_single_gaussian": dict(d=3, N=32, kernel="laplace", k=0.0, L=1.8, grad=False),
    "biharmonic3d_n256": dict(d=3, N=256, kernel="biharmonic", k=0.0, L=1.8, grad=False),
    "batch64": dict(d=3, N=0, kernel="mixed", k=0.0, L=1.8, grad=False),
    "batch64_grids": dict(d=3, N=0, kernel="mixed", k=0.0, L=1.8, grad=False),
}
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
# split-operand tensor-core forms of the 3D fused pass: (16-bit parts, partial products)
TC_PRECISIONS = ["tc_bf16x2", "tc_fp16x2", "tc_bf16x3"]
TC_PRODUCTS = {"tc_bf16x2": 3, "tc_fp16x2": 3, "tc_bf16x3": 6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="helmholtz3d_k60_n256", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"] + TC_PRECISIONS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def measured_peak_bf16(sustained: bool):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        return float(pk["bf16_tflops_sustained" if sustained else "bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_BF16_TFLOPS, "fallback"


def tc_flops_per_launch(N: int, precision: str) -> float:
    """Tensor-core FLOPs of one fused pass: per tile of 8 pencils the four real
    GEMMs F1 (128 x 2N2 x N2), F3 and I1 (8N2 x 32 x 32) and I3 (128 x N2 x 2N2),
    2 FLOPs per multiply-add, times the partial products of the split."""
    n = 2 * N
    N2 = n // 16
    per_tile = 2 * (128 * 2 * N2 * N2 + 2 * 8 * N2 * 32 * 32 + 128 * N2 * 2 * N2)
    return per_tile * (n * n / 8) * TC_PRODUCTS[precision]


APPLY_KERNEL_SOURCES = ("pencil_fft.cuh", "apply_dispatch.cuh", "apply_f32.cu", "apply_f64.cu", "fourstep.cuh", "fourstep.cu")


def kernel_source_hash(extra=()) -> str:
    """Hash of the apply kernels' sources (the kernels the roofline is about)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1604_03155_gb300", "csrc")
    for fn in APPLY_KERNEL_SOURCES + tuple(extra):
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fn.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(pass_name: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None).  Tensor-core passes are keyed
    "fused_axis0[tc_...]" and hashed together with their own source."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.md")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash(("tc_fused.cu",) if "[tc_" in pass_name else ())
    for ln in open(path):
        parts = [p.strip() for p in ln.strip().strip("|").split("|")]
        if len(parts) >= 4 and parts[0] == pass_name and parts[1] == workload and parts[3] == want:
            try:
                return float(parts[2])
            except ValueError:
                return None
    return None


def pass_bytes(d: int, N: int, F: int, csize: int) -> dict:
    """Algorithmic bytes per launch of each pass (pruned schedule, U = N^d complex
    elements): reads of the nonzero half only, writes of the kept half only."""
    U = N ** d * csize
    oct_b = (N + 1) ** d * csize
    if d == 3:
        return {"fwd_rows": 3 * U, "fwd_axis1": 6 * U, "fused_axis0": 4 * U + F * oct_b + F * 4 * U,
                "inv_axis1": F * 6 * U, "inv_rows": F * 3 * U}
    return {"fwd_rows": 3 * U, "fused_axis0": 2 * U + F * oct_b + F * 2 * U, "inv_rows": F * 3 * U}


# ---------------------------------------------------------------------------
# oracle (CPU) timing: the cpu_baseline leg and the reference arm
# ---------------------------------------------------------------------------

def oracle_step(wl: dict, f: np.ndarray, Gf, Gjf):
    from oracle import apply as A
    phi = A.apply_fft2n(Gf, f)
    grads = [A.apply_fft2n(g, f) for g in Gjf] if wl["grad"] else []
    return phi, grads


def oracle_setup(wl: dict):
    from oracle import kernel as K
    d, N = wl["d"], wl["N"]
    T = K.T_octant_by_sums(d, N, wl["kernel"], wl["k"], wl["L"])
    Gf = K.ghat_full_from_octant(K.ghat_octant_by_sums(T, N))
    Gjf = []
    if wl["grad"]:
        for j in range(d):
            Tj = K.T_octant_by_sums(d, N, wl["kernel"], wl["k"], wl["L"], deriv_axis=j)
            Gjf.append(K.ghat_full_from_octant(K.ghat_octant_by_sums(Tj, N, odd_axis=j), odd_axis=j))
    return Gf, Gjf


def time_oracle(wl: dict, f: np.ndarray, steps: int, Gf=None, Gjf=None):
    if Gf is None:
        Gf, Gjf = oracle_setup(wl)
    f = np.asarray(f, dtype=np.complex128)
    wall, cpu = 0.0, 0.0
    out = None
    for _ in range(steps):
        t0, c0 = time.perf_counter(), time.process_time()
        out = oracle_step(wl, f, Gf, Gjf)
        wall += time.perf_counter() - t0
        cpu += time.process_time() - c0
    pts = wl["N"] ** wl["d"] * steps
    return {"value": pts / wall, "seconds": wall, "cores": round(cpu / wall, 2), "out": out}


def _oracle_worker(wl: dict, N: int, barrier, cmd, res):
    """One host core's share of the oracle timing (a spawned process: numpy and
    the oracle only): set up the workload's kernel on an N^d grid once, then per
    command one full apply, started together with the other workers."""
    sw = dict(wl, N=N)
    f = density_sample(wl, N)
    t0 = time.perf_counter()
    Gf, Gjf = oracle_setup(sw)
    res.put(("ready", time.perf_counter() - t0))
    while cmd.get() is not None:
        barrier.wait()
        t0, c0 = time.perf_counter(), time.process_time()
        oracle_step(sw, f, Gf, Gjf)
        res.put((t0, time.perf_counter(), time.process_time() - c0))


class OraclePool:
    """`procs` worker processes (spawn start method, so they are safe beside a
    CUDA context) that run the oracle apply concurrently, one per core."""

    def __init__(self, wl: dict, N: int, procs: int):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.N, self.d, self.procs = N, wl["d"], procs
        self.barrier = ctx.Barrier(procs)
        self.cmds = [ctx.Queue() for _ in range(procs)]
        self.res = ctx.Queue()
        self.ps = [ctx.Process(target=_oracle_worker, args=(wl, N, self.barrier, c, self.res), daemon=True)
                   for c in self.cmds]
        for p in self.ps:
            p.start()
        self.setup_seconds = []  # each worker's precompute (kernel octants and multipliers)
        for _ in self.ps:
            tag, secs = self.res.get(timeout=600)
            assert tag == "ready"
            self.setup_seconds.append(secs)

    def step(self) -> dict:
        """One apply on every worker at once: points/s of the whole host, wall
        seconds and the cores actually busy (CPU seconds / wall seconds)."""
        for c in self.cmds:
            c.put(1)
        r = [self.res.get(timeout=1800) for _ in self.ps]
        wall = max(x[1] for x in r) - min(x[0] for x in r)
        cpu = sum(x[2] for x in r)
        return {"value": self.procs * self.N ** self.d / wall, "seconds": wall, "cores": round(cpu / wall, 2)}

    def close(self):
        for c in self.cmds:
            c.put(None)
        for p in self.ps:
            p.join(timeout=60)


def host_cpu() -> dict:
    """nproc and the CPU model of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count() or 1, "cpu_model": model}


def cpu_baseline_sample_N(wl: dict) -> int:
    """Grid size of the oracle sample: the workload's own N when the apply is
    small (2D, or 3D N <= 64), else 64 (a 128^3 FFT convolution, a few seconds
    per core)."""
    if wl["d"] == 2 or wl["N"] <= 64:
        return min(wl["N"], 512) if wl["d"] == 2 else wl["N"]
    return 64


def cpu_baseline(wl: dict, name: str) -> dict:
    """The FP64 oracle as it stands on this host: all cores (one worker process
    each, one apply each, at once) and a single core, on the workload's sources,
    k and L sampled on a grid of cpu_baseline_sample_N points per axis."""
    hc = host_cpu()
    Ns = cpu_baseline_sample_N(dict(wl, name=name))
    w = dict(wl, name=name)
    pool = OraclePool(w, Ns, hc["nproc"])
    allc = pool.step()
    pool.close()
    one = OraclePool(w, Ns, 1)
    single = one.step()
    single_setup = one.setup_seconds[0]
    one.close()
    return {"value": allc["value"], "unit": "grid pts/s", "cores": allc["cores"], "kind": "oracle",
            "sample": (f"{hc['nproc']} worker processes at once, each one full apply "
                       f"({'phi + gradients' if wl['grad'] else 'phi'}) of the {name} workload's sources, k and L "
                       f"on an N={Ns} grid ({Ns ** wl['d']} points; the workload's N is {wl['N']}), FP64 oracle "
                       f"with its own FFT, {allc['seconds']:.1f} s wall"),
            "nproc": hc["nproc"], "cpu_model": hc["cpu_model"],
            "single_thread": {"value": single["value"], "unit": "grid pts/s", "cores": single["cores"],
                              "seconds": single["seconds"], "precompute_seconds": single_setup,
                              "precompute": f"the oracle's kernel octants and multipliers for the N={Ns} grid"}}


def oracle_reference(wl: dict, f_host: np.ndarray, npts: int = 40, seed: int = 1604) -> dict:
    """The FP64 oracle's values the forms are compared with: its full result
    (2N FFT form) on grids of at most 2^21 points, else its direct sums at
    sampled nodes (the 2^d corners and seeded random nodes; each value is the
    full sum over the grid)."""
    from oracle import apply as A
    from oracle import kernel as K
    d, N = wl["d"], wl["N"]
    f64 = np.asarray(f_host, dtype=np.complex128)
    if N ** d <= 2 ** 21:
        Gf, Gjf = oracle_setup(wl)
        phi_o, grads_o = oracle_step(wl, f64, Gf, Gjf)
        return {"kind": "full", "phi": phi_o, "grad": np.stack(grads_o) if grads_o else None,
                "what": "every output of the FP64 oracle (2N FFT form)"}
    T = K.T_octant_by_sums(d, N, wl["kernel"], wl["k"], wl["L"])
    corners = [tuple(c) for c in np.ndindex(*(2,) * d)]
    corners = [tuple((N - 1) * v for v in c) for c in corners]
    rng = np.random.default_rng(seed)
    pts = corners + [tuple(int(v) for v in rng.integers(0, N, d)) for _ in range(npts - len(corners))]
    vals = A.apply_direct_at_octant(T, f64, pts)
    grads = None
    if wl["grad"]:
        grads = np.stack([A.apply_direct_at_octant(K.T_octant_by_sums(d, N, wl["kernel"], wl["k"], wl["L"],
                                                                       deriv_axis=j), f64, pts, odd_axis=j)
                          for j in range(d)])
    return {"kind": "sampled", "points": pts, "phi": vals, "grad": grads,
            "what": f"the FP64 oracle's direct sums at {len(pts)} nodes (the {len(corners)} corners and "
                    f"{len(pts) - len(corners)} seeded random nodes), relative L2 over those nodes"}


def form_errors(ref: dict, phi, grad=None) -> dict:
    """Relative L2 of one form's phi (and gradient) against the oracle reference."""
    from oracle import apply as A
    if ref["kind"] == "full":
        e = {"phi": A.rel_l2(phi.cpu().numpy(), ref["phi"])}
        if grad is not None and ref["grad"] is not None:
            e["grad"] = A.rel_l2(grad.cpu().numpy(), ref["grad"])
        return e
    import torch
    idx = tuple(torch.tensor(c, device=phi.device) for c in zip(*ref["points"]))
    e = {"phi": A.rel_l2(phi[idx].cpu().numpy(), ref["phi"])}
    if grad is not None and ref["grad"] is not None:
        e["grad"] = A.rel_l2(np.stack([grad[j][idx].cpu().numpy() for j in range(grad.shape[0])]), ref["grad"])
    return e


def max_over_ranks(value: float, device) -> float:
    """The maximum of `value` over the ranks of the default process group (the
    slowest rank sets the job's time); `value` itself with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def density_for(name: str, wl: dict, rank: int = 0):
    from paper_1604_03155_gb300 import inputs as I
    if name == "laplace3d_single_gaussian":
        return I.workload(name).density()
    base = I.workload(name)
    src = I.random_gaussians(base.seed + 7919 * rank, base.n_gauss, base.d)
    return I.sample_gaussians(src, base.N)


def reference_sample_N(wl: dict, steps: int, budget_s: float = 120.0) -> int:
    """Grid size of one reference step: the largest power of two <= the
    workload's N whose oracle apply, estimated from a timed apply at N = 16 and
    the N^d log N cost of the FFT form, lets `steps` steps fit the budget."""
    d, N = wl["d"], wl["N"]
    n0 = 16
    cal = dict(wl, N=n0)
    f = density_sample(wl, n0)
    Gf, Gjf = oracle_setup(cal)
    oracle_step(cal, f, Gf, Gjf)
    t = time.perf_counter()
    oracle_step(cal, f, Gf, Gjf)
    t0 = time.perf_counter() - t
    per_step = budget_s / max(1, steps)
    n = n0
    while 2 * n <= N:
        m = 2 * n
        est = t0 * (m / n0) ** d * math.log2(2 * m) / math.log2(2 * n0)
        if est > per_step:
            break
        n = m
    return n


def density_sample(wl: dict, N: int):
    """The workload's density (same sources) sampled on an N^d grid."""
    from paper_1604_03155_gb300 import inputs as I
    name = wl["name"]
    if name == "laplace3d_single_gaussian":
        return I.workload(name).density(N).astype(np.complex128)
    if name.startswith("batch64"):  # the batch's first Helmholtz density stands for the batch
        base = I.batch_recipe()[32]
        return I.sample_gaussians(I.random_gaussians(base.seed, base.n_gauss, 3), N).astype(np.complex128)
    base = I.workload(name)
    return I.sample_gaussians(I.random_gaussians(base.seed, base.n_gauss, base.d), N).astype(np.complex128)


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, args.steps)
    wl = dict(wl, name=args.workload)
    if args.workload.startswith("batch64"):
        # per step one density of the batch (its first Helmholtz one: N, k), in grid points per second
        from paper_1604_03155_gb300 import inputs as I
        w = I.batch_recipe()[32]
        wl = dict(wl, N=w.N, kernel=w.kernel, k=w.k)
    Ns = reference_sample_N(wl, steps)
    hc = host_cpu()
    pool = OraclePool(wl, Ns, hc["nproc"])
    for _ in range(max(0, min(args.warmup, 1))):
        pool.step()
    rs = [pool.step() for _ in range(steps)]
    pool.close()
    wall = sum(r["seconds"] for r in rs)
    value = hc["nproc"] * Ns ** wl["d"] * steps / wall
    cores = round(sum(r["cores"] * r["seconds"] for r in rs) / wall, 2)
    unit = "grid pts/s"
    sample = (f"per step {hc['nproc']} worker processes at once (one per host core), each one full apply "
              f"(phi{' + gradients' if wl['grad'] else ''}) of the {args.workload} workload's sources, k and L on "
              f"an N={Ns} grid ({Ns ** wl['d']} points; the workload's N is {wl['N']}), FP64 oracle with its own "
              f"FFT; N chosen so that {steps} steps take about two minutes")
    line = {
        "impl": "reference",
        "metric": "grid pts/s per potential (N^d/s), % HBM roofline, vs plain FP64 at stated rel err",
        "value": value, "unit": unit, "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
        "ms_per_step": 1000 * wall / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, **{k: v for k, v in wl.items() if k != "name"}},
        "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample,
                         "nproc": hc["nproc"], "cpu_model": hc["cpu_model"]},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------

def run_ours(args, wl):
    import torch
    import torch.distributed as dist

    from paper_1604_03155_gb300.vp import Plan

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    d, N, F = wl["d"], wl["N"], (1 + wl["d"]) if wl["grad"] else 1
    prec = args.precision
    f32io = prec != "fp64"
    cdt = torch.complex64 if f32io else torch.complex128
    npdt = np.complex64 if f32io else np.complex128

    stream = torch.cuda.Stream(device=dev)
    t0 = time.perf_counter()
    plan = Plan(d, N, wl["kernel"], wl["k"], wl["L"], precision=prec, grad_mode="exact")
    if wl["grad"]:
        plan.get_array("ghatj", 0)  # builds the derivative multipliers (precompute)
    precompute_s = time.perf_counter() - t0
    plan.set_stream(stream)
    # tile shapes of the FP32 passes from the autotuner (cached per device, driver and grid)
    autotune = {}
    if prec == "fp32":
        t0 = time.perf_counter()
        autotune = {"shapes": plan.autotune(), "seconds": time.perf_counter() - t0}

    f_host = density_for(args.workload, wl, rank).astype(npdt)
    f = torch.from_numpy(f_host).to(dev)
    phi = torch.empty_like(f)
    grad = torch.empty((d,) + f.shape, dtype=cdt, device=dev) if wl["grad"] else None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        if wl["grad"]:
            plan.apply_grad(f, phi, grad)
        else:
            plan.apply(f, phi)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
    torch.cuda.synchronize(dev)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(vis.split(",")[local] if vis else local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    plan.get_timing()  # reset the per-pass counters
    plan.set_timing(True)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))  # evict L2 (256 MB > 129 MB), outside the timed events
            starts[i].record(stream)
            step()
            stops[i].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    plan.set_timing(False)
    passes = plan.get_timing()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in zip(starts, stops))
    if world > 1:
        total_ms = max_over_ranks(total_ms, dev)
    ms_per_step = total_ms / args.steps
    value = (N ** d) * world / (ms_per_step / 1000.0)

    # roofline of the dominant pass (per launch, events on the plan's stream)
    csize = 8 if f32io else 16
    pb = pass_bytes(d, N, F, csize)
    dom = max((k for k in passes if passes[k][0] > 0), key=lambda k: passes[k][1])
    dom_launches, dom_ms = passes[dom]
    dom_avg_s = dom_ms / dom_launches / 1000.0
    peak, peak_kind = measured_peak_hbm()
    achieved = pb[dom] / dom_avg_s / 1e9
    traffic = ncu_traffic(f"{dom}[{prec}]" if (prec in TC_PRECISIONS and dom == "fused_axis0") else dom,
                          args.workload)
    launches_per_step = plan.launch_count(wl["grad"])

    # end to end through the C ABI with host buffers (pinned), copies inside
    f_pin = torch.from_numpy(f_host).pin_memory()
    phi_pin = torch.empty_like(f_pin).pin_memory()
    grad_pin = torch.empty((d,) + f_pin.shape, dtype=cdt).pin_memory() if wl["grad"] else None
    e2e_steps = max(3, min(args.steps, 20))
    plan.set_stream(stream)

    def e2e_time(direct: bool) -> float:
        # pinned buffers read and written in place by the first and last pass
        # (direct), or staged through device memory with explicit copies
        plan.set_host_access(direct)
        for _ in range(2):
            plan.apply_grad(f_pin, phi_pin, grad_pin) if wl["grad"] else plan.apply(f_pin, phi_pin)
        te = time.perf_counter()
        for _ in range(e2e_steps):
            plan.apply_grad(f_pin, phi_pin, grad_pin) if wl["grad"] else plan.apply(f_pin, phi_pin)
        return (time.perf_counter() - te) / e2e_steps

    e2e_staged_s = e2e_time(False)
    e2e_seq_s = e2e_time(True)

    # the pipelined entry point: one call over e2e_pipe_steps densities (a ring
    # of 4 pinned inputs and outputs; every step copies its whole input in and
    # its outputs out), the copies of one density overlapping the transforms
    # of its neighbours
    ring = 4
    f_ring = [torch.from_numpy(f_host).pin_memory() for _ in range(ring)]
    phi_ring = [torch.empty_like(f_pin).pin_memory() for _ in range(ring)]
    grad_ring = [torch.empty_like(grad_pin).pin_memory() for _ in range(ring)] if wl["grad"] else None
    e2e_pipe_steps = max(8, min(args.steps, 200))

    def pipe_call(n):
        plan.apply_pipeline([f_ring[i % ring] for i in range(n)], [phi_ring[i % ring] for i in range(n)],
                            [grad_ring[i % ring] for i in range(n)] if wl["grad"] else None,
                            with_grad=bool(wl["grad"]))

    pipe_call(ring)
    if world > 1:
        dist.barrier()
    te = time.perf_counter()
    pipe_call(e2e_pipe_steps)
    e2e_s = max_over_ranks((time.perf_counter() - te) / e2e_pipe_steps, dev)
    last = (e2e_pipe_steps - 1) % ring
    pipe_ok = bool(torch.equal(phi_ring[last], phi.cpu()))
    if wl["grad"]:
        pipe_ok = pipe_ok and bool(torch.equal(grad_ring[last], grad.cpu()))
    U_b = (N ** d) * csize

    def time_form(form: str, reps: int = 20):
        """ms per step of the same apply in another precision on this plan, the
        per-pass timings of those steps and the outputs of the last one."""
        plan.set_precision(form)
        ff = f.to(torch.complex128) if form == "fp64" else f
        pp = torch.empty_like(ff)
        gg = torch.empty((d,) + ff.shape, dtype=ff.dtype, device=dev) if wl["grad"] else None
        s_ = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        e_ = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        with torch.cuda.stream(stream):
            for _ in range(3):
                plan.apply_grad(ff, pp, gg) if wl["grad"] else plan.apply(ff, pp)
            torch.cuda.synchronize(dev)
            plan.get_timing()
            plan.set_timing(True)
            for i in range(reps):
                flush.fill_(float(i))
                s_[i].record(stream)
                plan.apply_grad(ff, pp, gg) if wl["grad"] else plan.apply(ff, pp)
                e_[i].record(stream)
        torch.cuda.synchronize(dev)
        plan.set_timing(False)
        tim = plan.get_timing()
        plan.status()
        plan.set_precision(prec)
        return sum(a.elapsed_time(b) for a, b in zip(s_, e_)) / reps, tim, pp, gg

    def cufft_form(reps: int = 20) -> dict:
        """The same apply with cuFFT (torch.fft) for comparison only: f zero-padded to
        (2N)^d, one forward transform, per field a multiply by the full (2N)^d
        multiplier (unfolded from the plan's FP64 octants) and an inverse transform,
        cropped to N^d.  Not a product path."""
        n2 = 2 * N
        m = torch.arange(n2, device=dev)
        fold = torch.minimum(m, n2 - m)

        def full(octant, odd_axis=None):
            g = torch.from_numpy(octant).to(dev)
            idx = [fold.view([n2 if a == b else 1 for b in range(d)]) for a in range(d)]
            G = g[tuple(idx)]
            if odd_axis is not None:
                sgn = torch.where(m > N, -1.0, 1.0).to(torch.float64).view([n2 if b == odd_axis else 1 for b in range(d)])
                G = G * sgn
            return G.to(torch.complex64)

        Gs = [full(plan.get_array("ghat"))]
        if wl["grad"]:
            Gs += [full(plan.get_array("ghatj", j), j) for j in range(d)]
        crop = tuple(slice(0, N) for _ in range(d))
        fpad = torch.zeros((n2,) * d, dtype=torch.complex64, device=dev)

        def cstep():
            fpad[crop] = f
            F = torch.fft.fftn(fpad)
            return [torch.fft.ifftn(F * G)[crop] for G in Gs]

        with torch.cuda.stream(stream):
            for _ in range(3):
                outs = cstep()
            s_ = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
            e_ = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
            for i in range(reps):
                flush.fill_(float(i))
                s_[i].record(stream)
                outs = cstep()
                e_[i].record(stream)
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in zip(s_, e_)) / reps
        ref = outs[0].cpu().numpy()
        mine = phi.cpu().numpy()
        diff = float(np.linalg.norm((mine - ref).ravel()) / np.linalg.norm(ref.ravel()))
        del Gs, fpad, outs
        torch.cuda.empty_cache()
        return {"value": (N ** d) / (ms / 1000.0), "ms_per_step": ms, "speedup_of_this_form": ms / ms_per_step,
                "rel_l2_phi_vs_this_form": diff,
                "what": "torch.fft (cuFFT) C2C on the zero-padded (2N)^d grid, full multiplier, no pruning or fusion"}

    cufft = cufft_form() if f32io else None

    # the FP64 oracle's reference values for the error of every form (rank 0, N = 1)
    ref = oracle_reference(dict(wl, name=args.workload), f_host) if (rank == 0 and world == 1) else None
    errs = form_errors(ref, phi, grad) if ref is not None else None

    def form_line(form: str, reps: int) -> dict:
        ms_f, tim, pp, gg = time_form(form, reps)
        out = {"value": (N ** d) / (ms_f / 1000.0), "ms_per_step": ms_f, "speedup_of_this_form": ms_f / ms_per_step}
        if ref is not None:
            out["rel_l2_vs_oracle"] = form_errors(ref, pp, gg)
        if form in TC_PRECISIONS:
            fl_, fms = tim.get("fused_axis0", (0, 0.0))
            if fl_:
                t_s = fms / fl_ / 1000.0
                fl = tc_flops_per_launch(N, form)
                tpk, tkind = measured_peak_bf16(sustained=False)
                out["fused_axis0_ms"] = t_s * 1000.0
                out["tensor"] = {"kernel": "fused_axis0 (tcgen05)", "flops_per_launch": fl,
                                 "achieved_tflops": fl / t_s / 1e12, "peak_tflops": tpk, "peak_source": tkind,
                                 "frac": fl / t_s / 1e12 / tpk}
        del pp, gg
        torch.cuda.empty_cache()
        return out

    # FP64 form on the same grid (same kernels in double), for "vs plain FP64";
    # the split tensor-core forms of the fused pass (3D, 2N = 256 or 512) beside
    # the FP32 form; with a tensor-core --precision the FP32 form is the extra
    fp64 = form_line("fp64", 10) if prec != "fp64" else None
    extras = {}
    if prec == "fp32" and d == 3 and N in (128, 256) and not wl["grad"]:
        for form in TC_PRECISIONS:
            extras[form] = form_line(form, 20)
    fp32_form = form_line("fp32", 20) if prec in TC_PRECISIONS else None

    line = None
    if rank == 0:
        line = {
            "metric": "grid pts/s per potential (N^d/s), % HBM roofline, vs plain FP64 at stated rel err",
            "value": value, "unit": "grid pts/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64"}.get(prec, "f32 + " + prec[3:] + " tensor-core fused pass"),
            "data": "synthetic",
            "config": {"workload": args.workload, "d": d, "N": N, "kernel": wl["kernel"], "k": wl["k"],
                       "L": wl["L"], "fields": F, "grad_mode": "exact" if wl["grad"] else None,
                       "precision": prec,
                       "l2": "flushed before every timed step (256 MB write)", "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
                         "algorithmic_bytes_per_launch": pb[dom], "avg_launch_ms": dom_avg_s * 1000.0},
            "step_roofline": {"algorithmic_bytes_per_step": sum(pb[k] for k in passes if passes[k][0] > 0),
                              "achieved": sum(pb[k] for k in passes if passes[k][0] > 0) / (ms_per_step / 1000.0) / 1e9,
                              "peak": peak, "unit": "GB/s",
                              "frac": sum(pb[k] for k in passes if passes[k][0] > 0) / (ms_per_step / 1000.0) / 1e9 / peak},
            "passes": {k: {"launches": v[0], "avg_ms": (v[1] / v[0] if v[0] else None),
                           "frac_of_hbm": (pb[k] / (v[1] / v[0] / 1000.0) / 1e9 / peak) if v[0] else None}
                       for k, v in passes.items()},
            "clocks": clk,
            "e2e": {"value": (N ** d) * world / e2e_s, "unit": "grid pts/s", "h2d_bytes_per_step": U_b,
                    "d2h_bytes_per_step": U_b * F, "steps": e2e_pipe_steps,
                    "api": "vp_apply_pipeline: pinned host buffers, copy-engine transfers overlapping the "
                           "transforms of neighbouring densities",
                    "output_matches_device_apply": pipe_ok,
                    "sequential_value": (N ** d) / e2e_seq_s,
                    "sequential_api": "vp_apply per step, pinned buffers read and written in place",
                    "staged_value": (N ** d) / e2e_staged_s},
            "gpu_launches": launches_per_step * args.steps,
            "precompute_s": precompute_s,
            "autotune": autotune,
            "fp64_form": fp64,
            "cufft_form": cufft,
        }
        if extras:
            line["tensor_core_forms"] = extras
        if errs is not None:
            line["rel_l2_vs_oracle"] = errs
            line["oracle_reference"] = ref["what"]
        if fp32_form is not None:
            line["fp32_form"] = fp32_form
            fused_launches, fused_ms = passes.get("fused_axis0", (0, 0.0))
            if fused_launches:
                t_s = fused_ms / fused_launches / 1000.0
                fl = tc_flops_per_launch(N, prec)
                tpk, tkind = measured_peak_bf16(sustained=False)
                line["tensor"] = {"kernel": "fused_axis0 (tcgen05)", "flops_per_launch": fl,
                                  "achieved_tflops": fl / t_s / 1e12, "peak_tflops": tpk, "peak_source": tkind,
                                  "frac": fl / t_s / 1e12 / tpk}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(wl, args.workload)
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """64 densities (N in {48,64,96,128}, half Laplace, half Helmholtz) per step,
    in one persistent launch replayed from a CUDA graph; the same work through
    per-density launches is timed beside it."""
    import torch

    from paper_1604_03155_gb300 import inputs as I
    from paper_1604_03155_gb300 import vp

    dev = torch.device("cuda", 0)
    grids = args.workload == "batch64_grids"
    if grids:  # per-axis sizes: (Ns, kernel, k, density) per density
        recipe = [(Ns, kern, k, h) for Ns, kern, k, h in I.batch_recipe_grids()]
    else:
        recipe = [((w.N,) * 3, w.kernel, w.k, w.density()) for w in I.batch_recipe()]
    t0 = time.perf_counter()
    plans = [vp.Plan(3, Ns if grids else Ns[0], kern, k, 1.8, precision="fp32") for Ns, kern, k, _ in recipe]
    precompute_s = time.perf_counter() - t0
    hs = [h.astype(np.complex64) for _, _, _, h in recipe]
    fs = [torch.from_numpy(h).to(dev) for h in hs]
    outs = [torch.empty_like(f) for f in fs]
    stream = torch.cuda.Stream(device=dev)
    b = vp.Batch(plans, stream=stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    pts = sum(int(np.prod(Ns)) for Ns, _, _, _ in recipe)
    U_bytes = 8 * pts
    oct_bytes = sum(8 * int(np.prod([n + 1 for n in Ns])) for Ns, _, _, _ in recipe)
    algo = 27 * U_bytes + oct_bytes - 0  # 3+6+(4+4)+6+3 U and one multiplier octant per density

    def timed(strategy, steps, chunk=0):
        b.set_strategy(strategy)
        b.set_chunk(chunk)
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                b.apply(fs, outs)
        torch.cuda.synchronize(dev)
        st = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        with torch.cuda.stream(stream):
            for i in range(steps):
                flush.fill_(float(i))
                st[i].record(stream)
                b.apply(fs, outs)
                en[i].record(stream)
        torch.cuda.synchronize(dev)
        b.status()
        return sum(a.elapsed_time(c) for a, c in zip(st, en)) / steps

    # the autotuner's choice (strategy and chunk), made on the first apply
    b.set_strategy(vp.VP_BATCH_AUTO)
    b.set_chunk(0)
    with torch.cuda.stream(stream):
        b.apply(fs, outs)
    torch.cuda.synchronize(dev)
    auto_strategy, auto_chunk = b.strategy(), b.chunk()
    # the persistent launch at every chunk size the autotuner tries; the
    # headline is the fastest
    chunks = {c: timed(vp.VP_BATCH_PERSISTENT, max(3, args.steps // 4), c) for c in (4, 8, 16, 32)}
    best_chunk = min(chunks, key=chunks.get)
    clocks = ClockSampler(0)
    clocks.start()
    ms = timed(vp.VP_BATCH_PERSISTENT, args.steps, best_chunk)
    clk = clocks.stop()
    ms_seq = timed(vp.VP_BATCH_PER_DENSITY, max(3, args.steps // 4))
    ms_one = timed(vp.VP_BATCH_PERSISTENT_ONE_PER_SM, max(3, args.steps // 4))
    ms_gs = timed(vp.VP_BATCH_GRAPH_STREAMS, max(3, args.steps // 4))
    peak, peak_kind = measured_peak_hbm()
    achieved = algo / (ms / 1000.0) / 1e9
    line = {
        "metric": "grid pts/s per potential (N^d/s), % HBM roofline, vs plain FP64 at stated rel err",
        "value": pts / (ms / 1000.0), "unit": "grid pts/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "densities": len(recipe),
                   "sizes": sorted({n for Ns, _, _, _ in recipe for n in Ns}), "per_axis_sizes": grids,
                   "sum_points": pts, "l2": "flushed before every timed step (256 MB write)"},
        "persistent_chunk": best_chunk, "persistent_ms_by_chunk": chunks,
        "autotuner_choice": {"strategy": {1: "persistent", 2: "persistent_one_cta_per_sm", 3: "per_density",
                                          4: "graph_of_streams"}.get(auto_strategy, auto_strategy),
                             "chunk": auto_chunk},
        "roofline": {"bound": "hbm", "kernel": "batch_kernel", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind, "traffic": None,
                     "algorithmic_bytes_per_launch": algo, "avg_launch_ms": ms},
        "per_density_launches": {"value": pts / (ms_seq / 1000.0), "ms_per_step": ms_seq},
        "persistent_one_cta_per_sm": {"value": pts / (ms_one / 1000.0), "ms_per_step": ms_one},
        "graph_of_streams": {"value": pts / (ms_gs / 1000.0), "ms_per_step": ms_gs},
        "speedup_vs_per_density": ms_seq / ms,
        "clocks": clk, "gpu_launches": args.steps, "precompute_s": precompute_s,
    }
    print(json.dumps(line), flush=True)
    b.close()


# ---------------------------------------------------------------------------
# Experiments beside the headline line (python bench.py experiment NAME ...):
#   grids    -- the FP32 apply on cubic and per-axis grids (vp_plan_create_aniso),
#               16 Gaussian sources, CUDA events on the plan's stream, 256 MB L2
#               flush before every timed apply; ms per apply, grid points per
#               second and per-pass times, one JSON line per grid
#   nystrom  -- the Nystrom entry kernels (Section 4, the remark after the
#               discrete convolution): dense blocks T(p_i - p'_j) for random
#               (or sub-box) target and source nodes, and batches of kernel
#               entries at random offsets; entries per second and output
#               bandwidth, one JSON line
#   unet     -- the learned preconditioner network (tensor-core convolutions):
#               forward and loss + gradients at S^3, ms per call, one JSON line
# ---------------------------------------------------------------------------
def exp_grids(argv):
    import torch

    from paper_1604_03155_gb300 import inputs as I
    from paper_1604_03155_gb300 import vp
    ap = argparse.ArgumentParser(prog="bench.py experiment grids")
    ap.add_argument("--grids", default="128x128x128,128x128x64,64x96x128,96x128x128")
    ap.add_argument("--kernel", default="helmholtz")
    ap.add_argument("--k", type=float, default=30.0)
    ap.add_argument("--reps", type=int, default=50)
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    for g in a.grids.split(","):
        Ns = [int(v) for v in g.split("x")]
        d = len(Ns)
        plan = vp.Plan(d, tuple(Ns), a.kernel, a.k if a.kernel == "helmholtz" else 0.0, 0.0, precision="fp32")
        stream = torch.cuda.Stream(device=dev)
        plan.set_stream(stream)
        src = I.random_gaussians(I.BASE_SEED + 11, 16, d)
        X = np.meshgrid(*[I.grid_coords(N) for N in Ns], indexing="ij")
        f = np.zeros(Ns, dtype=np.complex128)
        for c, sg, am in zip(src.centres, src.sigmas, src.amps):
            f += am * np.exp(-sum((X[j] - c[j]) ** 2 for j in range(d)) / sg ** 2)
        ft = torch.from_numpy(f.astype(np.complex64)).to(dev)
        phi = torch.empty_like(ft)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
        with torch.cuda.stream(stream):
            for _ in range(3):
                plan.apply(ft, phi)
            plan.set_timing(True)
            s_ = [torch.cuda.Event(enable_timing=True) for _ in range(a.reps)]
            e_ = [torch.cuda.Event(enable_timing=True) for _ in range(a.reps)]
            for i in range(a.reps):
                flush.fill_(float(i))
                s_[i].record(stream)
                plan.apply(ft, phi)
                e_[i].record(stream)
        torch.cuda.synchronize(dev)
        plan.set_timing(False)
        passes = {k: v[1] / v[0] for k, v in plan.get_timing().items() if v[0]}
        ms = sum(x.elapsed_time(y) for x, y in zip(s_, e_)) / a.reps
        plan.close()
        pts = int(np.prod(Ns))
        print(json.dumps(dict(grid=g, points=pts, ms=ms, pts_per_s=pts / (ms * 1e-3), passes_ms=passes)), flush=True)


def exp_nystrom(argv):
    import torch

    from paper_1604_03155_gb300 import vp
    ap = argparse.ArgumentParser(prog="bench.py experiment nystrom")
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
    print(json.dumps({"d": a.d, "N": a.N, "kernel": a.kernel, "dtype": a.dtype, "boxes": a.boxes, **out}), flush=True)
    plan.close()


def exp_unet(argv):
    """The learned preconditioner network at S^3: forward and loss + gradients
    (forward, backward, weight gradients) through the C-ABI, with the seeded
    initial weights rounded to BF16 and a seeded input."""
    import torch

    from paper_1604_03155_gb300 import inputs as I
    from paper_1604_03155_gb300.vp import UNet
    ap = argparse.ArgumentParser(prog="bench.py experiment unet")
    ap.add_argument("--S", type=int, default=128)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    layers = [(I.bf16_round(w), I.bf16_round(b)) for w, b in I.unet_init_weights(3, 16)]
    net = UNet(a.S, 16, weights=layers)
    n = a.S ** 3
    x = torch.from_numpy(I.normal(77, 3 * n).astype(np.float32).reshape(3, a.S, a.S, a.S)).to(dev)
    tgt = torch.from_numpy(I.normal(78, 2 * n).astype(np.float32).reshape(2, a.S, a.S, a.S)).to(dev)
    out = net.forward(x)
    out_ms = {}
    for name, fn in [("forward", lambda: net.forward(x, out)), ("loss_grad", lambda: net.loss_grad(x, tgt))]:
        for _ in range(a.warmup):
            fn()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(a.reps):
            fn()
        e.record()
        torch.cuda.synchronize()
        out_ms[name + "_ms"] = s.elapsed_time(e) / max(a.reps, 1)
    net.status()
    print(json.dumps({"S": a.S, "channels": 16, **out_ms, "output_finite": bool(torch.isfinite(out).all())}), flush=True)
    net.close()


EXPERIMENTS = {"grids": exp_grids, "nystrom": exp_nystrom, "unet": exp_unet}


def main():
    if len(sys.argv) > 2 and sys.argv[1] == "experiment":
        if sys.argv[2] not in EXPERIMENTS:
            raise SystemExit(f"unknown experiment {sys.argv[2]!r}; one of {sorted(EXPERIMENTS)}")
        return EXPERIMENTS[sys.argv[2]](sys.argv[3:])
    args = parse()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    elif args.workload in ("batch64", "batch64_grids"):
        run_batch(args)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
