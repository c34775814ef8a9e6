#!/usr/bin/env python3
"""Benchmark of compressed-basis GMRES on GB300.

Workload: 3D convection-diffusion on a 128^3 grid (n = 2,097,152, 14,581,760 nnz,
7-point upwind stencil, Pe = 10), b = A x* with seeded x* ~ U[-1,1], x0 = 0,
restart m = 100, CGS with one re-orthogonalisation pass, tol 1e-10 relative true
residual.  One step = one time-to-solution for every basis format of the workload
(f64, f32, f16, i32, i16), inputs resident in HBM.

Metric: time-to-1e-10 residual speedup of CB-GMRES (f32 basis, the paper's
recommended format) over FP64-basis GMRES run by the same library on the same GPU;
alongside it the achieved HBM bandwidth of the basis-GEMV kernels (roofline).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  Under torchrun (N > 1) every rank solves its own
replica of the system (the single-system solve has no data-parallel split without a
halo exchange); times are the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-10 residual speedup vs FP64-basis GMRES; basis-GEMV HBM GB/s"
WORKLOAD = "convdiff3d_128^3_pe10_upwind_restart100_tol1e-10"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--grid", type=int, default=128)
    p.add_argument("--formats", default="f64,f32,f16,i32,i16")
    p.add_argument("--headline", default="f32")
    p.add_argument("--arith", default="df32")
    p.add_argument("--adapt", action="store_true",
                   help="adaptive basis format: promote a format up its ladder when a cycle loses accuracy")
    p.add_argument("--precond", default="none", choices=["none", "jacobi", "bj4"],
                   help="right preconditioner of the conv-diff workload (bj4: block-Jacobi, 4-row blocks)")
    p.add_argument("--tol", type=float, default=1e-10)
    p.add_argument("--maxit", type=int, default=40000)
    p.add_argument("--restart", type=int, default=100)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-fp64", action="store_true", help="skip the native-FP64-arithmetic comparison solves")
    p.add_argument("--cpu-steps", type=int, default=25,
                   help="Arnoldi steps of the 1-thread oracle sample (the first steps of a cycle: biased low)")
    p.add_argument("--ortho", choices=["cgs", "mgs"], default="cgs",
                   help="orthogonalisation of the single-system solver (Fig. 1's CGS, or MGS)")
    p.add_argument("--batch-nsys", type=int, default=512,
                   help="systems of the batch workload (512 is the benchmark; fewer for profiling)")
    p.add_argument("--schedule", type=int, nargs=2, metavar=("CLUSTER", "SPLIT_ROWS"),
                   help="batch workload: this schedule instead of autotuning (for profiling)")
    p.add_argument("--spmv-group", type=int, default=0,
                   help="headline workload: SpMV schedule (0: timed at create; k > 0: k lanes per CSR row; "
                        "-1: the sliced-ELL copy) -- for profiling, where timing under a profiler misleads")
    p.add_argument("--workload", choices=["convdiff128", "batch512", "random27", "learned96", "restart_sweep",
                                          "multirhs", "poisson64"],
                   default="convdiff128")
    return p.parse_args()


# ------------------------------------------------------------------------ clocks
def smi_gpu_id(local: int) -> str:
    """The nvidia-smi id of this process's cuda:<local>: its UUID (nvidia-smi indices
    count physical GPUs and ignore CUDA_VISIBLE_DEVICES), else the visible-devices entry."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(local).uuid)
        if u and u != "None":
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = [e.strip() for e in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if e.strip()]
    return vis[local] if local < len(vis) else str(local)


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region (read only)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local: int):
        self.idx = smi_gpu_id(local)
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)
        return self

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
        if self.thread:
            self.thread.join(timeout=2)
        return dict(parse_clock_lines(self.lines), gpu=self.idx)


def parse_clock_lines(lines) -> dict:
    """Clock record from `nvidia-smi --query-gpu=<ClockSampler.Q> --format=csv,noheader,nounits`
    lines: median SM clock, maximum SM clock and power, and every throttle reason seen
    Active in any sample.  Lines that do not parse (a header, [N/A] fields) are skipped."""
    sm, smax, power, reasons = [], [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1])); smax.append(float(f[2]))
            power.append(float(f[3]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "power_w_max": max(power) if power else None,
            "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------ helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measured_tensor_peak():
    """Dense BF16 tensor peak: the sustained cuBLAS figure (a kernel timed inside a long
    loop) from MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return "bf16", "measured bf16_tflops_sustained (MEASURED_PEAKS.json)", float(d["bf16_tflops_sustained"])
    except (OSError, KeyError, ValueError):
        return "bf16", "fallback 1700 TFLOP/s sustained", 1700.0


def shard_units(nunits: int, world: int, rank: int) -> range:
    """Contiguous share of rank `rank` out of `world` of nunits independent units (the
    systems of a batch): sizes differ by at most one, the shares cover every unit once."""
    base, extra = divmod(nunits, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def max_over_ranks(vals: dict, device) -> dict:
    """Element-wise maximum of per-rank timings over all ranks of the process group (the
    slowest replica decides a whole-job time).  Keys must be the same on every rank."""
    import torch
    import torch.distributed as dist
    keys = sorted(vals)
    t = torch.tensor([float(vals[k]) for k in keys], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return {k: float(t[i]) for i, k in enumerate(keys)}


def ncu_traffic_per_element(fmt: str):
    """DRAM bytes per basis element of the basis-GEMV kernels from the committed ncu
    summary (profiles/basis_gemv_convdiff96.md, line `traffic_bytes_per_element <cls> <fmt> <x>`)."""
    path = os.path.join(ROOT, "profiles", "basis_gemv_convdiff96.md")
    out = {}
    try:
        with open(path) as f:
            for ln in f:
                t = ln.strip().strip("`").split()
                if len(t) == 4 and t[0] == "traffic_bytes_per_element" and t[2] == fmt:
                    out[t[1]] = float(t[3])
    except OSError:
        pass
    return out


def build_problem(grid: int):
    import workloads as W
    A = W.convdiff3d(grid)
    xs = W.exact_solution(A.n, 2)
    b = W.rhs_from_solution(A, xs)
    return A, xs, b


def oracle_sample(A, b, fmt: str, steps: int, restart: int, threads: int):
    """Time the oracle (as it stands) on the first `steps` Arnoldi steps of the solve."""
    import oracle as O
    O.set_threads(threads)
    t0 = time.perf_counter()
    r = O.gmres(A, b, m=restart, fmt=O.FORMATS[fmt], tol=0.0, maxit=steps)
    return time.perf_counter() - t0, r["iters"]


# ------------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    A, xs, b = build_problem(args.grid)
    steps = max(2, min(args.cpu_steps, 12))
    threads = os.cpu_count() or 1
    times = {"f64": [], args.headline: []}
    for it in range(args.warmup + args.steps):
        for fmt in times:
            t, _ = oracle_sample(A, b, fmt, steps, args.restart, threads)
            if it >= args.warmup:
                times[fmt].append(t)
    t64 = sum(times["f64"]); th = sum(times[args.headline])
    v = t64 / th
    sample = (f"first {steps} Arnoldi steps of the {WORKLOAD} solve with the f64 and {args.headline} "
              f"basis, oracle (plain C, {threads} host threads), per step")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "x", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "ms_per_step": 1000 * (t64 + th) / args.steps,
            "config": {"workload": WORKLOAD, "n": A.n, "nnz": A.nnz, "restart": args.restart,
                       "headline_format": args.headline, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "x", "cores": threads, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": v, "unit": "x", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------ CPU baseline helpers
def host_cpu() -> dict:
    """Host threads and CPU model of the machine this process runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count() or 1, "model": model}


def oracle_timed(threads: int, fn):
    """Run fn() with the oracle on `threads` host threads; (seconds, result)."""
    import oracle as O
    O.set_threads(threads)
    t0 = time.perf_counter()
    r = fn()
    dt = time.perf_counter() - t0
    O.set_threads(os.cpu_count() or 1)
    return dt, r


def oracle_step_seconds(A, b, fmt: str, restart: int, threads: int, steps: int | None = None, **kw):
    """Seconds per Arnoldi step of the oracle (as it stands) over its first `steps` steps
    (default: one full restart cycle, j = 1..restart)."""
    import oracle as O
    steps = steps or restart
    dt, r = oracle_timed(threads, lambda: O.gmres(A, b, m=restart, fmt=O.FORMATS[fmt], tol=0.0, maxit=steps, **kw))
    return dt / max(1, r["iters"])


def cpu_line(value_tts_all: float, tts_one: float | None, gpu_s: float, sample: str, host: dict,
             extrapolated: bool, **extra) -> dict:
    """cpu_baseline object: value = oracle time-to-solution / GPU time-to-solution of the
    line's headline configuration, on all host threads (1-thread figure beside it)."""
    d = {"value": round(value_tts_all / gpu_s, 2),
         "unit": "x (oracle time-to-solution / GPU time-to-solution)",
         "cores": host["nproc"], "kind": "oracle", "sample": sample, "extrapolated": extrapolated,
         "host": host, "oracle_s_all_threads": round(value_tts_all, 4), "gpu_s": round(gpu_s, 5)}
    if tts_one is not None:
        d["oracle_s_1_thread"] = round(tts_one, 4)
        d["value_1_thread"] = round(tts_one / gpu_s, 2)
    d.update(extra)
    return d


def roofline_from_profile(prof: dict, fmt: str, kernel_names: dict, peak: float, peak_kind: str) -> dict:
    """Roofline of the basis-GEMV kernel class (dot or axpy) with the larger share of a
    profiled solve: algorithmic bytes per launch / average CUDA-event launch time."""
    cls = max(("basis_dot", "basis_axpy"), key=lambda c: prof[c]["ms"])
    nl = max(1, prof[cls]["launches"])
    avg_ms = prof[cls]["ms"] / nl
    avg_bytes = prof[cls]["bytes"] / nl
    ach = avg_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0.0
    return {"bound": "hbm", "kernel": f"{kernel_names[cls]} ({fmt})", "achieved": round(ach, 1), "peak": peak,
            "unit": "GB/s", "frac": round(ach / peak, 4), "traffic": None,
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
            "algorithmic_bytes_per_launch": avg_bytes, "avg_launch_ms": avg_ms}


def kernel_class_table(prof: dict) -> dict:
    """Per kernel class of a profiled solve: share of the summed CUDA-event time, launches,
    average microseconds per launch and algorithmic GB/s (the library's byte model)."""
    total = sum(p["ms"] for p in prof.values())
    out = {}
    for c, p in prof.items():
        if p["launches"] <= 0:
            continue
        out[c] = {"share": round(p["ms"] / total, 4) if total > 0 else None,
                  "launches": int(p["launches"]),
                  "us_per_launch": round(1e3 * p["ms"] / p["launches"], 2),
                  "gbs": round(p["bytes"] / (p["ms"] * 1e-3) / 1e9, 1) if p["ms"] > 0 and p["bytes"] > 0 else None}
    return out


def e2e_host_ratio(solvers: dict, base: str, head: str, b: np.ndarray, n: int, tol: float, maxit: int, reps: int,
                   flush=None):
    """Same metric end to end through cbgmres_solve_host (pinned host b and x, the copies
    inside the timed region): time(base) / time(head).  `flush` (if given) runs before each
    timed solve, outside the timed interval."""
    import torch
    bh = torch.from_numpy(b).pin_memory().numpy()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
    te = {}
    for f in (base, head):
        ts = []
        for _ in range(max(1, reps)):
            xh[:] = 0.0
            if flush is not None:
                flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            solvers[f].solve_host(bh, xh, tol=tol, maxit=maxit)
            ts.append(time.perf_counter() - t0)
        te[f] = sum(ts) / len(ts)
    return {"value": te[base] / te[head], "unit": "x", "h2d_bytes_per_step": 2 * 2 * 8 * n,
            "d2h_bytes_per_step": 2 * 8 * n, "seconds": {k: round(v, 4) for k, v in te.items()}}


# ------------------------------------------------------------------------ batch workload
BATCH_WORKLOAD = "batch512_stencil2d3d_lognormal0.5_restart30_tol1e-8_jacobi"


def batch_model_bytes(mats, iters, restarts, m, bs):
    """SpMV + 4 basis passes per Arnoldi step, summed over every system's cycles."""
    tot = 0.0
    for A, it, rs in zip(mats, iters, restarts):
        it, rs = int(it), int(rs)
        spmv = 12.0 * A.nnz + 4.0 * (A.n + 1) + 16.0 * A.n
        last = it - m * max(0, rs - 1)
        cols = (rs - 1) * m * (m + 1) / 2 + last * (last + 1) / 2 if rs > 0 else 0.0
        tot += it * spmv + 4.0 * A.n * bs * cols
    return tot


def run_batch(args):
    import tempfile

    import torch
    import oracle as O
    import paper_2009_12101_gb300 as cb
    import workloads as W
    cb.ensure_built()
    mats = W.stencil_batch(nsys=args.batch_nsys)
    # under torchrun every rank solves its contiguous share of the systems (no collective
    # on the data path; the batch time is the slowest rank's)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
        mine = shard_units(len(mats), world, rank)
        sel = list(mine)
        mats = [mats[i] for i in sel]
    else:
        sel = list(range(len(mats)))
    xs = [W.exact_solution(A.n, 4, salt=i) for i, A in zip(sel, mats)]
    bs_list = [W.rhs_from_solution(A, x) for A, x in zip(mats, xs)]
    b = np.concatenate(bs_list)
    fmts = ["f64", "f32", "f16"]
    tol, m = 1e-8, 30
    stream = torch.cuda.current_stream()
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    solvers, sched = {}, {}
    cache = os.path.join(tempfile.gettempdir(), "cbgmres_batch_tune.jsonl")
    for f in fmts:
        solvers[f] = cb.BatchedSolver(mats, restart=m, fmt=f, precond="jacobi", use_graph=True)
        x.zero_()
        if args.schedule:
            solvers[f].schedule(*args.schedule)
            sched[f] = tuple(args.schedule)
        else:
            sched[f] = solvers[f].tune(bd, x, tol=tol, cache_path=cache)
        sched[f] = tuple(sched[f]) + (solvers[f].spmv_lanes(),)
    for _ in range(args.warmup):
        for f in fmts:
            x.zero_(); solvers[f].solve(bd, x, tol=tol)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))).start()
    torch.cuda.synchronize()
    times = {f: [] for f in fmts}
    outs = {}
    launches = 0
    for _ in range(args.steps):
        for f in fmts:
            x.zero_()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs[f] = solvers[f].solve(bd, x, tol=tol)
            e1.record(stream)
            torch.cuda.synchronize()
            times[f].append(e0.elapsed_time(e1))
            launches += outs[f]["kernel_launches"]
    clk = clocks.stop()
    t = {f: sum(v) / len(v) for f, v in times.items()}
    if world > 1:
        t = max_over_ranks(t, "cuda")
    peak, peak_kind = measured_peaks()
    o = outs["f32"]
    mb = batch_model_bytes(mats, o["iters"], o["restarts"], m, 4)
    achieved = mb / (t["f32"] * 1e-3) / 1e9
    # the same systems one by one through the single-system solver (f32, Jacobi)
    seq_ms = None
    if not args.no_cpu and world == 1:
        tot = 0.0
        for A, bb in zip(mats, bs_list):
            with cb.Solver.from_csr(A, restart=m, fmt="f32", precond="jacobi") as s1:
                bt = torch.from_numpy(bb).cuda(); xt = torch.zeros(A.n, dtype=torch.float64, device="cuda")
                s1.solve(bt, xt, tol=tol)   # warm
                xt.zero_()
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream); s1.solve(bt, xt, tol=tol); e1.record(stream); torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
        seq_ms = tot
    # end to end: pinned host b -> device, solve, x -> host
    bh = torch.from_numpy(b).pin_memory(); xh = torch.zeros(b.size, dtype=torch.float64).pin_memory()
    te = {}
    for f in ("f64", "f32"):
        ts = []
        for _ in range(max(1, args.steps)):
            xh.zero_()
            torch.cuda.synchronize(); t0 = time.perf_counter()
            bdev = bh.cuda(non_blocking=True); xdev = xh.cuda(non_blocking=True)
            solvers[f].solve(bdev, xdev, tol=tol)
            xh.copy_(xdev); torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        te[f] = sum(ts) / len(ts)
    if world > 1:
        te = max_over_ranks(te, "cuda")
    # CPU baseline: the oracle's full solves (f32 basis, Jacobi) of every 32nd system on all
    # host threads and on one, extrapolated to the batch by rows x GPU iterations
    cpu = None
    if not args.no_cpu and world == 1:
        hc = host_cpu()
        pick = list(range(0, len(mats), 32))
        work = lambda idx: sum(mats[i].n * max(1, int(o["iters"][i])) for i in idx)
        t_all = t_one = 0.0
        for i in pick:
            A, bb = mats[i], bs_list[i]
            solve = lambda: O.gmres(A, bb, m=m, fmt=O.F32, precond=O.PC_JACOBI, tol=tol, maxit=100000)
            dt, _ = oracle_timed(hc["nproc"], solve); t_all += dt
            dt, _ = oracle_timed(1, solve); t_one += dt
        scale = work(range(len(mats))) / work(pick)
        cpu = cpu_line(t_all * scale, t_one * scale, t["f32"] / 1000,
                       f"oracle full solves (f32 basis, Jacobi, restart 30, tol 1e-8) of {len(pick)} of the "
                       f"{len(mats)} systems (every 32nd), extrapolated to the batch by rows x GPU iterations",
                       hc, True)
    line = {
        "metric": METRIC, "value": round(t["f64"] / t["f32"], 4), "unit": "x", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sum(t.values()), 3),
        "higher_is_better": True, "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "df32", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD.replace("batch512", f"batch{len(mats)}"), "nsys": len(mats),
                   "total_rows": int(b.size), "restart": m,
                   "tol": tol, "formats": fmts, "schedule_cluster_split_lanes": {f: list(v) for f, v in sched.items()},
                   "value_is": "time(f64 basis) / time(f32 basis), whole batch in one persistent launch",
                   "l2": "no flush: basis of the batch (0.5-2 GB) exceeds the 129 MB L2"},
        "time_to_solution_s": {f: round(v / 1000, 4) for f, v in t.items()},
        "speedup_vs_f64": {f: round(t["f64"] / v, 4) for f, v in t.items()},
        "iterations_total": {f: int(outs[f]["iters"].sum()) for f in fmts},
        "iterations_max": {f: int(outs[f]["iters"].max()) for f in fmts},
        "status": {f: int(outs[f]["status"]) for f in fmts},
        "max_relres": {f: float(outs[f]["relres"].max()) for f in fmts},
        "sequential_single_solver_f32_s": round(seq_ms / 1000, 4) if seq_ms else None,
        "batching_speedup_f32": round(seq_ms / t["f32"], 2) if seq_ms else None,
        "roofline": {"bound": "hbm", "kernel": "k_batched (f32)", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
                     "algorithmic_bytes": mb, "note": "model bytes (SpMV + 4 basis passes per step) / batch time"},
        "cpu_baseline": cpu,
        "e2e": {"value": te["f64"] / te["f32"], "unit": "x", "h2d_bytes_per_step": 2 * 2 * 8 * int(b.size),
                "d2h_bytes_per_step": 2 * 8 * int(b.size), "seconds": {k: round(v, 4) for k, v in te.items()}},
        "gpu_launches": launches, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    for s_ in solvers.values():
        s_.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------ precision pattern
R27_WORKLOAD = "random27_n1048576_band9+18_tol1e-10"


def l2_flusher(nbytes: int = 256 << 20):
    """A callable that writes `nbytes` (default 256 MiB, twice the 129 MB L2) of device
    memory on the current stream, evicting whatever a previous timed step left in L2."""
    import torch
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")

    def flush():
        buf.zero_()
    return flush


def timed_solve(solver, b, x, tol, maxit, stream, flush=None):
    """One solve from x = 0 timed by CUDA events on `stream`; `flush` (if given) runs
    before the first event, outside the timed interval."""
    import torch
    x.zero_()
    if flush is not None:
        flush()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = solver.solve(b, x, tol=tol, maxit=maxit)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), st


def run_random27(args):
    """bf16 / e4m3 basis with per-vector power-of-two scale vs f64 basis on the random
    nonsymmetric n = 2^20 matrices; timed: delta 0.1, m 100; sweep: delta x m, once.  Each
    format's solution is compared with the oracle's solution of the timed configuration."""
    import torch
    import oracle as O
    import paper_2009_12101_gb300 as cb
    import workloads as W
    cb.ensure_built()
    stream = torch.cuda.current_stream()
    fmts = ["f64", "f32", "bf16", "e4m3"]
    tol = 1e-10
    results, sweep, xg = {}, [], {}
    launches = 0
    peak, kind = measured_peaks()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))).start()
    for delta in (0.01, 0.1, 0.5):
        A = W.random27(1 << 20, delta)
        xs = W.exact_solution(A.n, 3)
        bnp = W.rhs_from_solution(A, xs)
        b = torch.from_numpy(bnp).cuda()
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        for m in (50, 100, 200):
            timed_cfg = delta == 0.1 and m == 100
            for f in fmts:
                s = cb.Solver.from_csr(A, restart=m, fmt=f, profile=True)
                reps = args.steps if timed_cfg else 1
                for _ in range(args.warmup):      # every configuration, so each row's time is warm
                    timed_solve(s, b, x, tol, args.maxit, stream)
                s.profile(reset=True)
                ts = []
                for _ in range(reps):
                    t, st = timed_solve(s, b, x, tol, args.maxit, stream)
                    ts.append(t)
                    if timed_cfg:
                        launches += st["kernel_launches"]
                prof = s.profile()
                xh = x.cpu().numpy()
                res = float(np.linalg.norm(bnp - O.spmv(A, xh)) / np.linalg.norm(bnp))
                err = float(np.linalg.norm(xh - xs) / np.linalg.norm(xs))
                row = {"delta": delta, "m": m, "fmt": f, "ms": sum(ts) / len(ts), "iters": st["iters"],
                       "status": st["status"], "true_relres": res, "x_err_vs_exact": err,
                       "dot_gbs": (prof["basis_dot"]["bytes"] / prof["basis_dot"]["ms"] / 1e6
                                   if prof["basis_dot"]["ms"] else None)}
                sweep.append(row)
                if timed_cfg:
                    results[f] = row
                    results[f]["roofline"] = roofline_from_profile(
                        prof, f, {"basis_dot": "k_basis_dot_tma", "basis_axpy": "k_basis_axpy"}, peak, kind)
                    xg[f] = xh.copy()
                    if f in ("f64", "bf16"):
                        results[f]["solver"] = s
                        continue
                s.close()
        if delta == 0.1:
            A01, b01 = A, bnp
    clk = clocks.stop()
    t = {f: results[f]["ms"] for f in fmts}
    # each format's error against the oracle's FP64 solution, stated per format, and the
    # oracle's time-to-solution as the CPU baseline
    hc = host_cpu()
    per_fmt = {}
    t_oracle = {}
    for f in fmts:
        dt, ro = oracle_timed(hc["nproc"], lambda: O.gmres(A01, b01, m=100, fmt=O.FORMATS[f], tol=tol,
                                                            maxit=args.maxit))
        t_oracle[f] = dt
        per_fmt[f] = {"oracle_iters": int(ro["iters"]), "gpu_iters": int(results[f]["iters"]),
                      "x_relerr_vs_oracle": float(np.linalg.norm(xg[f] - ro["x"]) / np.linalg.norm(ro["x"])),
                      "x_relerr_vs_f64_oracle": None, "oracle_true_relres": float(ro["true_relres"])}
        if f == "f64":
            x64o = ro["x"]
    for f in fmts:
        per_fmt[f]["x_relerr_vs_f64_oracle"] = float(np.linalg.norm(xg[f] - x64o) / np.linalg.norm(x64o))
    cpu = None
    if not args.no_cpu:
        s1 = oracle_step_seconds(A01, b01, "bf16", 100, 1, steps=20)
        cpu = cpu_line(t_oracle["bf16"], s1 * results["bf16"]["iters"], t["bf16"] / 1000,
                       f"oracle full solve of the timed configuration (delta 0.1, m 100, bf16 basis) on all host "
                       f"threads; 1 thread: the first 20 steps, extrapolated by the solve's steps", hc, False,
                       oracle_s_all_threads_by_format={f: round(v, 4) for f, v in t_oracle.items()})
    e2e = e2e_host_ratio({f: results[f]["solver"] for f in ("f64", "bf16")}, "f64", "bf16", b01, A01.n, tol,
                         args.maxit, args.steps)
    for f in ("f64", "bf16"):
        results[f].pop("solver").close()
    line = {"metric": METRIC, "value": round(t["f64"] / t["bf16"], 4), "unit": "x", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sum(t.values()), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "df32", "data": "synthetic",
            "config": {"workload": R27_WORKLOAD, "timed": "delta 0.1, m 100", "headline_format": "bf16",
                       "value_is": "time(f64 basis) / time(bf16 basis)",
                       "formats": fmts, "l2": "no flush: basis >= 0.2 GB exceeds L2"},
            "time_to_solution_s": {f: round(v / 1000, 4) for f, v in t.items()},
            "speedup_vs_f64": {f: round(t["f64"] / v, 4) for f, v in t.items()},
            "error_vs_oracle": per_fmt,
            "roofline": results["bf16"]["roofline"],
            "roofline_by_format": {f: results[f]["roofline"] for f in fmts},
            "sweep": [{k: v for k, v in r.items() if k != "roofline"} for r in sweep],
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------ learned preconditioner
L96_WORKLOAD = "diffusion3d_cc96_lognormal1_learnedSPAI_f32_restart100_tol1e-10"


def run_learned96(args):
    """Per-row MLP SPAI trained on 2000 (r, e) pairs from FP64 GMRES, vs Jacobi and none."""
    import torch
    import oracle as O
    import paper_2009_12101_gb300 as cb
    import workloads as W
    cb.ensure_built()
    stream = torch.cuda.current_stream()
    N = 96
    A = W.diffusion3d_cc(N)[0]
    xs = W.exact_solution(A.n, 5)
    bnp = W.rhs_from_solution(A, xs)
    b = torch.from_numpy(bnp).cuda()
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    gen = torch.Generator(device="cuda"); gen.manual_seed(20201206)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))).start()
    spai = cb.LearnedSpai(A, N, N * N)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with cb.Solver.from_csr(A, restart=10, fmt="f64", arith="fp64") as s64:
        cb.collect_pairs(spai, s64, nrhs=667, iterates=3, gen=gen)
    e1.record(stream); torch.cuda.synchronize()
    t_pairs = e0.elapsed_time(e1)
    e0.record(stream)
    l0, l1 = spai.train(steps=400, lr=3e-3)
    e1.record(stream); torch.cuda.synchronize()
    t_train = e0.elapsed_time(e1)
    # algorithmic FLOPs of one training step: forward (7x64 + 64x64 + 64x7 MACs per row) and
    # backward (dH2 64x7, dH1 64x64, weight gradients 64x64 + 64x7 + 7x64 MACs per row)
    flops_step = 2.0 * A.n * (7 * 64 + 64 * 64 + 64 * 7 + 64 * 7 + 64 * 64 + 64 * 64 + 64 * 7 + 7 * 64)
    tf = flops_step * 400 / (t_train * 1e-3) / 1e12
    _, tpk_kind, tpk = measured_tensor_peak()
    train_info = {"algorithmic_flop_per_step": flops_step, "tflops": round(tf, 2),
                  "roofline": {"bound": "tensor", "kernel": "k_mlp_tc<train> (BF16, FP32 accumulate)",
                               "achieved": round(tf, 2), "peak": tpk, "unit": "TFLOP/s", "frac": round(tf / tpk, 5),
                               "traffic": None, "peak_source": tpk_kind,
                               "note": "per training step: the fused network pass plus the gradient sum and "
                                       "the Adam update (two small kernels)"}}
    pv = spai.values()
    out, solvers, launches = {}, {}, 0
    peak, kind = measured_peaks()
    roof = None
    for pc in ("none", "jacobi", "spai"):
        s = cb.Solver.from_csr(A, restart=100, fmt="f32", precond=pc, profile=True)
        if pc == "spai":
            s.set_spai(pv)
        for _ in range(args.warmup):
            timed_solve(s, b, x, 1e-10, args.maxit, stream)
        s.profile(reset=True)
        ts = []
        for _ in range(args.steps):
            t, st = timed_solve(s, b, x, 1e-10, args.maxit, stream)
            ts.append(t)
            launches += st["kernel_launches"]
        if pc == "spai":
            roof = roofline_from_profile(s.profile(), "f32, learned SPAI",
                                         {"basis_dot": "k_basis_dot_tma", "basis_axpy": "k_basis_axpy"}, peak, kind)
        res = float(np.linalg.norm(bnp - O.spmv(A, x.cpu().numpy())) / np.linalg.norm(bnp))
        out[pc] = {"ms": sum(ts) / len(ts), "iters": st["iters"], "status": st["status"], "true_relres": res}
        solvers[pc] = s
    clk = clocks.stop()
    cpu = None
    if not args.no_cpu:
        hc = host_cpu()
        pvh = pv.cpu().numpy()
        kw = dict(precond=O.PC_SPAI, pvals=pvh)
        s_all = oracle_step_seconds(A, bnp, "f32", 100, hc["nproc"], **kw)
        s_one = oracle_step_seconds(A, bnp, "f32", 100, 1, steps=25, **kw)
        it = out["spai"]["iters"]
        cpu = cpu_line(s_all * it, s_one * it, out["spai"]["ms"] / 1000,
                       f"oracle with the trained SPAI (f32 basis): one full restart cycle (100 steps) on all "
                       f"host threads, the first 25 steps on 1 thread; time-to-solution extrapolated by the "
                       f"solve's {it} steps", hc, True)
    e2e = e2e_host_ratio(solvers, "jacobi", "spai", bnp, A.n, 1e-10, args.maxit, args.steps)
    for s in solvers.values():
        s.close()
    line = {"metric": METRIC, "value": round(out["jacobi"]["ms"] / out["spai"]["ms"], 4), "unit": "x",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sum(v["ms"] for v in out.values()), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "df32", "data": "synthetic",
            "config": {"workload": L96_WORKLOAD, "value_is": "time(Jacobi) / time(learned SPAI), f32 basis",
                       "pairs": spai.npairs, "train_steps": 400,
                       "l2": "no flush: basis (0.36 GB) exceeds the 129 MB L2"},
            "solves": out,
            "train": {"pairs_ms": t_pairs, "train_ms": t_train, "loss_first": l0, "loss_last": l1, **train_info},
            "speedup_learned_vs_none": round(out["none"]["ms"] / out["spai"]["ms"], 4),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
    spai.close()
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------ restart sweep (E6)
def run_restart_sweep(args):
    """10 fixed restart cycles for m = 10..300, every format, numerics ignored: the speedup
    over the f64 basis as the basis share of the traffic grows (Section 5.4, Fig. restart)."""
    import torch
    import paper_2009_12101_gb300 as cb
    cb.ensure_built()
    A, xs, bnp = build_problem(args.grid)
    stream = torch.cuda.current_stream()
    b = torch.from_numpy(bnp).cuda()
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    fmts = ["f64", "f32", "f16", "bf16", "e4m3", "i32", "i16"]
    peak, kind = measured_peaks()
    rows, launches, roof = [], 0, None
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))).start()
    keep = {}
    for m in (10, 25, 50, 100, 150, 200, 250, 300):
        t = {}
        for f in fmts:
            s = cb.Solver.from_csr(A, restart=m, fmt=f, profile=True)
            for _ in range(args.warmup):
                timed_solve(s, b, x, 0.0, 10 * m, stream)
            s.profile(reset=True)
            ts = []
            for _ in range(args.steps):
                tt, st = timed_solve(s, b, x, 0.0, 10 * m, stream)
                launches += st["kernel_launches"]
                ts.append(tt)
            t[f] = sum(ts) / len(ts)
            if m == 300 and f == "f32":
                roof = roofline_from_profile(s.profile(), "f32, m 300",
                                             {"basis_dot": "k_basis_dot_tma", "basis_axpy": "k_basis_axpy"}, peak, kind)
            if m == 100 and f in ("f64", "f32"):
                keep[f] = s
            else:
                s.close()
        rows.append({"m": m, "ms": t, "speedup_vs_f64": {f: round(t["f64"] / v, 4) for f, v in t.items()}})
    clk = clocks.stop()
    cpu = None
    t100 = rows[3]["ms"]["f32"] / 1000
    if not args.no_cpu:
        hc = host_cpu()
        s_all = oracle_step_seconds(A, bnp, "f32", 100, hc["nproc"])
        s_one = oracle_step_seconds(A, bnp, "f32", 100, 1, steps=25)
        cpu = cpu_line(s_all * 1000, s_one * 1000, t100,
                       "oracle, m = 100, f32 basis: one full restart cycle on all host threads, the first 25 "
                       "steps on 1 thread; the 10 fixed cycles (1000 steps) extrapolated", hc, True)
    e2e = e2e_host_ratio(keep, "f64", "f32", bnp, A.n, 0.0, 1000, args.steps)
    for s in keep.values():
        s.close()
    line = {"metric": METRIC, "value": rows[-1]["speedup_vs_f64"]["f32"], "unit": "x", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sum(sum(r["ms"].values()) for r in rows), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "df32", "data": "synthetic",
            "config": {"workload": f"restart_sweep_{WORKLOAD}", "cycles": 10,
                       "value_is": "time(f64 basis) / time(f32 basis) at m = 300; rows: every m and format",
                       "l2": "no flush: every basis exceeds the 129 MB L2"},
            "rows": rows, "roofline": roof, "cpu_baseline": cpu,
            "e2e": dict(e2e, note="m = 100, 10 fixed cycles, f64 / f32 basis"),
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------ multi-RHS basis product
def run_multirhs(args):
    """H = V^T W for k = 8 vectors sharing one basis (n = 2^21, 100 columns): the f16 basis
    on the tensor cores (tcgen05, exact digit products) and on the CUDA cores (double-float),
    the f32 basis on the CUDA cores, and 8 single-vector launches for comparison."""
    import torch
    import oracle as O
    import paper_2009_12101_gb300 as cb
    cb.ensure_built()
    n, ncols, k = 1 << 21, 100, 8
    ld = n
    rng = np.random.default_rng(20201207)
    stream = torch.cuda.current_stream()
    v32 = rng.standard_normal((ncols, ld)) / np.sqrt(n)
    V32 = torch.from_numpy(v32.astype(np.float32)).cuda().view(torch.uint8)
    v16 = v32.astype(np.float16)
    V16 = torch.from_numpy(v16).cuda().view(torch.uint8)
    scales = torch.ones(ncols, dtype=torch.float64, device="cuda")      # resident, like V and W
    Wnp = rng.standard_normal((k, n))
    W = torch.from_numpy(Wnp).cuda()
    ws = torch.empty(cb.lib().cbg_basis_dot_multi_workspace(ld, ncols, k), dtype=torch.uint8, device="cuda")
    H = torch.empty(ncols, k, dtype=torch.float64, device="cuda")
    H1 = [torch.empty(ncols, 1, dtype=torch.float64, device="cuda") for _ in range(k)]
    cases = {
        "f16_tensor_k8": lambda: cb.basis_dot_multi("f16", n, V16, ld, scales, W, workspace=ws, path="tensor", out=H),
        "f16_cuda_k8": lambda: cb.basis_dot_multi("f16", n, V16, ld, scales, W, workspace=ws, path="cuda", out=H),
        "f32_cuda_k8": lambda: cb.basis_dot_multi("f32", n, V32, ld, scales, W, workspace=ws, path="cuda", out=H),
        "f16_tensor_8x_k1": lambda: [cb.basis_dot_multi("f16", n, V16, ld, scales, W[r:r + 1], workspace=ws,
                                                        path="tensor", out=H1[r]) for r in range(k)],
    }
    out = {}
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))).start()
    for name, fn in cases.items():
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    launches = args.steps * (2 + 2 + 2 + 2 * k)     # product + reduction kernels per call
    Ht = cases["f16_tensor_k8"]().cpu().numpy().copy()
    Hc = cases["f16_cuda_k8"]().cpu().numpy().copy()
    agree = float(np.max(np.abs(Ht - Hc)) / np.max(np.abs(Hc)))
    # end to end: W from pinned host memory, the product, H back to the host
    Wh = torch.from_numpy(Wnp).pin_memory()
    Hh = torch.empty(ncols, k, dtype=torch.float64).pin_memory()
    te = {}
    for path in ("cuda", "tensor"):
        ts = []
        for _ in range(max(1, args.steps)):
            torch.cuda.synchronize(); t0 = time.perf_counter()
            Wd = Wh.cuda(non_blocking=True)
            cb.basis_dot_multi("f16", n, V16, ld, scales, Wd, workspace=ws, path=path, out=H)
            Hh.copy_(H); torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        te[path] = sum(ts) / len(ts)
    e2e = {"value": te["cuda"] / te["tensor"], "unit": "x", "h2d_bytes_per_step": 8 * k * n,
           "d2h_bytes_per_step": 8 * k * ncols, "seconds": {p: round(v, 5) for p, v in te.items()}}
    cpu = None
    if not args.no_cpu:
        hc = host_cpu()
        cols = list(range(0, ncols, 10))            # 10 of the 100 columns, all 8 vectors
        dec = [O.decode(O.F16, v16[c].view(np.uint16), 1.0) for c in cols]
        fn = lambda: [[O.dot(d, Wnp[r]) for r in range(k)] for d in dec]
        t_all, _ = oracle_timed(hc["nproc"], fn)
        t_one, _ = oracle_timed(1, fn)
        sc = ncols / len(cols)
        cpu = cpu_line(t_all * sc, t_one * sc, out["f16_tensor_k8"] / 1000,
                       "oracle inner products of 10 of the 100 decoded f16 columns with all 8 vectors, "
                       "extrapolated to the 100 x 8 product", hc, True)
    peak, kind = measured_peaks()
    vbytes16 = ncols * n * 2 + k * n * 8                     # algorithmic bytes: V codes + W
    tflops = 2 * 2 * 128 * 112 * n / (out["f16_tensor_k8"] * 1e-3) / 1e12   # 2 V slices, M = 128, N = 112
    line = {"metric": METRIC, "value": round(out["f16_cuda_k8"] / out["f16_tensor_k8"], 4), "unit": "x",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(out["f16_tensor_k8"], 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16 digits / fp32 accumulate",
            "data": "synthetic",
            "config": {"workload": "multirhs_n2097152_cols100_k8",
                       "value_is": "time(f16 basis, CUDA cores) / time(f16 basis, tensor cores)",
                       "l2": "no flush: V (0.42 GB f16) exceeds the 129 MB L2"},
            "ms": {kk: round(v, 4) for kk, v in out.items()},
            "tensor_vs_cuda_max_rel_diff": agree,
            "roofline": {"bound": "hbm", "kernel": "k_dot_multi_tc (f16 basis, k = 8)",
                         "achieved": round(vbytes16 / (out["f16_tensor_k8"] * 1e-3) / 1e9, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(vbytes16 / (out["f16_tensor_k8"] * 1e-3) / 1e9 / peak, 4),
                         "traffic": None, "peak_source": f"{kind} hbm_gbs (MEASURED_PEAKS.json)",
                         "tensor_tflops_issued": round(tflops, 1)},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------ plain FP64 GMRES (Poisson)
P64_WORKLOAD = "poisson2d_64x64_restart100_tol1e-10_f64"


def run_poisson64(args):
    """2D 5-point Poisson on a 64 x 64 grid (n = 4096), plain FP64 GMRES(100) with CGS and
    re-orthogonalisation, no preconditioner, tol 1e-10; the f32 basis beside it.  The basis
    (3.3 MB) stays in L2: a latency and correctness configuration."""
    import torch
    import oracle as O
    import paper_2009_12101_gb300 as cb
    import workloads as W
    cb.ensure_built()
    stream = torch.cuda.current_stream()
    A = W.poisson2d(64)
    xs = W.exact_solution(A.n, 1)
    bnp = W.rhs_from_solution(A, xs)
    b = torch.from_numpy(bnp).cuda()
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    fmts = ("f64", "f32")
    peak, kind = measured_peaks()
    solvers = {f: cb.Solver.from_csr(A, restart=100, fmt=f, profile=True) for f in fmts}
    flush = l2_flusher()       # the 3.3 MB basis would otherwise stay in L2 between solves
    out, launches = {}, 0
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))).start()
    for f, s in solvers.items():
        for _ in range(args.warmup):
            timed_solve(s, b, x, 1e-10, args.maxit, stream, flush)
        s.profile(reset=True)
        ts = []
        for _ in range(args.steps):
            t, st = timed_solve(s, b, x, 1e-10, args.maxit, stream, flush)
            ts.append(t)
            launches += st["kernel_launches"]
        res = float(np.linalg.norm(bnp - O.spmv(A, x.cpu().numpy())) / np.linalg.norm(bnp))
        out[f] = {"ms": sum(ts) / len(ts), "iters": st["iters"], "status": st["status"], "true_relres": res,
                  "roofline": roofline_from_profile(s.profile(), f, {"basis_dot": "k_basis_dot_tma",
                                                                     "basis_axpy": "k_basis_axpy"}, peak, kind)}
    clk = clocks.stop()
    hc = host_cpu()
    t_all, ro = oracle_timed(hc["nproc"], lambda: O.gmres(A, bnp, m=100, fmt=O.F64, tol=1e-10, maxit=args.maxit))
    t_one, _ = oracle_timed(1, lambda: O.gmres(A, bnp, m=100, fmt=O.F64, tol=1e-10, maxit=args.maxit))
    xg = None
    with cb.Solver.from_csr(A, restart=100, fmt="f64") as s:
        xt = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        st = s.solve(b, xt, tol=1e-10, maxit=args.maxit)
        xg = xt.cpu().numpy()
    cpu = cpu_line(t_all, t_one, out["f64"]["ms"] / 1000,
                   "oracle full solve (f64 basis, GMRES(100), tol 1e-10) on all host threads and on 1 (n = 4096 is "
                   "below the oracle's threading threshold, so both run on one core)", hc, False,
                   oracle_iters=int(ro["iters"]), gpu_iters=int(st["iters"]),
                   x_relerr_vs_oracle=float(np.linalg.norm(xg - ro["x"]) / np.linalg.norm(ro["x"])))
    e2e = e2e_host_ratio(solvers, "f64", "f32", bnp, A.n, 1e-10, args.maxit, args.steps, flush)
    for s in solvers.values():
        s.close()
    line = {"metric": METRIC, "value": round(out["f64"]["ms"] / out["f32"]["ms"], 4), "unit": "x", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sum(v["ms"] for v in out.values()), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "df32", "data": "synthetic",
            "config": {"workload": P64_WORKLOAD, "n": A.n, "nnz": A.nnz, "restart": 100,
                       "value_is": "time(f64 basis) / time(f32 basis)",
                       "l2": "flushed before every timed solve (256 MiB write outside the timed interval); "
                             "the 3.3 MB basis is L2-resident within a solve, so the HBM roofline does not bind"},
            "solves": {f: {k: v for k, v in d.items() if k != "roofline"} for f, d in out.items()},
            "time_to_solution_s": {f: round(d["ms"] / 1000, 5) for f, d in out.items()},
            "roofline": out["f64"]["roofline"], "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch512":
        return run_batch(args)
    if args.workload == "random27":
        return run_random27(args)
    if args.workload == "learned96":
        return run_learned96(args)
    if args.workload == "restart_sweep":
        return run_restart_sweep(args)
    if args.workload == "multirhs":
        return run_multirhs(args)
    if args.workload == "poisson64":
        return run_poisson64(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2009_12101_gb300 as cb
    cb.ensure_built()
    cb.lib()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    fmts = args.formats.split(",")
    if "f64" not in fmts:
        fmts = fmts + ["f64"]      # the baseline of the speedup
    A, xs, b = build_problem(args.grid)
    n = A.n
    stream = torch.cuda.current_stream()
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    solvers = {f: cb.Solver.from_csr(A, restart=args.restart, fmt=f, arith=args.arith, precond=args.precond,
                                     spmv_group=args.spmv_group,
                                     adapt=args.adapt, ortho=args.ortho, profile=True)
               for f in fmts}

    def solve_all(record):
        out = {}
        for f in fmts:
            x.zero_()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = solvers[f].solve(bd, x, tol=args.tol, maxit=args.maxit)
            e1.record(stream)
            out[f] = (e0, e1, st)
        return out

    for _ in range(args.warmup):
        solve_all(False)
    for s in solvers.values():
        s.profile(reset=True)

    clocks = ClockSampler(local).start()
    barrier()
    g0 = torch.cuda.Event(enable_timing=True); g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    runs = [solve_all(True) for _ in range(args.steps)]
    g1.record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = g0.elapsed_time(g1)

    per_fmt = {f: [r[f][0].elapsed_time(r[f][1]) for r in runs] for f in fmts}
    stats = {f: runs[-1][f][2] for f in fmts}
    launches = sum(r[f][2]["kernel_launches"] for r in runs for f in fmts)
    t_fmt = {f: sum(v) / len(v) for f, v in per_fmt.items()}
    if world > 1:
        t_fmt = max_over_ranks(t_fmt, "cuda")
    speedup = {f: t_fmt["f64"] / t_fmt[f] for f in fmts}
    value = speedup[args.headline]

    # live roofline of the basis GEMV kernels (headline format, timed region)
    peak, peak_kind = measured_peaks()
    prof = {f: solvers[f].profile() for f in fmts}
    ph = prof[args.headline]
    cls = max(("basis_dot", "basis_axpy"), key=lambda c: ph[c]["ms"])
    launches_cls = max(1, ph[cls]["launches"])
    avg_ms = ph[cls]["ms"] / launches_cls
    avg_bytes = ph[cls]["bytes"] / launches_cls
    achieved = avg_bytes / (avg_ms * 1e-3) / 1e9
    tpe = ncu_traffic_per_element(args.headline).get(cls)
    fb = cb.FORMAT_BYTES[args.headline]
    traffic = tpe * (avg_bytes / fb) if tpe else None
    gemv = {}
    for f in fmts:
        for c in ("basis_dot", "basis_axpy"):
            p = prof[f][c]
            if p["ms"] > 0:
                gemv[f"{f}/{c}"] = round(p["bytes"] / (p["ms"] * 1e-3) / 1e9, 1)
    kname = {"basis_dot": "k_basis_dot_tma" if args.arith == "df32" else "k_basis_dot",
             "basis_axpy": "k_basis_axpy"}[cls]
    roofline = {"bound": "hbm", "kernel": f"{kname} ({args.headline}, {args.arith})",
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
                "algorithmic_bytes_per_launch": avg_bytes, "avg_launch_ms": avg_ms,
                "basis_gemv_gbs_by_format": gemv,
                "kernel_classes": kernel_class_table(ph)}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        bh = torch.from_numpy(b).pin_memory().numpy()
        xh = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
        te = {}
        for f in ("f64", args.headline):
            ts = []
            for _ in range(max(1, args.steps)):
                xh[:] = 0.0
                barrier()
                t0 = time.perf_counter()
                solvers[f].solve_host(bh, xh, tol=args.tol, maxit=args.maxit)
                ts.append(time.perf_counter() - t0)
            te[f] = sum(ts) / len(ts)
        if world > 1:
            te = max_over_ranks({"f64": te["f64"], args.headline: te[args.headline]}, "cuda")
        e2e = {"value": te["f64"] / te[args.headline], "unit": "x",
               "h2d_bytes_per_step": 2 * 2 * 8 * n, "d2h_bytes_per_step": 2 * 8 * n,
               "seconds": {k: round(v, 4) for k, v in te.items()}}

    # FP64 arithmetic beside the double-float reading: the same solves with native FP64
    # basis products and SpMV (what the paper's arithmetic costs on this GPU)
    arith64 = None
    if args.arith == "df32" and not args.no_fp64:
        reps = max(1, min(args.steps, 3))
        s64 = {f: cb.Solver.from_csr(A, restart=args.restart, fmt=f, arith="fp64", precond=args.precond,
                                     ortho=args.ortho) for f in ("f64", args.headline)}
        clocks64 = ClockSampler(local).start()
        t64a, it64a = {}, {}
        for f, s in s64.items():
            timed_solve(s, bd, x, args.tol, args.maxit, stream)
            ts = []
            for _ in range(reps):
                tt, st = timed_solve(s, bd, x, args.tol, args.maxit, stream)
                ts.append(tt)
            t64a[f], it64a[f] = sum(ts) / len(ts), st["iters"]
            s.close()
        clk64 = clocks64.stop()
        if world > 1:
            t64a = max_over_ranks(t64a, "cuda")
        arith64 = {"time_to_solution_s": {f: round(v / 1000, 4) for f, v in t64a.items()},
                   "speedup_vs_f64": {f: round(t64a["f64"] / v, 4) for f, v in t64a.items()},
                   "iterations": it64a,
                   "double_float_gain": {f: round(t64a[f] / t_fmt[f], 4) for f in t64a},
                   "note": "basis products and per-step SpMV in native FP64 (CBG_ARITH_FP64), same solves; "
                           "double_float_gain = time(FP64 arithmetic) / time(double-float arithmetic)",
                   "solves_per_format": reps, "clocks": clk64}

    # CPU baseline: the oracle (rank 0, N = 1 only) over one full restart cycle per
    # format on all host threads, and on one thread for the headline format; the
    # time-to-solution is extrapolated with the solve's step count
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        hc = host_cpu()
        hf = args.headline
        s_all = {f: oracle_step_seconds(A, b, f, args.restart, hc["nproc"]) for f in ("f64", hf)}
        s_one = oracle_step_seconds(A, b, hf, args.restart, 1, steps=args.cpu_steps)
        tts_all = {f: s_all[f] * stats[f]["iters"] for f in s_all}
        cpu = cpu_line(tts_all[hf], s_one * stats[hf]["iters"], t_fmt[hf] / 1000,
                       (f"oracle (plain C, {hc['nproc']} host threads): one full restart cycle (Arnoldi steps "
                        f"j = 1..{args.restart}) of the {WORKLOAD} solve with the {hf} and f64 basis; 1 thread: "
                        f"the first {args.cpu_steps} steps with the {hf} basis (short steps: biased low); "
                        f"time-to-solution extrapolated as seconds per step x the solve's steps "
                        f"({stats[hf]['iters']})"),
                       hc, True,
                       oracle_s_per_step_all_threads={f: round(v, 5) for f, v in s_all.items()},
                       oracle_s_per_step_1_thread={hf: round(s_one, 5)},
                       oracle_time_to_solution_s_all_threads={f: round(v, 3) for f, v in tts_all.items()},
                       oracle_f64_over_headline=round(tts_all["f64"] / tts_all[hf], 4))

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "x", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "df32" if args.arith == "df32" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + ("" if args.precond == "none" else f"_{args.precond}")
                                   + ("_adaptive" if args.adapt else "") + ("_mgs" if args.ortho == "mgs" else ""),
                       "n": n, "nnz": A.nnz, "restart": args.restart, "precond": args.precond,
                       "orthogonalisation": args.ortho,
                       "adaptive_format": bool(args.adapt),
                       "tol": args.tol, "headline_format": args.headline, "formats": fmts,
                       "arith": ("basis products and the per-step SpMV in double-float (FP32 pairs); "
                                 "residual SpMV, norms, Givens, least squares in FP64"
                                 if args.arith == "df32" else "all FP64"),
                       "parallelism": f"replicas{world}" if world > 1 else "single-gpu",
                       "l2": "no flush: every basis (>= 0.4 GB per format) exceeds the 129 MB L2"},
            "time_to_solution_s": {f: round(t_fmt[f] / 1000, 4) for f in fmts},
            "speedup_vs_f64": {f: round(v, 4) for f, v in speedup.items()},
            "iterations": {f: stats[f]["iters"] for f in fmts},
            "final_format": {f: stats[f]["fmt_final"] for f in fmts},
            "spmv_schedule": {f: solvers[f].spmv_group() for f in fmts},
            "true_relres": {f: stats[f]["true_relres"] for f in fmts},
            "status": {f: stats[f]["status"] for f in fmts},
            "roofline": roofline,
            "arith_fp64": arith64,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    for s in solvers.values():
        s.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
