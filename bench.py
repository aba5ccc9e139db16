#!/usr/bin/env python
"""Benchmark of the generalized-Poisson pressure solve (one solve = one step).

Workload (default): the 3D 256^3 stratified-convection pressure solve --
x,y periodic, z walls, 20x density contrast with 1% seeded noise, dt at
Ma = 0.01 -- solved to relative residual 1e-8 by the mixed-precision mode
(float32 flexible CG + geometric multigrid inside float64 iterative
refinement).  A step is the whole hot path: coefficient assembly from
rho^n, rho^{n+1}, c_s^2, dt; multigrid hierarchy set-up; the refinement
solve to tolerance.  Inputs (4 x 134 MB) already sit in HBM and exceed L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  value = cells solved to rtol per second
over the whole job (GDOF/s; N GPUs run independent replicas: weak scaling).
The float64 Jacobi-PCG baseline is timed on the same GPU after the timed
region; `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-1e-8 residual & GDOF-iter/s: mixed+learned vs FP64 PCG, same GPU"
UNIT = "GDOF/s"
WORKLOADS = {
    "convection256": dict(kind="conv3d", n=256, desc="3D 256^3 convection, rho contrast 20 + 1% noise, "
                                                    "Ma=0.01, x/y periodic, z walls, rtol 1e-8"),
    "convection128": dict(kind="conv3d", n=128, desc="3D 128^3 convection (reduced), Ma=0.01, rtol 1e-8"),
    "plain64": dict(kind="plain2d", n=64, desc="2D 64^2 polytrope, Ma=0.1, rtol 1e-10"),
    "batch64": dict(kind="batch", n=64, desc="64 uneven 2D solves, sides from {128,256,512,1024}^2, Ma log-uniform "
                                             "[1e-3,1e-1], density contrast U[5,30], rtol 1e-8, one batched graph"),
    "learned256": dict(kind="train2d", n=256, desc="2D 256^2 held-out problems of the learned-part family (seeds "
                                                   "30000+, contrast U[5,30], Ma log-uniform [1e-3,1e-1]), "
                                                   "rtol 1e-8, learned warm start + preconditioner"),
    "semiconvection512": dict(kind="semi3d", n=512, desc="3D 512^3 two-component semiconvection (R_rho 1.1, "
                                                         "1% T and helium perturbations), Ma=0.001, rtol 1e-8"),
}
DEFAULT_MODE = {"train2d": "learned"}
# dram__bytes_read.sum + dram__bytes_write.sum of one launch, from an ncu
# capture of the same kernel build on this workload, keyed (workload, kernel)
NCU_TRAFFIC: dict = {
    # plain level-0 sweep of the 256^3 workload: 293.7 MB read + 46.4 MB written
    ("convection256", "k_rbgs_row"): 340.05e6,
}


def sweep_kernel(n):
    """Name of the sweep kernel the library picks for a finest level of n = (nx, ny, nz) cells."""
    nx, ny, nz = n
    if ny > 1 and ny % 16 == 0 and nz >= 2 and nx in (128, 256):
        return "k_rbgs_row"
    if ny > 1 and nx % 32 == 0 and ny % 8 == 0 and nz >= 2:
        return "k_rbgs_zm"
    if ny == 1 and nx % 256 == 0 and nz >= 2:
        return "k_rbgs_zm2d"
    return "k_rbgs"
WEIGHTS = os.path.join(ROOT, "paper_1112_3507_gb300", "weights", "unet_16_32_48_64.bin")


def make_problem(name: str, seed: int = 1):
    from paper_1112_3507_gb300 import inputs as I
    w = WORKLOADS[name]
    if w["kind"] == "conv3d":
        return I.config_convection_3d(w["n"], seed=seed)
    if w["kind"] == "semi3d":
        return I.config_semiconvection_3d(w["n"], seed=7)
    if w["kind"] == "train2d":
        return I.config_training_2d(30000 + seed - 1, n=w["n"])
    return I.config_plain_2d(w["n"], seed=seed)


def downsized(name: str, m: int, seed: int = 1):
    """The workload's recipe on an m-cell-per-axis grid (oracle iteration counts)."""
    from paper_1112_3507_gb300 import inputs as I
    kind = WORKLOADS[name]["kind"]
    if kind == "conv3d":
        return I.config_convection_3d(m, seed=seed)
    if kind == "semi3d":
        return I.config_semiconvection_3d(m, seed=7)
    return make_problem(name, seed)


def job_time(elapsed_s: float, world: int, device=None) -> float:
    """The job's time: the maximum over ranks of each rank's elapsed seconds."""
    if world <= 1:
        return elapsed_s
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cells_per_step: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput in GDOF/s: every rank solves its own replica."""
    return world * cells_per_step * steps / seconds / 1e9


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def oracle_calibrate(name: str, seed: int = 1):
    """The workload's problem and oracle operator, and the oracle's own
    iteration count to the workload's tolerance: measured on downsized grids
    of the same recipe and extrapolated by the fitted growth per doubling."""
    from oracle import poisson as P
    w = WORKLOADS[name]
    p = make_problem(name, seed)
    op = P.operator_from_problem(p)
    counts = []
    n = w["n"]
    big = n // 8 if n > 256 else n // 4               # largest downsized grid the oracle solves in seconds
    sizes = [big // 4, big // 2, big] if w["kind"] in ("conv3d", "semi3d") else [n]
    for m in sizes:
        q = downsized(name, m, seed) if len(sizes) > 1 else p
        _, c, _ = P.solve_pcg_jacobi(P.operator_from_problem(q), q.f, rtol=p.rtol, maxiter=200000)
        counts.append(c)
    if len(counts) > 1:
        growth = (counts[-1] / counts[0]) ** (1.0 / (len(counts) - 1))
        est_iters = counts[-1] * growth ** round(np.log2(n / big))
    else:
        est_iters = counts[0]
    return p, op, counts, float(est_iters)


def oracle_steps(name: str, steps: int, warmup: int, iters_per_step: int = 2) -> dict:
    """The reference arm: calibrate once, then time warmup + steps bounded
    samples, each `iters_per_step` full-size iterations of the oracle's
    float64 Jacobi-PCG (its set-up included); each sample's time per
    iteration times the oracle's iteration count to tolerance is that step's
    estimated time to tolerance."""
    from oracle import poisson as P
    p, op, counts, est_iters = oracle_calibrate(name)
    per_iter = []
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        P.solve_pcg_jacobi(op, p.f, rtol=0.0, maxiter=iters_per_step)
        if k >= warmup:
            per_iter.append((time.perf_counter() - t0) / iters_per_step)
    return dict(per_iter_s=per_iter, est_iters=est_iters, downsized_counts=counts, N=p.size,
                iters_per_step=iters_per_step)


def oracle_sample(name: str, iters: int = 2, seed: int = 1) -> dict:
    """Time the oracle's float64 Jacobi-PCG on the workload (single-threaded
    numpy): one run of 1 iteration and one of 1 + `iters` iterations give the
    set-up time and the time per iteration.  The oracle's own iteration count
    to the workload's tolerance is measured on downsized grids (n/16, n/8,
    n/4) and extrapolated by the fitted growth per grid doubling.  Returns the
    estimated time to tolerance and the GDOF/s it implies."""
    from oracle import poisson as P
    p, op, counts, est_iters = oracle_calibrate(name, seed)
    P.solve_pcg_jacobi(op, p.f, rtol=0.0, maxiter=1)          # warm-up (first-touch of the arrays)
    t0 = time.perf_counter()
    P.solve_pcg_jacobi(op, p.f, rtol=0.0, maxiter=1)
    t1 = time.perf_counter()
    _, it, _ = P.solve_pcg_jacobi(op, p.f, rtol=0.0, maxiter=1 + iters)
    t2 = time.perf_counter()
    t_iter = max((t2 - t1) - (t1 - t0), 1e-9) / max(it - 1, 1)
    t_setup = max((t1 - t0) - t_iter, 0.0)
    est_s = t_setup + t_iter * est_iters
    return dict(t_iter_s=t_iter, t_setup_s=t_setup, sample_iters=it + 1, est_iters=float(est_iters),
                downsized_counts=counts, est_time_s=est_s, value=p.size / est_s / 1e9, N=p.size)


def oracle_subprocess(name: str, iters: int, call: str | None = None) -> dict:
    """Run an oracle timing in a single-threaded child process."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    call = call or "bench.oracle_sample(%r, %d)" % (name, iters)
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print('ORACLE_JSON', json.dumps(%s))" % (ROOT, call))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    for line in r.stdout.splitlines():
        if line.startswith("ORACLE_JSON"):
            return json.loads(line.split(" ", 1)[1])
    raise RuntimeError("oracle sample failed:\n" + r.stdout[-2000:] + r.stderr[-2000:])


def cpu_block(s: dict, name: str) -> dict:
    return {"value": s["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{s['sample_iters']} iterations of the FP64 oracle's Jacobi-PCG on {name} "
                       f"({s['t_iter_s']:.3f} s/iter + {s['t_setup_s']:.2f} s set-up, single-threaded numpy) "
                       f"x its iteration count to rtol "
                       f"extrapolated from downsized grids {s['downsized_counts']} -> {s['est_iters']:.0f}; "
                       f"estimated time to tolerance {s['est_time_s']:.1f} s")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    r = oracle_subprocess(args.workload, 0, call="bench.oracle_steps(%r, %d, %d)" % (args.workload, args.steps,
                                                                                   args.warmup))
    t_iter = statistics.median(r["per_iter_s"])
    est = t_iter * r["est_iters"]
    value = r["N"] / est / 1e9
    cpu = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": (f"per step {r['iters_per_step']} full-size iterations of the FP64 oracle's Jacobi-PCG on "
                      f"{args.workload} (single-threaded numpy; median {t_iter:.3f} s/iter over {args.steps} "
                      f"steps) x its iteration count to rtol extrapolated from downsized grids "
                      f"{r['downsized_counts']} -> {r['est_iters']:.0f}; estimated time to tolerance {est:.1f} s")}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": est * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload]["desc"], "cells": r["N"]},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def time_kernel(torch, fn, reps: int, stream) -> float:
    """Average duration (s) of fn() launched `reps` times, CUDA events on `stream`."""
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e-3 / reps


def run_batch(args):
    """The batched workload: one step = coefficient assembly + rhs for 64
    uneven 2D grids and one lm_batch_solve; compared with the same solves one
    grid at a time (mixed mode) and with the float64 Jacobi-PCG baseline."""
    import torch

    from paper_1112_3507_gb300 import lowmach as lm

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    from paper_1112_3507_gb300 import inputs as I
    probs = I.config_batch(count=64, seed=42)
    ncells = sum(p.size for p in probs)
    tens = [[torch.as_tensor(a.ravel(), device=dev) for a in (p.rho_old, p.rho_new, p.cs2, p.f)] for p in probs]
    grids = [lm.Grid.for_problem(p) for p in probs]

    def load():
        for p, g, t in zip(probs, grids, tens):
            g.set_coefficients(t[0], t[1], t[2], p.dt, stream)
            g.set_rhs(t[3], stream)

    def step():
        load()
        return lm.batch_solve(grids, rtol=1e-8, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = lm.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    results = [step() for _ in range(args.steps)]
    e1.record(stream)
    e1.synchronize()
    launches = lm.kernel_launches() - launches0
    clk = clocks.stop()
    t_step = e0.elapsed_time(e1) * 1e-3 / args.steps
    res = results[-1]
    assert all(r["status"] == 0 and r["rel_residual"] <= 1e-8 for r in res)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    def seq(mode):
        load()
        return [g.solve(mode=mode, rtol=1e-8, stream=stream, max_iter=args.max_iter) for g in grids]

    seq("mixed")
    t_seq, rs = timed(lambda: seq("mixed"))
    t_jac, rj = timed(lambda: seq("jacobi"))
    line = {"workload": WORKLOADS["batch64"]["desc"], "cells": ncells, "ms_per_batch": t_step * 1e3,
            "gdof_per_s": ncells / t_step / 1e9, "steps": args.steps, "warmup": args.warmup,
            "inner_iters_max": max(r["iters"] for r in res), "outer_iters_max": max(r["outer_iters"] for r in res),
            "sequential_mixed_ms": t_seq * 1e3, "sequential_fp64_jacobi_ms": t_jac * 1e3,
            "speedup_vs_sequential_mixed": t_seq / t_step, "speedup_vs_fp64_pcg": t_jac / t_step,
            "jacobi_iters_total": sum(r["iters"] for r in rj), "gpu_launches_per_batch": launches / args.steps,
            "clocks": clk}
    print(json.dumps(line), flush=True)
    for g in grids:
        g.close()


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1112_3507_gb300 import lowmach as lm

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    kind = WORKLOADS[args.workload]["kind"]
    mode = args.mode or DEFAULT_MODE.get(kind, "mixed")
    # the learned workload cycles through 8 held-out problems; the others solve one
    probs = [make_problem(args.workload, seed=1 + k) for k in range(8 if kind == "train2d" else 1)]
    p = probs[0]
    N = p.size
    dev_in = [[torch.as_tensor(a.ravel(), device=dev) for a in (q.rho_old, q.rho_new, q.cs2, q.f)] for q in probs]
    g = lm.Grid.for_problem(p)
    if mode == "learned":
        g.load_network(WEIGHTS)
    solve_kw = dict(mode=mode, rtol=p.rtol, max_iter=args.max_iter)
    small = 4 * 8 * N < 2 * 129e6           # inputs that fit in L2 get it flushed between steps
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device=dev) if small else None

    def step(k):
        ro, rn, c2, f = dev_in[k % len(probs)]
        g.set_coefficients(ro, rn, c2, probs[k % len(probs)].dt, stream)
        g.set_rhs(f, stream)
        return g.solve(stream=stream, **solve_kw)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    launches0 = lm.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    results = []
    for k in range(args.steps):
        if flush is not None:
            flush.fill_(float(k))
        ev[k][0].record(stream)
        results.append(step(k))
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = lm.kernel_launches() - launches0
    barrier()
    clk = clocks.stop()
    elapsed = sum(a.elapsed_time(b) for a, b in ev) * 1e-3
    if args.only_steps:                 # profiling runs: the timed solves and nothing else
        if rank == 0:
            print(json.dumps({"only_steps": True, "ms_per_step": elapsed * 1e3 / args.steps,
                              "gpu_launches": launches, "solve": results[-1]}), flush=True)
        g.close()
        return
    elapsed = job_time(elapsed, world, dev)
    res = results[-1]
    assert all(r["status"] == 0 and r["rel_residual"] <= p.rtol for r in results), results
    value = job_value(N, args.steps, world, elapsed)
    t_solve = elapsed / args.steps

    # ---- end to end through the C ABI with host buffers (pinned)
    host = [[torch.from_numpy(np.ascontiguousarray(a.ravel())).pin_memory().numpy()
             for a in (q.rho_old, q.rho_new, q.cs2, q.f)] for q in probs]
    xout = torch.empty(N, dtype=torch.float64).pin_memory().numpy()

    def e2e_step(k):
        hn = host[k % len(probs)]
        g.set_coefficients(hn[0], hn[1], hn[2], probs[k % len(probs)].dt, stream)
        g.set_rhs(hn[3], stream)
        r = g.solve(stream=stream, **solve_kw)
        g.solution(xout, stream)
        return r

    e2e_step(0)
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        e2e_step(k)
    torch.cuda.synchronize()
    e2e_t = job_time(time.perf_counter() - t0, world, dev)

    # ---- the float64 Jacobi-PCG baseline, the float64 multigrid mode and the
    # mixed mode without the network, same GPU, same problems
    base = {}
    others = ["jacobi", "fp64-mg"] + (["mixed"] if mode != "mixed" else [])
    for bmode in others:
        def step_b(k):
            ro, rn, c2, f = dev_in[k % len(probs)]
            g.set_coefficients(ro, rn, c2, probs[k % len(probs)].dt, stream)
            g.set_rhs(f, stream)
            return g.solve(stream=stream, mode=bmode, rtol=p.rtol, max_iter=args.max_iter, allow=(0, -3))
        step_b(0)
        reps = len(probs) if kind == "train2d" else 1
        torch.cuda.synchronize()
        b0 = time.perf_counter()
        rb = [step_b(k) for k in range(reps)]
        torch.cuda.synchronize()
        tb = (time.perf_counter() - b0) / reps
        base[bmode] = {"time_to_tol_ms": tb * 1e3, "iters": rb[-1]["iters"], "status": rb[-1]["status"],
                       "rel_residual": rb[-1]["rel_residual"],
                       "gdof_iter_per_s": N * float(np.mean([r["iters"] for r in rb])) / tb / 1e9}

    # ---- roofline of the dominant kernel (the red-black sweep of the V-cycle),
    # timed alone through its row-level entry point, on the launching stream
    step(0)
    x32 = torch.randn(N, dtype=torch.float32, device=dev)
    f32 = torch.randn(N, dtype=torch.float32, device=dev)
    y32 = torch.empty_like(x32)
    reps = 20
    t_sw = time_kernel(torch, lambda: g.mg_sweep(x32, f32, y32, 0, stream=stream), reps, stream)
    t_ap = time_kernel(torch, lambda: g.apply(x32, y32, prec=lm.PREC_FP32, stream=stream), reps, stream)
    x64 = torch.randn(N, dtype=torch.float64, device=dev)
    y64 = torch.empty_like(x64)
    t_k64 = time_kernel(torch, lambda: g.apply(x64, y64, prec=lm.PREC_FP64, stream=stream), reps, stream)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    sweep_bytes = 20              # read x, f, rho, c~; write x (float32); faces formed on the fly
    achieved = sweep_bytes * N / t_sw / 1e9
    kname = sweep_kernel(tuple(p.n))
    traffic = NCU_TRAFFIC.get((args.workload, kname))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_block(oracle_subprocess(args.workload, args.oracle_iters), args.workload)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_solve * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64 (float32 multigrid/Krylov, float64 residual/refinement)"
            + (", bf16 network" if mode == "learned" else ""),
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "cells": N, "mode": mode,
                       "problems": len(probs), "rtol": p.rtol,
                       "l2": ("flushed between steps (256 MB write)" if small else
                              "inputs exceed L2 (4 x %.0f MB)" % (N * 8 / 1e6)),
                       "parallelism": f"replicas x{world}"},
            "time_to_tol_ms": t_solve * 1e3,
            "solve": {"iters": res["iters"], "outer_iters": res["outer_iters"], "vcycles": res["vcycles"],
                      "rel_residual": res["rel_residual"],
                      "gdof_iter_per_s": N * float(np.mean([r["iters"] for r in results])) / t_solve / 1e9},
            "fp64_jacobi_pcg": base["jacobi"], "fp64_mg_fcg": base["fp64-mg"],
            "speedup_vs_fp64_pcg": base["jacobi"]["time_to_tol_ms"] / (t_solve * 1e3),
            "e2e": {"value": job_value(N, args.steps, world, e2e_t), "unit": UNIT,
                    "h2d_bytes_per_step": 4 * 8 * N, "d2h_bytes_per_step": 8 * N},
            "roofline": {"kernel": kname + " (float32 red-black Gauss-Seidel sweep, row a4)", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "bytes_per_cell": sweep_bytes, "launch_us": t_sw * 1e6,
                         "peak_source": ("MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks
                                         else "fallback 6800 GB/s (of fallback)"),
                         "also": {"apply32": {"bytes_per_cell": 16, "launch_us": t_ap * 1e6,
                                                 "achieved": 16 * N / t_ap / 1e9,
                                                 "frac": 16 * N / t_ap / 1e9 / peak},
                                  "k_apply64": {"launch_us": t_k64 * 1e6,
                                                "note": "float64 ALU-bound on GB300, not HBM-bound"}}},
            "cpu_baseline": cpu,
            "clocks": clk,
            "gpu_launches": launches,
        }
        if mode != "mixed":
            line["mixed_no_network"] = base["mixed"]
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="convection256")
    ap.add_argument("--mode", default=None, help="solve mode (default: learned for learned256, else mixed)")
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--oracle-iters", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-steps", action="store_true",
                    help="run warm-up and timed solves only (for profiler launch lists)")
    args = ap.parse_args()
    args.max_iter = args.max_iter
    if args.impl == "reference":
        run_reference(args)
    elif WORKLOADS[args.workload]["kind"] == "batch":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
