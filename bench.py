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
    "gresho256": dict(kind="gresho2d", n=256, desc="Gresho vortex (Sec. 5.5.2), periodic 256^2, Ma=0.01, "
                                                   "sound-speed-induced dt (CFL 0.5); one step = advection, "
                                                   "projection rhs, coefficients, mixed solve to 1e-11 warm-started "
                                                   "from P^n, projection update, EOS"),
    "fe256": dict(kind="fe3d", n=256, desc="3D 256^3 points, Q1 finite elements (cubic, h = 1/255), convection "
                                           "recipe coefficients (rho contrast 20 + 1% noise, Ma=0.01), x/y "
                                           "periodic, z walls, rtol 1e-8"),
}
DEFAULT_MODE = {"train2d": "learned"}
# dram__bytes_read.sum + dram__bytes_write.sum of one launch, from an ncu
# capture of the same kernel build on this workload, keyed (workload, kernel)
NCU_TRAFFIC: dict = {
    # plain level-0 sweep of the 256^3 workload (the L2-prefetching whole-row
    # kernel): 296.9 MB read + 48.3 MB written (profiles/k_rbgs_row_convection256_level0.md)
    ("convection256", "k_rbgs_row"): 345.13e6,
}


def sweep_kernel(n):
    """Name of the sweep kernel the library picks for a finest level of n = (nx, ny, nz) cells."""
    nx, ny, nz = n
    if ny > 1 and ny % 16 == 0 and nz >= 2 and nx in (128, 256, 512):
        return "k_rbgs_row"
    if ny > 1 and nx % 32 == 0 and ny % 8 == 0 and nz >= 2:
        return "k_rbgs_zm"
    if ny == 1 and nx % 128 == 0 and nz >= 2:
        return "k_rbgs_zm2d"
    return "k_rbgs"
WEIGHTS = os.path.join(ROOT, "paper_1112_3507_gb300", "weights", "unet_16_32_48_64.bin")


def make_problem(name: str, seed: int = 1):
    from paper_1112_3507_gb300 import inputs as I
    w = WORKLOADS[name]
    if w["kind"] in ("conv3d", "fe3d"):
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
ORACLE_SEEDS = (1, 2, 3)


def host_cores() -> int:
    """Host cores this process may run on (its CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_calibrate(name: str, seeds=ORACLE_SEEDS):
    """The oracle's own iteration count to the workload's tolerance, averaged
    over `seeds`.  3D workloads: measured on downsized grids of the same
    recipe (n/16, n/8, n/4 for n <= 256) and extrapolated by the fitted growth
    per grid doubling (an estimate); 2D workloads: the full-size count."""
    from oracle import poisson as P
    w = WORKLOADS[name]
    n = w["n"]
    big = n // 8 if n > 256 else n // 4               # largest downsized grid the oracle solves in seconds
    three_d = w["kind"] in ("conv3d", "semi3d")
    sizes = [big // 4, big // 2, big] if three_d else [n]
    per_seed, ests = [], []
    for seed in (seeds if w["kind"] != "semi3d" else seeds[:1]):
        counts = []
        for m in sizes:
            q = downsized(name, m, seed) if three_d else make_problem(name, seed)
            _, c, _ = P.solve_pcg_jacobi(P.operator_from_problem(q), q.f, rtol=q.rtol, maxiter=200000)
            counts.append(c)
        if len(counts) > 1:
            growth = (counts[-1] / counts[0]) ** (1.0 / (len(counts) - 1))
            ests.append(counts[-1] * growth ** round(np.log2(n / big)))
        else:
            ests.append(counts[0])
        per_seed.append(counts)
    return per_seed, float(np.mean(ests)), three_d


_OW = None      # (operator, rhs) of an oracle worker process


def _oracle_worker(name, k, rounds, barrier, out):
    """One oracle process: build the workload (seed 1) and its operator, then
    time `rounds` bounded samples in step with the other workers: the
    Jacobi-PCG set-up alone (maxiter = 0) and the set-up plus k iterations."""
    from oracle import poisson as P
    p = make_problem(name, 1)
    op = P.operator_from_problem(p)
    barrier.wait()
    for _ in range(rounds):
        barrier.wait()
        t0 = time.perf_counter()
        P.solve_pcg_jacobi(op, p.f, rtol=0.0, maxiter=0)
        t1 = time.perf_counter()
        P.solve_pcg_jacobi(op, p.f, rtol=0.0, maxiter=k)
        t2 = time.perf_counter()
        out.put((t1 - t0, max((t2 - t1) - (t1 - t0), 1e-9) / k))


def oracle_time(name: str, k: int, procs: int, rounds: int) -> list:
    """`rounds` bounded samples of the oracle on `procs` concurrent processes
    (spawned, one problem each, single-threaded numpy): per round the
    slowest process's set-up time and time per iteration."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(procs), ctx.Queue()
    ws = [ctx.Process(target=_oracle_worker, args=(name, k, rounds, barrier, out)) for _ in range(procs)]
    for w in ws:
        w.start()
    res = []
    for _ in range(rounds):
        got = [out.get(timeout=3600) for _ in range(procs)]
        res.append((max(g[0] for g in got), max(g[1] for g in got)))
    for w in ws:
        w.join()
    return res


def oracle_report(name: str, k: int = 3, steps: int = 1, warmup: int = 0, legs: str = "single,all") -> dict:
    """Calibrate the oracle's iteration count (seeds 1-3), then time the
    workload's bounded sample on the legs asked for: "single" (one
    single-threaded process) and "all" (one process per host core at once,
    independent replicas).  Per step: the estimated time to tolerance =
    set-up + time per iteration x iterations."""
    per_seed, est_iters, extrapolated = oracle_calibrate(name)
    N = make_problem(name, 1).size if WORKLOADS[name]["kind"] != "batch" else 0
    out = dict(N=N, est_iters=est_iters, per_seed_counts=per_seed, extrapolated=extrapolated, k=k,
               host_cores=host_cores())
    want = legs.split(",")
    todo = ([("single", 1)] if "single" in want or host_cores() == 1 else []) + \
        ([("all", host_cores())] if "all" in want and host_cores() > 1 else [])
    for leg, procs in todo:
        r = oracle_time(name, k, procs, warmup + steps)[warmup:]
        est = [su + it * est_iters for su, it in r]
        out[leg] = dict(procs=procs, setup_s=[su for su, _ in r], per_iter_s=[it for _, it in r], est_time_s=est,
                        value=[procs * N / e / 1e9 for e in est])
    return out


def oracle_subprocess(call: str) -> dict:
    """Run an oracle timing in a child process with single-threaded numpy."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print('ORACLE_JSON', json.dumps(%s))" % (ROOT, call))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3600,
                       cwd=ROOT)
    for line in r.stdout.splitlines():
        if line.startswith("ORACLE_JSON"):
            return json.loads(line.split(" ", 1)[1])
    raise RuntimeError("oracle sample failed:\n" + r.stdout[-2000:] + r.stderr[-2000:])


def _leg_text(r: dict, leg: str, name: str) -> str:
    L = r[leg]
    return (f"{L['procs']} concurrent single-threaded process(es), each {r['k']} iterations of the FP64 oracle's "
            f"Jacobi-PCG on {name} seed 1 (median {statistics.median(L['per_iter_s']) * 1e3:.4g} ms/iteration + "
            f"{statistics.median(L['setup_s']) * 1e3:.4g} ms set-up)")


def cpu_block(r: dict, name: str) -> dict:
    """cpu_baseline: the all-cores leg (one replica per host core), with the
    single-thread leg beside it."""
    main = "all" if "all" in r else "single"
    est = ("extrapolated from downsized grids" if r["extrapolated"] else "measured at full size")
    counts = " ".join(str(c) for c in r["per_seed_counts"])
    blk = {"value": statistics.median(r[main]["value"]), "unit": UNIT, "cores": r[main]["procs"], "kind": "oracle",
           "host_cores": r["host_cores"],
           "sample": (f"{_leg_text(r, main, name)} x the oracle's iteration count to rtol, {est} "
                      f"(seeds 1-3: {counts} -> {r['est_iters']:.0f}); estimated time to tolerance "
                      f"{statistics.median(r[main]['est_time_s']):.4g} s per solve; value = replicas x cells / "
                      f"that time")}
    if main == "all" and "single" in r:
        blk["single_thread"] = {"value": statistics.median(r["single"]["value"]), "cores": 1,
                                "sample": _leg_text(r, "single", name),
                                "est_time_s": statistics.median(r["single"]["est_time_s"])}
    return blk


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if WORKLOADS[args.workload]["kind"] in ("fe3d", "gresho2d"):
        print(json.dumps({"impl": "reference", "unavailable": "the CPU arm times the cell-centred oracle's "
                          "Jacobi-PCG solve; this workload has no timed oracle arm"}), flush=True)
        return
    r = oracle_subprocess("bench.oracle_report(%r, %d, %d, %d, 'all')" % (args.workload, args.oracle_iters,
                                                                            args.steps, args.warmup))
    leg = r["all"] if "all" in r else r["single"]
    est = statistics.median(leg["est_time_s"])
    value = statistics.median(leg["value"])
    cpu = cpu_block(r, args.workload)
    cpu["sample"] = f"per step: {cpu['sample']}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": est * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload]["desc"], "cells": r["N"]},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def fp64_roof(t_s: float, N: int, bytes_per_cell: int, fp64_ops_per_cell: int, hbm_gbs: float,
              fp64_per_s: float, note: str) -> dict:
    """A float64 kernel against its roof min(HBM, float64 issue): the time
    it would take at each bound, the larger of the two (the roof), and the
    fraction of that roof the measured time reaches."""
    t_hbm = bytes_per_cell * N / (hbm_gbs * 1e9)
    out = {"launch_us": t_s * 1e6, "bytes_per_cell": bytes_per_cell, "hbm_bound_us": t_hbm * 1e6,
           "hbm_frac": t_hbm / t_s, "note": note}
    if fp64_ops_per_cell is None:
        # an op count the source does not fix (library reciprocals): the
        # float64 operations a cell the measured time corresponds to
        out["fp64_ops_per_cell_implied"] = t_s * fp64_per_s / N
        return out
    t_fp64 = fp64_ops_per_cell * N / fp64_per_s
    roof = max(t_hbm, t_fp64)
    out.update({"fp64_ops_per_cell": fp64_ops_per_cell, "fp64_bound_us": t_fp64 * 1e6,
                "bound": "fp64" if t_fp64 >= t_hbm else "hbm", "frac_of_roof": roof / t_s})
    return out


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
        # every grid's coefficient assembly in one launch, then the right-hand sides
        lm.batch_set_coefficients(grids, [t[0] for t in tens], [t[1] for t in tens], [t[2] for t in tens],
                                  [p.dt for p in probs], stream)
        for g, t in zip(grids, tens):
            g.set_rhs(t[3], stream)

    def step():
        load()
        return lm.batch_solve(grids, rtol=1e-8, stream=stream, nu1=1, nu2=2, inner_rtol=1e-2)

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
    if args.only_steps:                 # profiling runs: the timed batches and nothing else
        print(json.dumps({"only_steps": True, "ms_per_batch": t_step * 1e3,
                          "gpu_launches_per_batch": launches / args.steps}), flush=True)
        for g in grids:
            g.close()
        return

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
    # the learned workload cycles through 8 held-out problems, the convection
    # workloads through seeds 1-3; the two-component recipe has one seed (7)
    nprob = {"train2d": 8, "conv3d": 3, "plain2d": 3}.get(kind, 1)
    probs = [make_problem(args.workload, seed=1 + k) for k in range(nprob)]
    p = probs[0]
    N = p.size
    dev_in = [[torch.as_tensor(a.ravel(), device=dev) for a in (q.rho_old, q.rho_new, q.cs2, q.f)] for q in probs]
    g = lm.Grid.for_problem(p)
    if mode == "learned":
        g.load_network(WEIGHTS)
    solve_kw = dict(mode=mode, rtol=p.rtol, max_iter=args.max_iter)
    if args.host_checks:
        solve_kw["check_every"] = 1
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
    # the float64 roof: this GPU's measured float64 FMA rate (lm_probe_rate),
    # and the float64 kernels against min(HBM, float64 issue)
    fp64_rate = lm.probe_rate(0, 20000, stream)
    fp32_rate = lm.probe_rate(1, 200000, stream)
    ro0, rn0, c20, _ = dev_in[0]
    t_asm = time_kernel(torch, lambda: g.set_coefficients(ro0, rn0, c20, probs[0].dt, stream), 5, stream)
    jac_iters = max(base["jacobi"]["iters"], 1)
    t_jac_iter = base["jacobi"]["time_to_tol_ms"] * 1e-3 / jac_iters
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
        cpu = cpu_block(oracle_subprocess("bench.oracle_report(%r, %d)" % (args.workload, args.oracle_iters)),
                        args.workload)

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
                                  "k_apply64": fp64_roof(t_k64, N, 48, 14, peak, fp64_rate,
                                                         "y = A x and x.(A x): 13 float64 operations a cell "
                                                         "for the stencil, 1 for the dot"),
                                  "k_assemble": fp64_roof(t_asm, N, 72, None, peak, fp64_rate,
                                                          "c~ and three faces: 14 float64 operations and 4 "
                                                          "correctly rounded float64 reciprocals a cell; timed "
                                                          "through lm_set_coefficients (includes its host sync)"),
                                  "fp64_jacobi_pcg_iteration": fp64_roof(
                                      t_jac_iter, N, 120, 21, peak, fp64_rate,
                                      "apply + p.q (14 ops), x/r update with r.r and r.z (5), p update (2); "
                                      "three launches, 120 B a cell")}},
            "fp64_peak": {"fma_per_s": fp64_rate, "tflops": 2 * fp64_rate / 1e12,
                          "fp32_fma_per_s": fp32_rate, "ratio_fp32_to_fp64": fp32_rate / fp64_rate,
                          "source": "lm_probe_rate: 8 independent FMA chains a thread, 8 blocks of 256 threads "
                                    "per SM, CUDA events (of measured)"},
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


def run_fe(args):
    """The operator in Q1 finite elements on 256^3 points: one step = the
    coefficients from the state (lm_fe_set_state), the load vector V f
    (lm_fe_mass_times) and the mixed solve (lm_fe_solve) to 1e-8."""
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
    n = WORKLOADS[args.workload]["n"]
    probs = [make_problem(args.workload, seed=1 + k) for k in range(3)]
    p = probs[0]
    N = p.size
    h = (1.0 / (n - 1),) * 3              # cubic elements; the walled z axis spans [0, 1]
    g = lm.FEGrid(p.n, h, p.bc)
    dev_in = [[torch.as_tensor(a.ravel(), device=dev) for a in (q.rho_old, q.rho_new, q.cs2, q.f)] for q in probs]
    b = torch.empty(N, dtype=torch.float64, device=dev)
    x = torch.zeros(N, dtype=torch.float64, device=dev)

    def step(k, mode="mixed"):
        ro, rn, c2, f = dev_in[k % len(probs)]
        g.set_state(ro, rn, c2, probs[k % len(probs)].dt, stream)
        g.mass_times(f, b, stream)
        return g.solve(b, x, mode=mode, rtol=p.rtol, stream=stream, max_iter=args.max_iter,
                       allow=(0,) if mode == "mixed" else (0, -3))

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
        ev[k][0].record(stream)
        results.append(step(k))
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = lm.kernel_launches() - launches0
    barrier()
    clk = clocks.stop()
    elapsed = job_time(sum(a.elapsed_time(c) for a, c in ev) * 1e-3, world, dev)
    assert all(r["status"] == 0 and r["rel_residual"] <= p.rtol for r in results), results
    res = results[-1]
    t_solve = elapsed / args.steps

    # end to end: pinned host inputs copied in and the solution copied out inside the timed region
    host = [[torch.from_numpy(np.ascontiguousarray(a.ravel())).pin_memory() for a in (q.rho_old, q.rho_new,
                                                                                      q.cs2, q.f)]
            for q in probs]
    xout = torch.empty(N, dtype=torch.float64).pin_memory()

    def e2e_step(k):
        for d, hsrc in zip(dev_in[k % len(probs)], host[k % len(probs)]):
            d.copy_(hsrc, non_blocking=True)
        r = step(k)
        xout.copy_(x, non_blocking=True)
        return r

    e2e_step(0)
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        e2e_step(k)
    torch.cuda.synchronize()
    e2e_t = job_time(time.perf_counter() - t0, world, dev)

    # the float64 Jacobi-PCG on the same system
    torch.cuda.synchronize()
    b0 = time.perf_counter()
    rj = step(0, mode="jacobi")
    torch.cuda.synchronize()
    t_jac = time.perf_counter() - b0

    # roofline of the float32 finite-element apply (k_fe3_32), timed alone
    x32 = torch.randn(N, dtype=torch.float32, device=dev)
    y32 = torch.empty_like(x32)
    reps = 20
    t_ap = time_kernel(torch, lambda: g.apply(x32, y32, prec=lm.PREC_FP32, stream=stream), reps, stream)
    x64 = torch.randn(N, dtype=torch.float64, device=dev)
    y64 = torch.empty_like(x64)
    t_ap64 = time_kernel(torch, lambda: g.apply(x64, y64, prec=lm.PREC_FP64, stream=stream), reps, stream)
    fp64_rate = lm.probe_rate(0, 20000, stream)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    ap_bytes = 16                         # read x, kappa_e, V c~; write y (float32)
    achieved = ap_bytes * N / t_ap / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": job_value(N, args.steps, world, elapsed), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_solve * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (float32 flexible CG, float64 residual/refinement)", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "points": N, "mode": "mixed",
                       "problems": len(probs), "rtol": p.rtol, "l2": "inputs exceed L2 (4 x %.0f MB)" % (N * 8 / 1e6),
                       "parallelism": f"replicas x{world}"},
            "time_to_tol_ms": t_solve * 1e3,
            "solve": {"iters": res["iters"], "outer_iters": res["outer_iters"], "vcycles": res["vcycles"],
                      "rel_residual": res["rel_residual"]},
            "fp64_jacobi_pcg": {"time_to_tol_ms": t_jac * 1e3, "iters": rj["iters"], "status": rj["status"],
                                "rel_residual": rj["rel_residual"]},
            "speedup_vs_fp64_pcg": t_jac / t_solve,
            "e2e": {"value": job_value(N, args.steps, world, e2e_t), "unit": UNIT,
                    "h2d_bytes_per_step": 4 * 8 * N, "d2h_bytes_per_step": 8 * N},
            "roofline": {"kernel": "k_fe3_32 (float32 Q1 finite-element apply, row f1)", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "bytes_per_point": ap_bytes, "launch_us": t_ap * 1e6,
                         "peak_source": ("MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks
                                         else "fallback 6800 GB/s (of fallback)"),
                         "also": {"k_fe_apply64": fp64_roof(t_ap64, N, 32, 60, peak, fp64_rate,
                                                            "y = B x in float64 on cubic elements: 20 "
                                                            "neighbours, about 60 float64 operations a point")}},
            "cpu_baseline": None,
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


def run_gresho(args):
    """Time stepping of the Gresho vortex: W warm-up steps, then K timed
    fractional steps of the resident state (CUDA events around each step on
    the launching stream; every step ends with the solve's host check)."""
    import torch

    from paper_1112_3507_gb300 import inputs as I
    from paper_1112_3507_gb300 import lowmach as lm
    from paper_1112_3507_gb300.fractional import FractionalStep

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = WORKLOADS[args.workload]["n"]
    g = I.gresho_vortex(n, 0.01, cfl=0.5 * args.dt_factor)
    N = n * n
    fs = FractionalStep(g["n"], g["h"], g["bc"], g["gamma"], rtol=1e-11)
    fs.set_state(g["rho"], g["mom"], g["e"], stream)

    def ke():
        m = fs.mom.view(3, N)
        return float(((m * m).sum(0) / fs.rho).sum()) * 0.5 * g["h"][0] * g["h"][2]

    ke0 = ke()
    for _ in range(args.warmup):
        fs.step(g["dt"], stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = lm.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters = []
    for k in range(args.steps):
        ev[k][0].record(stream)
        iters.append(fs.step(g["dt"], stream)["iters"])
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = lm.kernel_launches() - launches0
    clk = clocks.stop()
    t_step = sum(a.elapsed_time(b) for a, b in ev) * 1e-3 / args.steps
    ke1 = ke()

    # phases of one step, each timed alone on the stream
    dt = g["dt"]
    ph = {
        "advect": lambda: lm.advect(fs.n, fs.h, fs.bc, dt, fs.rho, fs.mom, fs.e, fs.rho1, fs.mom_s, fs.e_s,
                                    stream=stream),
        "projection_rhs": lambda: lm.projection_rhs(fs.n, fs.h, fs.bc, dt, fs.p, fs.rho, fs.cs2, fs.mom, fs.mom_s,
                                                    fs.rho1, fs.f, fs.uf_s, stream=stream),
        "coefficients": lambda: fs.grid.set_coefficients(fs.rho, fs.rho1, fs.cs2, dt, stream),
        "projection_update": lambda: lm.projection_update(fs.n, fs.h, fs.bc, dt, fs.p, fs.rho1, fs.mom_s,
                                                          fs.uf_s, fs.e_s, fs.mom1, fs.uf1, fs.e1, stream=stream),
        "eos": lambda: lm.eos_ideal(fs.gamma, fs.rho1, fs.mom1, fs.e1, fs.p_pred, None, stream=stream),
    }
    phases = {k: time_kernel(torch, f, 10, stream) * 1e6 for k, f in ph.items()}
    phases["solve_and_rest"] = t_step * 1e6 - sum(phases.values())

    # the same steps with the float64 Jacobi-PCG solve
    fj = FractionalStep(g["n"], g["h"], g["bc"], g["gamma"], mode="jacobi", rtol=1e-11)
    fj.set_state(g["rho"], g["mom"], g["e"], stream)
    fj.step(g["dt"], stream)
    torch.cuda.synchronize()
    j0 = time.perf_counter()
    jit = [fj.step(g["dt"], stream)["iters"] for _ in range(5)]
    torch.cuda.synchronize()
    t_jac = (time.perf_counter() - j0) / 5
    fj.close()

    # end to end: host initial state in, K steps, final state out
    host = [torch.from_numpy(np.ascontiguousarray(a.ravel())).pin_memory()
            for a in (g["rho"], np.concatenate([m.ravel() for m in g["mom"]]), g["e"])]
    outs = [torch.empty(N, dtype=torch.float64).pin_memory(), torch.empty(3 * N, dtype=torch.float64).pin_memory(),
            torch.empty(N, dtype=torch.float64).pin_memory(), torch.empty(N, dtype=torch.float64).pin_memory()]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fs.rho.copy_(host[0], non_blocking=True)
    fs.mom.copy_(host[1], non_blocking=True)
    fs.e.copy_(host[2], non_blocking=True)
    lm.eos_ideal(fs.gamma, fs.rho, fs.mom, fs.e, fs.p, fs.cs2, stream=stream)
    for _ in range(args.steps):
        fs.step(g["dt"], stream)
    for o, d in zip(outs, (fs.rho, fs.mom, fs.e, fs.p)):
        o.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    e2e_t = (time.perf_counter() - t0) / args.steps

    fp64_rate = lm.probe_rate(0, 20000, stream)
    adv_ops = 230                 # float64 operations a 2D cell in k_advect (two axes, five quantities)
    line = {
        "metric": METRIC, "value": N / t_step / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 step, f32+f64 solve", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "cells": N, "dt": g["dt"], "ma": 0.01,
                   "dt_factor": args.dt_factor,
                   "l2": "state resident in L2 (5 x %.1f MB)" % (N * 8 / 1e6)},
        "solve_iters_per_step": float(np.mean(iters)), "kinetic_energy_ratio": ke1 / ke0,
        "phases_us": phases,
        "fp64_jacobi_pcg_step_ms": t_jac * 1e3, "fp64_jacobi_iters_per_step": float(np.mean(jit)),
        "speedup_vs_fp64_pcg": t_jac / t_step,
        "e2e": {"value": N / e2e_t / 1e9, "unit": UNIT, "h2d_bytes_per_step": 5 * 8 * N / args.steps,
                "d2h_bytes_per_step": 6 * 8 * N / args.steps},
        "roofline": {"kernel": "k_advect (float64 MUSCL advection, steps (i)-(iii))", "bound": "alu",
                     "achieved": adv_ops * N / (phases["advect"] * 1e-6) / 1e12,
                     "peak": fp64_rate / 1e12, "unit": "T float64 op/s",
                     "frac": adv_ops * N / (phases["advect"] * 1e-6) / fp64_rate, "traffic": None,
                     "peak_source": "lm_probe_rate float64 FMA/s, one operation an FMA (of measured)"},
        "cpu_baseline": None, "clocks": clk, "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)
    fs.close()


def run_kernel(args):
    """A few launches of one kernel, nothing else: the command the ncu captures
    of the sweep, the float32 apply and the network are taken on."""
    import torch

    from paper_1112_3507_gb300 import lowmach as lm
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    if args.kernel == "net":
        net = lm.Net.load(WEIGHTS)
        B, H, W = 16, 256, 256
        x = torch.randn(B * H * W * 3, device="cuda")
        y = torch.empty(B * H * W, device="cuda")
        for _ in range(3):
            net.forward(x, y, B, H, W)
        torch.cuda.synchronize()
        net.close()
    elif args.kernel == "fe32":
        p = make_problem("fe256", 1)
        n = WORKLOADS["fe256"]["n"]
        g = lm.FEGrid(p.n, (1.0 / (n - 1),) * 3, p.bc)
        g.set_state(p.rho_old, p.rho_new, p.cs2, p.dt)
        x = torch.randn(p.size, dtype=torch.float32, device="cuda")
        y = torch.empty_like(x)
        for _ in range(4):
            g.apply(x, y, prec=lm.PREC_FP32, stream=stream)
        torch.cuda.synchronize()
        g.close()
    else:
        if WORKLOADS[args.workload]["kind"] == "batch":
            raise SystemExit("--kernel runs on a single-grid workload")
        if args.kernel == "sweep512":
            from paper_1112_3507_gb300 import inputs as I
            p = I.make_problem(512, 64, 512, ma=0.01, contrast=20.0, noise=0.01, seed=1)
        elif args.kernel == "ops2d":
            from paper_1112_3507_gb300 import inputs as I
            p = I.make_problem(4096, 4096, ma=0.01, contrast=15.0, noise=0.01, seed=3)
        else:
            p = make_problem(args.workload, 1)
        g = lm.Grid.for_problem(p)
        g.set_problem(p)
        x = torch.randn(p.size, dtype=torch.float32, device="cuda")
        f = torch.randn_like(x)
        y = torch.empty_like(x)
        for _ in range(4):
            if args.kernel in ("sweep", "sweep512", "ops2d"):
                g.mg_sweep(x, f, y, 0, stream=stream)
            if args.kernel in ("apply32", "ops2d"):
                g.apply(x, y, prec=lm.PREC_FP32, stream=stream)
        torch.cuda.synchronize()
        g.close()
    print(json.dumps({"kernel": args.kernel, "workload": args.workload, "status": "ok"}), flush=True)


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
    ap.add_argument("--host-checks", action="store_true",
                    help="single-grid solves check the inner residual on the host after every iteration "
                         "(check_every = 1: one graph launch per iteration instead of the device-side loop), "
                         "so that ncu can time each kernel; for launch lists, not for timing")
    ap.add_argument("--only-steps", action="store_true",
                    help="run warm-up and timed solves only (for profiler launch lists)")
    ap.add_argument("--dt-factor", type=float, default=1.0,
                    help="gresho256: the time step as a multiple of the sound-speed-induced one (CFL 0.5)")
    ap.add_argument("--kernel", choices=["sweep", "sweep512", "apply32", "ops2d", "net", "fe32"], default=None,
                    help="profiling runs: a few launches of one kernel on the workload's finest grid "
                         "(sweep: lm_mg_sweep, apply32: lm_apply in float32; sweep512: lm_mg_sweep on a "
                         "512 x 512 x 64 grid of the convection recipe, 512-cell rows; ops2d: lm_mg_sweep and "
                         "float32 lm_apply on a 4096^2 2D grid; net: U-Net forward on "
                         "16 images of 256^2; fe32: lm_fe_apply in float32 on the fe256 points), then exit")
    args = ap.parse_args()
    if args.kernel:
        run_kernel(args)
    elif args.impl == "reference":
        run_reference(args)
    elif WORKLOADS[args.workload]["kind"] == "batch":
        run_batch(args)
    elif WORKLOADS[args.workload]["kind"] == "fe3d":
        run_fe(args)
    elif WORKLOADS[args.workload]["kind"] == "gresho2d":
        run_gresho(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
