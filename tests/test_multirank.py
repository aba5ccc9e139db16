"""The N>1 path of bench.py on CPU: ranks are independent replicas whose
only exchange is the max-over-ranks of their elapsed time (gloo, world 2)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        elapsed = 1.0 + rank                          # rank 1 is the slow one
        t = bench.job_time(elapsed, world, device="cpu")
        v = bench.job_value(1000, 10, world, t)
        out.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_job_time_is_max_over_ranks_and_value_counts_all_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [t for _, t, _ in got] == [2.0, 2.0]
    # 2 replicas x 1000 cells x 10 steps in 2 s
    assert all(v == pytest.approx(2 * 1000 * 10 / 2.0 / 1e9) for _, _, v in got)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time(3.5, 1) == 3.5
    assert bench.job_value(10, 2, 1, 4.0) == pytest.approx(5e-9)


def test_reference_arm_does_no_work_off_rank_0(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        workload, warmup, steps, oracle_iters, gpus = "plain64", 0, 1, 1, 2
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""


def bench_host_cores():
    sys.path.insert(0, ROOT)
    import bench
    return bench.host_cores()


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the CPU oracle and prints one JSON line
    with the GPU arm's metric and unit (run on the smallest workload)."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "plain64", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, RANK="0"))
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GDOF/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] == line["cpu_baseline"]["host_cores"] == bench_host_cores()
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["steps"] == 2
