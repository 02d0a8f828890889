"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks.

Every rank runs its own replica (independent problems, no data-path
collective); the only exchange is the max over ranks of the timed region,
and rank 0 reports the whole-job throughput over the slowest rank.
"""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        local_t = 2.0 + rank          # rank 1 is the slower replica
        t_max = bench.reduce_max(local_t, ws, "cpu")
        v = bench.job_tflops(ws, 1.0e12, 4, t_max)
        faults = bench.reduce_sum(float(10 + rank), ws, "cpu")   # fault counts add over ranks
        q.put((rank, ws, r, local, t_max, v, faults))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_max_timing():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ws, r, local, t_max, v, faults in res:
        assert ws == 2 and r == rank and local == rank
        assert t_max == 3.0                      # max over ranks
        assert v == pytest.approx(2 * 1.0e12 * 4 / 3.0 / 1e12)
        assert faults == 21.0                    # 10 + 11, on every rank


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: called.append(1))

    class A:
        steps, warmup = 1, 3
    assert bench.reference_arm(A()) is None
    assert not called


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the CPU oracle timed on a row sample of the
    bench workload) prints one JSON line with the keys the benchmark contract
    names, on the same metric and configuration as the library's arm."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["config"] == bench.main_config()
    for k in ("value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["warmup"] >= 3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
