"""The multi-rank host logic of bench.py on CPU: gloo ranks, world size 2.

Each rank solves its own system (the path partitions by right-hand side), so
the only cross-rank traffic is the barrier and the timing reduction:
whole-job throughput = units of all ranks / slowest rank's time.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = 100.0 * (rank + 1)          # rank 0: 100 units in 1 s, rank 1: 200 units in 4 s
    ms = 1000.0 * (1 + 3 * rank)
    bench.barrier(dist)
    v = bench.aggregate_rate(units, ms, dist)
    m = bench.max_over_ranks(ms, dist)
    q.put((rank, v, m))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29611
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, m in out:
        assert m == 4000.0
        assert v == pytest.approx(300.0 / 4.0)


def test_reference_arm_under_torchrun_two_ranks():
    """--impl reference under torchrun: rank 0 prints one JSON line, rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=29612", os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "1", "--grid", "12", "--k", "4"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
