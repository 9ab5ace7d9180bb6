"""The multi-rank path of bench.py on CPU: world size 2 over gloo.

The solve does not shard (one image per solve), so N GPUs run N replicas; the
whole-job rate is the units all ranks processed over the slowest rank's time.
These tests run that aggregation and the reference arm's rank handling as
real processes, without a GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    local_ms = 10.0 * (rank + 1)          # rank 1 is the slow one
    ms, rate = bench.job_rate(local_ms, 1000.0, world, "cpu")
    q.put((rank, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_and_all_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == pytest.approx(20.0)                  # max over ranks
        assert rate == pytest.approx(2 * 1000.0 / 0.020)  # units of both ranks / slowest time


def test_job_rate_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, rate = bench.job_rate(4.0, 8.0, 1, "cpu")
    assert ms == 4.0 and rate == pytest.approx(2000.0)


def test_reference_arm_under_torchrun_prints_once():
    """Two ranks launched like the multi-GPU bench: rank 0 alone times the
    oracle and prints one JSON line; rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
           "--workload", "two_disks_128"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
