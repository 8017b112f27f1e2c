"""Host logic of bench.py's multi-rank launch on CPU ranks (gloo, world size 2).

Several GPUs run independent replicas of the particle move (the move shards by
particle with no exchange inside the timed region), so the multi-rank logic is
the timing reduction (the job lasts as long as its slowest rank), the
whole-job rate, and the reference arm (rank 0 alone works, the others exit 0).
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank           # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, world, "cpu")
        rate = bench.whole_job_rate(4096, world, ms_max)
        out.put((rank, ms_max, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_world2():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(world))
    for rank, ms_max, rate in res:
        assert ms_max == 150.0
        assert rate == pytest.approx(2 * 4096 / 0.150)


def test_rate_single_rank():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_rate(100, 1, 1000.0) == pytest.approx(100.0)


def test_reference_arm_two_ranks_prints_once():
    """torchrun with two CPU ranks: rank 0 times the oracle and prints one JSON line, rank 1 exits 0."""
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-seconds", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["n_gpus"] == 2
    assert line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle"
