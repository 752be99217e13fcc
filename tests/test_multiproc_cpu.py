"""The multi-process path of bench.py on CPU (gloo, world size 2): every rank
solves its own replica, the job is timed by the slowest rank and counts the
targets of all ranks.  No GPU and no collective on the data path."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        worst = bench.max_over_ranks(times[rank], dist)
        out[rank] = (worst, bench.job_rate(1000, 3, world, worst))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(120.0, 80.0), (50.0, 50.0), (10.0, 400.0)])
def test_slowest_rank_times_the_job(times):
    world = 2
    manager = mp.get_context("spawn").Manager()   # no fork of a threaded process
    out = manager.dict()
    mp.spawn(_rank, args=(world, _free_port(), list(times), out), nprocs=world, join=True)
    worst = max(times)
    for r in range(world):
        assert out[r][0] == worst
        assert out[r][1] == pytest.approx(1000 * 3 * world / (worst / 1000.0))


def test_single_process_is_unchanged():
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.job_rate(10, 2, 1, 1000.0) == pytest.approx(20.0)


def test_reference_arm_under_torchrun_prints_one_line():
    """`bench.py --impl reference` launched as two ranks (the launch used for
    N > 1): rank 0 alone times the oracle and prints; the other rank exits 0
    without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
