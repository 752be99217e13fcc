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
