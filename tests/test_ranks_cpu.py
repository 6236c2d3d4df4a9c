"""The benchmark's multi-rank logic on CPU (gloo, world size 2): every rank
renders its own batch, the job's time is the slowest rank's, and the job's
throughput counts every rank's views (weak scaling, no collective on the data
path)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        ms = [12.5, 17.25][rank]                     # rank 1 is the slow one
        slow = bench.max_over_ranks(ms, dist, "cpu")
        out[rank] = (slow, bench.job_rate(8 * 50, world, slow))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_views():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slow, rate = res[0]
    assert slow == 17.25
    assert rate == pytest.approx(world * 8 * 50 / (17.25 / 1e3))


def test_single_rank_is_unchanged():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_rate(8, 1, 1000.0) == pytest.approx(8.0)
