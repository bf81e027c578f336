"""The benchmark's multi-rank aggregation on CPU ranks (gloo, world size 2): every rank learns the
slowest rank's step time, and the job value counts every rank's frames over that time.  The data
path itself has no collective (each rank analyses its own sequence: replicas)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, frames, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], dist, "cpu")
        out[rank] = (ms, bench.job_value(world, frames, ms))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    world, frames = 2, 4000
    times = [531.0, 560.5]  # per-rank ms per step
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, times, frames, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == max(times)
        assert value == pytest.approx(world * frames / (max(times) / 1000.0))


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 4000, 500.0) == pytest.approx(8000.0)
