"""The N > 1 path of bench.py, on CPU with two gloo ranks.

Every rank runs its own replica of the workload (the step does not shard: one problem per
pool, weak scaling, no collective on the data path); the job's time is the slowest rank's,
the job's value counts every rank's cells, and only rank 0 prints.
"""

from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_local = 10.0 + 3.0 * rank                      # the ranks finish at different times
        ms = bench.max_over_ranks(ms_local, dist, device="cpu")
        value = bench.job_value(world, 1000, 5, ms)
        q.put((rank, ms, value, bench.prints_line(rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(world))
    for rank, ms, value, prints in got:
        assert ms == 13.0                                 # max over ranks
        assert value == pytest.approx(world * 1000 * 5 / 13e-3)
        assert prints == (rank == 0)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(7.5, None) == 7.5
    assert bench.job_value(1, 100, 4, 2.0) == pytest.approx(100 * 4 / 2e-3)
