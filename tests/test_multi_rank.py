"""The N>1 bench path on CPU: two gloo ranks.  Envs are independent, so
ranks shard them with no data-path collective; the only collective is the
max of the per-rank timed region, and the job rate is all ranks' units over
the slowest rank's time (weak scaling)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seeds = bench.env_seeds(4, rank)
        elapsed = [1.5, 2.5][rank]
        slowest = bench.max_over_ranks(elapsed, world, "cpu")
        rate = bench.job_rate(4 * 10, world, slowest)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        out.put((rank, slowest, rate, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate, gathered in res:
        assert slowest == 2.5  # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 40 / 2.5)
        # the ranks' envs are disjoint (no env is simulated twice)
        assert not set(gathered[0]) & set(gathered[1])


def test_single_rank_defaults():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.job_rate(8, 1, 2.0) == 4.0
    assert bench.env_seeds(3, 0) == [0, 1, 2]
