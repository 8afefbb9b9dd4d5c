"""Multi-process host logic of bench.py with world size 2 on gloo (CPU): the
views are dealt to ranks without overlap and the timing reduction takes the
slowest rank."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        slowest = bench._max_over_ranks(dist, 1.5 + rank)
        total = bench._sum_over_ranks(dist, 10.0 * (rank + 1))
        views = [bench.view_of(i, rank, world, 8) for i in range(4)]
        bench._barrier(dist)
        q.put((rank, slowest, total, views))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_views_and_time_by_the_slowest():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]
    assert [r[2] for r in res] == [30.0, 30.0]
    v0, v1 = res[0][3], res[1][3]
    assert set(v0).isdisjoint(v1) and sorted(v0 + v1) == list(range(8))
