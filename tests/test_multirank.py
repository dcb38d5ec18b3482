"""Multi-process paths on the CPU (gloo, world size 2).

The single-problem path does not shard (the triangular-solve dependencies
cross every row partition), so `bench.py --gpus N` runs N independent
replicas: each rank times its own iterations, the job's time is the slowest
rank's, and the job's rate counts every rank's iterations.  The batched form
shards its independent problems over the ranks (no collective on the data
path) and sums their iterations.  These tests run that sharding and
aggregation over two gloo ranks.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 150.0][rank]  # the second rank is slower
        total = bench.max_over_ranks(local_ms, dist)
        rate = bench.whole_job_rate(50, world, total)
        q.put((rank, total, rate))
    finally:
        dist.destroy_process_group()


def test_replicas_max_over_ranks_and_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, total, rate in got:
        assert total == 150.0  # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 50 / 0.150)  # 100 iterations in 150 ms


def test_single_process_aggregation():
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.whole_job_rate(10, 1, 20.0) == pytest.approx(500.0)


def _shard_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.shard(list(range(11)), rank, world)
        its = bench.sum_over_ranks(10 * len(mine) + rank, dist)  # iterations of this rank's problems
        slowest = bench.max_over_ranks([2.0, 3.0][rank], dist)
        q.put((rank, mine, its, slowest))
    finally:
        dist.destroy_process_group()


def test_batched_problems_shard_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    # every problem on exactly one rank, the shares within one of each other
    assert sorted(got[0][1] + got[1][1]) == list(range(11))
    assert abs(len(got[0][1]) - len(got[1][1])) <= 1
    for _, _, its, slowest in got:
        assert its == 10 * 11 + 0 + 1 and slowest == 3.0


def test_single_process_shard_is_everything():
    assert bench.shard(list(range(5)), 0, 1) == list(range(5))
    assert bench.sum_over_ranks(7.0, None) == 7.0
