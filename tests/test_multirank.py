"""Multi-process paths on the CPU (gloo, world size 2).

The single-problem path does not shard (the triangular-solve dependencies
cross every row partition), so `bench.py --gpus N` runs N independent
replicas: each rank times its own iterations, the job's time is the slowest
rank's, and the job's rate counts every rank's iterations.  These tests run
that aggregation over two gloo ranks.
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
