"""Multi-process paths on the CPU (gloo, world size 2).

The single-problem path does not shard (the triangular-solve dependencies
cross every row partition), so `bench.py --gpus N` runs N independent
replicas: each rank times its own iterations, the job's time is the slowest
rank's, and the job's rate counts every rank's iterations.  The batched form
shards its independent problems over the ranks (no collective on the data
path) and sums their iterations.  These tests run that sharding and
aggregation over two gloo ranks, and the served form's routing of requests
by matrix id to one server per rank.
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


# ---------------------------------------------------------------------------
# served form: requests routed by matrix id, one server per rank
# ---------------------------------------------------------------------------
def _served_rank_main(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist

    from paper_2603_28642_gb300 import serving, synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # weights: nonzeros of the 64 matrices of the serving recipe (6 per row, m = 1.5 n)
        weights = np.array([9 * p.n for p in synth.serving_matrices(64, n_hi=2000)])
        owner = serving.owners(weights, world)
        which = np.random.default_rng(100).integers(0, 64, size=500)
        mine = serving.requests_for(which, owner, rank)
        # stand-in latencies: a rank's own requests, 1 ms per request id
        lat = [float(r) for r in mine]
        tables = serving.gather(owner.tolist(), dist)
        served = serving.gather(mine.tolist(), dist)
        merged = serving.merge_latencies(serving.gather(lat, dist))
        q.put((rank, tables, served, merged, weights.tolist(), which.tolist()))
    finally:
        dist.destroy_process_group()


def test_served_routing_by_matrix_id_two_ranks():
    import numpy as np

    from paper_2603_28642_gb300 import serving

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_served_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted((q.get(timeout=5) for _ in range(2)), key=lambda t: t[0])
    tables = got[0][1]
    weights = np.asarray(got[0][4])
    which = np.asarray(got[0][5])
    # every rank computed the same owner table; every matrix has one owner
    assert got[0][1] == got[1][1] and tables[0] == tables[1]
    owner = np.asarray(tables[0])
    assert set(owner.tolist()) == {0, 1}
    # balanced: the heavier rank carries at most the lighter one plus the largest matrix
    load = [weights[owner == r].sum() for r in range(2)]
    assert abs(load[0] - load[1]) <= weights.max()
    # each request is served by exactly one rank, the owner of its matrix
    served = got[0][2]
    assert sorted(served[0] + served[1]) == list(range(len(which)))
    for r in range(2):
        assert all(owner[which[i]] == r for i in served[r])
    # merged percentiles = percentiles of all requests together
    allv = np.sort(np.arange(len(which), dtype=np.float64))
    for _, _, _, merged, _, _ in got:
        assert merged["requests"] == len(which)
        assert merged["p50_ms"] == serving.percentile(allv, 0.5)
        assert merged["p99_ms"] == serving.percentile(allv, 0.99)
        assert merged["mean_ms"] == pytest.approx(allv.mean())


def test_served_routing_single_rank_and_ties():
    import numpy as np

    from paper_2603_28642_gb300 import serving

    assert serving.owners([5, 5, 5], 1).tolist() == [0, 0, 0]
    # equal weights: the lower matrix id goes first, to the lower rank
    assert serving.owners([1, 1, 1, 1], 2).tolist() == [0, 1, 0, 1]
    assert serving.owners([10, 1, 1], 2).tolist() == [0, 1, 1]
    which = np.array([2, 0, 1, 2])
    assert serving.requests_for(which, np.array([0, 1, 1]), 1).tolist() == [0, 2, 3]
    assert serving.percentile([], 0.5) == 0.0
    assert serving.merge_latencies([[3.0], [1.0, 2.0]])["p50_ms"] == 2.0
