"""The served form on several GPUs: one server per rank, requests routed by
matrix id.

Every rank owns whole matrices: A, its factors and the Krylov state of the
requests for it live on that rank's GPU, and a request (a new right-hand side
for a resident matrix) goes to the rank that owns its matrix.  The data path
has no collective; the ranks only exchange their requests' latencies at the
end, to report one p50/p99 for the whole job.

Everything here is host logic over plain lists and arrays, the same on every
rank (each rank computes the whole routing table from the seeded workload
and keeps its own part), so it is tested with gloo ranks on the CPU.
"""
from __future__ import annotations

import heapq

import numpy as np


def owners(weights, world: int) -> np.ndarray:
    """Owner rank of each matrix: matrices in decreasing weight (ties: lower
    id first) go to the rank with the least weight so far (ties: lower rank).
    Deterministic, so every rank computes the same table."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = np.asarray(weights, dtype=np.float64)
    order = sorted(range(len(w)), key=lambda k: (-w[k], k))
    heap = [(0.0, r) for r in range(world)]
    out = np.empty(len(w), dtype=np.int64)
    for k in order:
        load, r = heapq.heappop(heap)
        out[k] = r
        heapq.heappush(heap, (load + float(w[k]), r))
    return out


def requests_for(which, owner, rank: int) -> np.ndarray:
    """Indices (ascending) of the requests rank `rank` serves: those whose
    matrix it owns.  `which[r]` is request r's matrix id."""
    which = np.asarray(which, dtype=np.int64)
    return np.nonzero(np.asarray(owner)[which] == rank)[0]


def percentile(sorted_ms, q: float) -> float:
    """The server's percentile rule: the element at round(q (n - 1)) of the
    sorted latencies."""
    n = len(sorted_ms)
    if n == 0:
        return 0.0
    i = min(n - 1, int(np.floor(q * (n - 1) + 0.5)))
    return float(sorted_ms[i])


def merge_latencies(per_rank) -> dict:
    """p50 / p99 / mean over every rank's request latencies (ms)."""
    allv = np.sort(np.concatenate([np.asarray(v, dtype=np.float64) for v in per_rank])) if per_rank else []
    return {"requests": int(len(allv)), "p50_ms": percentile(allv, 0.50), "p99_ms": percentile(allv, 0.99),
            "mean_ms": float(np.mean(allv)) if len(allv) else 0.0}


def gather(obj, dist):
    """Every rank's `obj`, in rank order (dist = torch.distributed or None)."""
    if dist is None:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out
