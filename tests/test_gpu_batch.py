"""Batched and served forms on the GPU.

* rlsq_batch_solve: each problem of an uneven batch (sizes, nonzeros per row,
  correction modes, lanes per row of its products chosen per problem)
  matches the CPU oracle (x within 1e-6 relative, equal iteration counts),
  and gives exactly the same bits alone and in the mix.
* server: requests over shared resident matrices give exactly the bits of
  the same solve done alone, complete under a memory budget that admits one
  request at a time, and overlap on the device (continuous batching).
"""
import time

import numpy as np
import pytest

import oracle
from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import synth

pytestmark = pytest.mark.gpu

MU = 1.0


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def uneven_problems(count=6, seed=70):
    """Problems shaped like the batched workload, at small sizes."""
    n, m, d = synth.batch_problem_sizes(count, master_seed=seed, n_lo=300, n_hi=1500)
    return [synth.sparse_problem(int(m[k]), int(n[k]), int(d[k]), seed=seed * 100 + k) for k in range(count)]


MODES = [B.CORR_CG, B.CORR_DENSE, B.CORR_NONE]
ORACLE_MODE = {B.CORR_CG: oracle.CG, B.CORR_DENSE: oracle.DENSE, B.CORR_NONE: oracle.NONE}


@pytest.fixture(scope="module")
def batch():
    probs = uneven_problems()
    handles = []
    for k, p in enumerate(probs):
        P = B.Problem.from_problem(p)
        P.factor(mu=MU, correction=MODES[k % 3])
        handles.append(P)
    return probs, handles


def test_batch_matches_oracle(batch):
    probs, handles = batch
    xs, infos, code = B.batch_solve(handles, [p.b for p in probs])
    assert code == 0
    for k, (p, x, info) in enumerate(zip(probs, xs, infos)):
        f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=MU)
        f.set_correction(ORACLE_MODE[MODES[k % 3]], 2)
        ref = oracle.lsmr(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b)
        assert info["status"] == 0 and ref.status == 0
        assert abs(info["iterations"] - ref.its) <= 1, (k, info["iterations"], ref.its)
        assert rel(x, ref.x) <= 1e-6


def test_batch_alone_equals_in_mix(batch):
    probs, handles = batch
    xs, infos, _ = B.batch_solve(handles, [p.b for p in probs])
    for k in (0, 3, 5):
        xa, ia, _ = B.batch_solve([handles[k]], [probs[k].b])
        assert ia[0]["iterations"] == infos[k]["iterations"]
        assert np.array_equal(xa[0], xs[k])  # bit-identical
    # a different mix (reversed order, subset) gives the same bits too
    sub = [4, 1, 2]
    xr, ir, _ = B.batch_solve([handles[k] for k in sub], [probs[k].b for k in sub])
    for j, k in enumerate(sub):
        assert np.array_equal(xr[j], xs[k])


def test_batch_tuned_lanes_alone_equals_in_mix():
    """Slots whose problems were autotuned (autotune = 2: lanes of the A, A^T,
    L2, L2^T products, chosen per problem) run with their own lanes in the
    batch: oracle parity, and the same bits alone and in any mix."""
    # the last problem has 12 entries per row (wider lanes) and a strong diagonal (fast convergence)
    probs = uneven_problems(count=5, seed=71) + [synth.sparse_problem(3000, 1500, 12, seed=72, diag_value=8.0)]
    hs = []
    for k, p in enumerate(probs):
        P = B.Problem.from_problem(p)
        P.factor(mu=MU, correction=B.CORR_CG, autotune=2 if k % 2 == 0 else 0)
        hs.append(P)
    xs, infos, code = B.batch_solve(hs, [p.b for p in probs])
    assert code == 0
    for k, (p, x, info) in enumerate(zip(probs, xs, infos)):
        f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=MU)
        f.set_correction(oracle.CG, 2)
        ref = oracle.lsmr(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b)
        assert info["status"] == 0 and abs(info["iterations"] - ref.its) <= 1, (k, info["iterations"], ref.its)
        assert rel(x, ref.x) <= 1e-6
    for k in range(len(probs)):
        xa, ia, _ = B.batch_solve([hs[k]], [probs[k].b])
        assert np.array_equal(xa[0], xs[k]) and ia[0]["iterations"] == infos[k]["iterations"]
    sub = [5, 2, 0]
    xr, _, _ = B.batch_solve([hs[k] for k in sub], [probs[k].b for k in sub])
    for j, k in enumerate(sub):
        assert np.array_equal(xr[j], xs[k])


def test_batch_fp32_apply():
    probs = uneven_problems(4, seed=71)
    hs = []
    for p in probs:
        P = B.Problem.from_problem(p)
        P.factor(mu=MU, correction=B.CORR_CG, precision=B.PREC_FP32)
        hs.append(P)
    xs, infos, code = B.batch_solve(hs, [p.b for p in probs])
    assert code == 0
    for p, x, info in zip(probs, xs, infos):
        x_ls = np.linalg.lstsq(p.to_scipy().toarray(), p.b, rcond=None)[0]
        assert rel(x, x_ls) <= 1e-6
        assert info["ratio"] < 1e-8


def _serve(srv, mats, jobs, timeout=120.0):
    tickets = [(srv.submit(mid, b), mid) for mid, b in jobs]
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t, mid in tickets:
            if t in out:
                continue
            r = srv.poll(t, mats[mid].n)
            if r is not None:
                out[t] = r
        assert time.time() - t0 < timeout
        time.sleep(0.002)
    return [out[t] for t, _ in tickets]


@pytest.fixture(scope="module")
def served():
    probs = [synth.sparse_problem(int(1.5 * n), n, 6, seed=4000 + k) for k, n in enumerate((800, 2000, 5000))]
    hs = []
    for p in probs:
        P = B.Problem.from_problem(p)
        P.factor(mu=MU, correction=B.CORR_CG)
        hs.append(P)
    return probs, hs


def test_server_results_equal_solo_solves(served):
    probs, hs = served
    srv = B.Server(hbm_budget_bytes=1 << 34, max_slots=8)
    ids = [srv.register(P) for P in hs]
    rng = np.random.default_rng(5)
    jobs = []
    for r in range(12):
        mid = int(rng.integers(0, len(hs)))
        jobs.append((ids[mid], synth.serving_rhs(probs[mid], r)))
    results = _serve(srv, probs, jobs)
    for (mid, b), (x, info, code) in zip(jobs, results):
        assert code == 0
        xa, ia, _ = B.batch_solve([hs[mid]], [b])
        assert ia[0]["iterations"] == info["iterations"]
        assert np.array_equal(xa[0], x)
    st = srv.stats()
    assert st["completed"] == 12 and st["queued"] == 0 and st["active"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    # continuous batching: fewer batched iterations than the solves' iterations summed
    assert st["ticks"] < sum(info["iterations"] for _, info, _ in results)
    srv.close()


def test_server_admission_under_small_budget(served):
    probs, hs = served
    # a budget for one request of the largest matrix at a time
    big = max(probs, key=lambda p: p.n)
    budget = 16 * big.m + 16 * big.n + 8 * big.m + 24 * big.n + 48 * big.n + 32 * (big.m - big.n) + 8192
    srv = B.Server(hbm_budget_bytes=budget, max_slots=4)
    ids = [srv.register(P) for P in hs]
    jobs = [(ids[k % 3], synth.serving_rhs(probs[k % 3], 100 + k)) for k in range(6)]
    results = _serve(srv, probs, jobs)
    assert all(code == 0 for _, _, code in results)
    st = srv.stats()
    assert st["completed"] == 6 and st["peak_bytes"] <= budget
    srv.close()


def test_server_rejects_bad_requests(served):
    probs, hs = served
    srv = B.Server(hbm_budget_bytes=1 << 30, max_slots=2)
    srv.register(hs[0])
    with pytest.raises(B.RlsqError) as e:
        srv.submit(7, probs[0].b)
    assert e.value.code == -12
    tiny = B.Server(hbm_budget_bytes=1024, max_slots=2)
    with pytest.raises(B.RlsqError) as e:
        tiny.register(hs[0])
    assert e.value.code == -11
    srv.close()
    tiny.close()


def test_batch_beyond_persistent_slots_same_bits():
    """More slots than one block can scan (1,030 > 1,024): the batch falls back
    to one launch per fused level group, with the same row arithmetic, so a
    problem's bits equal those of its solve alone (persistent path)."""
    n, m, d = synth.batch_problem_sizes(1030, master_seed=73, n_lo=20, n_hi=40)
    probs = [synth.sparse_problem(int(m[k]), int(n[k]), int(d[k]), seed=7300 + k) for k in range(1030)]
    hs = []
    for p in probs:
        P = B.Problem.from_problem(p)
        P.factor(mu=MU, correction=B.CORR_CG, host_threads=1)
        hs.append(P)
    xs, infos, code = B.batch_solve(hs, [p.b for p in probs])
    assert code == 0
    for k in (0, 517, 1029):
        xa, ia, _ = B.batch_solve([hs[k]], [probs[k].b])
        assert ia[0]["iterations"] == infos[k]["iterations"] and np.array_equal(xa[0], xs[k])
        p = probs[k]
        f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=MU)
        f.set_correction(oracle.CG, 2)
        ref = oracle.lsmr(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b)
        assert rel(xs[k], ref.x) <= 1e-6
