"""Row updates (Sec. 3.4) on a factored GPU handle against the oracle's
updated factor: the same L2 and A2 rows (bit for bit), and LSMR on the
augmented / reduced problem with the same iteration count (+-1) and x within
1e-6."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import synth

pytestmark = pytest.mark.gpu


def new_rows(n, k, d, seed):
    rng = np.random.default_rng(seed)
    rows = [np.sort(rng.choice(n, size=d, replace=False)) for _ in range(k)]
    ptr = np.zeros(k + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rows])
    return ptr, np.concatenate(rows).astype(np.int32), rng.standard_normal(int(ptr[-1]))


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def check_against_oracle(P, f, A, b):
    prow, a2, _, _ = P.split()
    oprow, oa2 = f.perm()
    assert np.array_equal(prow, oprow) and np.array_equal(a2, oa2)
    ptr, idx, val = P.factor_csr(B.PART_L2)
    L2 = f.L2()
    assert np.array_equal(ptr, L2.ptr) and np.array_equal(idx, L2.idx) and np.array_equal(val, L2.val)
    res = P.solve(b)
    ref = oracle.lsmr(f, A.shape[0], A.shape[1], A.indptr, A.indices, A.data, b)
    assert res.status == 0 and ref.status == 0
    assert abs(res.info["iterations"] - ref.its) <= 1
    assert rel(res.x, ref.x) <= 1e-6


def test_add_then_remove_rows():
    p = synth.config_problem(0)
    P = B.Problem.from_problem(p)
    P.factor(mu=1.0, correction=B.CORR_CG)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=1.0)
    f.set_correction(oracle.CG, 2)
    ptr, idx, val = new_rows(p.n, 20, 6, seed=11)
    info = P.add_rows(ptr, idx, val)
    assert f.add_rows(ptr, idx, val) == 0
    assert info["m"] == p.m + 20
    A = sp.vstack([p.to_scipy(), sp.csr_matrix((val, idx, ptr), shape=(20, p.n))]).tocsr()
    b = np.concatenate([p.b, np.random.default_rng(12).standard_normal(20)])
    check_against_oracle(P, f, A, b)
    # now remove some rows of A2 (old and new ones)
    _, a2 = f.perm()
    ids = np.sort(np.concatenate([a2[:5], a2[-3:]])).astype(np.int32)
    P.remove_rows(ids)
    assert f.remove_rows(ids) == 0
    keep = np.setdiff1d(np.arange(A.shape[0]), ids)
    check_against_oracle(P, f, A[keep].tocsr(), b[keep])


def test_remove_pivot_row_refused():
    p = synth.config_problem(0)
    P = B.Problem.from_problem(p)
    P.factor(mu=1.0, correction=B.CORR_CG)
    prow, _, _, _ = P.split()
    with pytest.raises(B.RlsqError) as e:
        P.remove_rows(np.array([prow[0]], dtype=np.int32))
    assert e.value.code == -1


def test_registered_problem_refuses_changes():
    """While a server holds the problem, its device data must stay: refactoring
    and row updates are refused (ARG) until the server is destroyed."""
    p = synth.config_problem(0)
    P = B.Problem.from_problem(p)
    P.factor(mu=1.0, correction=B.CORR_CG)
    srv = B.Server(hbm_budget_bytes=1 << 30, max_slots=2)
    srv.register(P)
    ptr, idx, val = new_rows(p.n, 2, 4, seed=3)
    for call in (lambda: P.add_rows(ptr, idx, val), lambda: P.factor(mu=1.0, correction=B.CORR_CG)):
        with pytest.raises(B.RlsqError) as e:
            call()
        assert e.value.code == -1
    assert P.m == p.m
    srv.close()
    assert P.add_rows(ptr, idx, val)["m"] == p.m + 2


def test_dense_correction_follows_row_updates():
    """With the dense correction the handle updates S^{-1} with the rows (block
    inversion, Sec. 3.4) instead of forming it again; its solves match the
    oracle, which forms S for the updated factor."""
    p = synth.config_problem(0)
    P = B.Problem.from_problem(p)
    P.factor(mu=1.0, correction=B.CORR_DENSE)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=1.0)
    ptr, idx, val = new_rows(p.n, 12, 6, seed=21)
    P.add_rows(ptr, idx, val)
    assert f.add_rows(ptr, idx, val) == 0
    f.set_correction(oracle.DENSE)
    A = sp.vstack([p.to_scipy(), sp.csr_matrix((val, idx, ptr), shape=(12, p.n))]).tocsr()
    b = np.concatenate([p.b, np.random.default_rng(22).standard_normal(12)])
    check_against_oracle(P, f, A, b)
    _, a2 = f.perm()
    ids = np.sort(np.concatenate([a2[:4], a2[-2:]])).astype(np.int32)
    P.remove_rows(ids)
    assert f.remove_rows(ids) == 0
    f.set_correction(oracle.DENSE)
    keep = np.setdiff1d(np.arange(A.shape[0]), ids)
    check_against_oracle(P, f, A[keep].tocsr(), b[keep])
