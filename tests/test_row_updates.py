"""Adding and removing rows without refactorising (Sec. 3.4), host only.

* the library's host update equals the oracle's bit for bit (L2, A2 rows,
  pivot rows after renumbering);
* with the exact LU (nothing dropped) a new L2 row l satisfies l U = a D, and
  the dense-S preconditioner of the updated factor applied to A'^T r is the
  least-squares correction of the augmented (or reduced) problem A';
* with the ILU factor, LSMR on the augmented problem still reaches its lstsq
  solution; removing a pivot row is refused (a refactorisation is needed).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import synth


def new_rows(n, k, d, seed):
    rng = np.random.default_rng(seed)
    rows = [np.sort(rng.choice(n, size=d, replace=False)) for _ in range(k)]
    ptr = np.zeros(k + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rows])
    idx = np.concatenate(rows).astype(np.int32)
    val = rng.standard_normal(len(idx))
    return ptr, idx, val


def stacked(prob, ptr, idx, val):
    A = prob.to_scipy()
    R = sp.csr_matrix((val, idx, ptr), shape=(len(ptr) - 1, prob.n))
    return sp.vstack([A, R]).tocsr()


@pytest.fixture()
def cfg0():
    return synth.config_problem(0)


def same_l2(H, f):
    ptr, idx, val = H.factor_csr(B.PART_L2)
    L2 = f.L2()
    return (np.array_equal(ptr, L2.ptr) and np.array_equal(idx, L2.idx) and np.array_equal(val, L2.val))


def test_add_rows_matches_oracle(cfg0):
    p = cfg0
    H = B.HostSetup(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=1.0, p=10, tau=1e-2)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=1.0, p=10, tau=1e-2)
    ptr, idx, val = new_rows(p.n, 5, 6, seed=1)
    H.add_rows(ptr, idx, val)
    assert f.add_rows(ptr, idx, val, p=10, tau=1e-2) == 0
    prow, a2, _, _ = H.split()
    oprow, oa2 = f.perm()
    assert np.array_equal(prow, oprow) and np.array_equal(a2, oa2)
    assert list(a2[-5:]) == list(range(p.m, p.m + 5))
    assert H.sizes()["nnz_L2"] == f.sizes()["nnz_L2"] and same_l2(H, f)


def test_remove_rows_matches_oracle(cfg0):
    p = cfg0
    H = B.HostSetup(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=1.0)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=1.0)
    _, a2 = f.perm()
    ids = np.sort(np.random.default_rng(2).choice(a2, size=7, replace=False)).astype(np.int32)
    H.remove_rows(ids)
    assert f.remove_rows(ids) == 0
    prow, na2, _, _ = H.split()
    oprow, oa2 = f.perm()
    assert np.array_equal(prow, oprow) and np.array_equal(na2, oa2)
    assert len(na2) == p.m - p.n - 7 and same_l2(H, f)
    # renumbering: every surviving row keeps its order
    keep = np.setdiff1d(np.arange(p.m), ids)
    assert np.array_equal(np.sort(np.concatenate([prow, na2])), np.arange(len(keep)))


def test_remove_pivot_row_refused(cfg0):
    p = cfg0
    H = B.HostSetup(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=1.0)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=1.0)
    prow, _ = f.perm()
    bad = np.array([prow[0]], dtype=np.int32)
    with pytest.raises(B.RlsqError) as e:
        H.remove_rows(bad)
    assert e.value.code == -1
    assert f.remove_rows(bad) == -1


def test_exact_factor_add_rows_is_exact():
    p = synth.sparse_problem(70, 45, 4, seed=41)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, p=-1, tau=0.0, mu=1.0)
    ptr, idx, val = new_rows(p.n, 6, 4, seed=3)
    assert f.add_rows(ptr, idx, val, p=-1, tau=0.0) == 0
    Uc, ud = f.U()
    U = Uc.to_scipy().toarray() + np.diag(ud)
    d = f.scaling()
    L2 = f.L2().to_scipy().toarray()
    R = sp.csr_matrix((val, idx, ptr), shape=(6, p.n)).toarray()
    np.testing.assert_allclose(L2[-6:] @ U, R * d, rtol=1e-10, atol=1e-12)   # l U = a D
    f.set_correction(oracle.DENSE)
    A2 = stacked(p, ptr, idx, val).toarray()
    r = np.random.default_rng(4).standard_normal(A2.shape[0])
    ref = np.linalg.lstsq(A2, r, rcond=None)[0]
    np.testing.assert_allclose(f.apply(A2.T @ r), ref, rtol=1e-9, atol=1e-10)


def test_exact_factor_remove_rows_is_exact():
    p = synth.sparse_problem(70, 45, 4, seed=42)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, p=-1, tau=0.0, mu=1.0)
    _, a2 = f.perm()
    ids = np.sort(a2[::3]).astype(np.int32)
    assert f.remove_rows(ids) == 0
    f.set_correction(oracle.DENSE)
    Ar = np.delete(p.to_scipy().toarray(), ids, axis=0)
    r = np.random.default_rng(5).standard_normal(Ar.shape[0])
    ref = np.linalg.lstsq(Ar, r, rcond=None)[0]
    np.testing.assert_allclose(f.apply(Ar.T @ r), ref, rtol=1e-9, atol=1e-10)


def test_ilu_update_still_preconditions(cfg0):
    p = cfg0
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=1.0)
    ptr, idx, val = new_rows(p.n, 20, 6, seed=6)
    assert f.add_rows(ptr, idx, val) == 0
    f.set_correction(oracle.CG, 2)
    A2 = stacked(p, ptr, idx, val)
    b2 = np.concatenate([p.b, np.random.default_rng(7).standard_normal(20)])
    res = oracle.lsmr(f, A2.shape[0], p.n, A2.indptr, A2.indices, A2.data, b2, atol=1e-8, maxit=2000)
    assert res.status == 0 and res.its < 100
    np.testing.assert_allclose(res.x, np.linalg.lstsq(A2.toarray(), b2, rcond=None)[0], rtol=1e-6)


def test_removing_every_row_of_A2_is_refused():
    """The problem needs m > n (eq. 1.1): at least one row of A2 stays."""
    prob = synth.sparse_problem(60, 40, 4, seed=3)
    s = B.HostSetup(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, mu=1.0)
    _, a2, _, _ = s.split()
    with pytest.raises(B.RlsqError) as e:
        s.remove_rows(a2.astype(np.int32))
    assert e.value.code == -2  # RLSQ_ERR_SHAPE
    s.remove_rows(a2[1:].astype(np.int32))  # all but one
    assert s.m == prob.n + 1
