"""Level fusion of the triangular systems (host logic, no GPU).

rlsq_factor fuses groups of consecutive levels by substituting, inside a
group, a row's dependencies on rows of the same group:
x_i = (rhs_i + sum_R c rhs_j - sum_T c x_j) / d_i.  These tests take the fused
systems from the host-only API and check them against the definition:
solving the fused form in level order gives the same x as solving the
original system (scipy's sparse triangular solve) to rounding; every remaining
T dependency lies in an earlier group; fusion never adds levels.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular

from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import synth

SYSTEMS = [(B.SYS_L1, True, False), (B.SYS_L1T, False, False), (B.SYS_U, False, True), (B.SYS_UT, True, True)]


@pytest.fixture(scope="module")
def setup():
    prob = synth.sparse_problem(30_001, 15_001, 6, seed=21, hidden_diag=True)
    H = B.HostSetup(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, mu=1.0, p=10, tau=1e-2)
    n = prob.n
    Lp, Li, Lv = H.factor_csr(B.PART_L1)
    Up, Ui, Uv = H.factor_csr(B.PART_U)
    L = sp.csr_matrix((Lv, Li, Lp), shape=(n, n))
    U = sp.csr_matrix((Uv, Ui, Up), shape=(n, n))
    _, _, _, ud = H.split()
    strict = {B.SYS_L1: L, B.SYS_L1T: L.T.tocsr(), B.SYS_U: U, B.SYS_UT: U.T.tocsr()}
    return H, n, strict, ud


def fused_solve(n, T, R, d, lev, b):
    """x from the fused rows, rows taken in the original level order."""
    Tp, Ti, Tv = T
    Rp, Ri, Rv = R
    x = np.zeros(n)
    for i in np.argsort(lev, kind="stable"):
        v = b[i]
        for e in range(Rp[i], Rp[i + 1]):
            v += Rv[e] * b[Ri[e]]
        for e in range(Tp[i], Tp[i + 1]):
            v -= Tv[e] * x[Ti[e]]
        x[i] = v / d[i]
    return x


@pytest.mark.parametrize("k", [2, 3, 0])
@pytest.mark.parametrize("which,lower,has_diag", SYSTEMS)
def test_fused_solve_equals_original(setup, which, lower, has_diag, k):
    H, n, strict, ud = setup
    S = strict[which]
    d = ud if has_diag else np.ones(n)
    lev = H.levels(which)
    sizes, T, R = H.fuse(which, k)
    # fusion never adds levels; fixed k gives at most ceil(levels / k)
    nlev = int(lev.max()) + 1
    assert sizes["levels"] <= nlev
    if k > 0:
        assert sizes["levels"] <= -(-nlev // k)
    # every remaining dependency lies in an earlier group (fixed k: group = level // k)
    Tp, Ti, _ = T
    rows = np.repeat(np.arange(n), np.diff(Tp))
    if k > 0:
        assert np.all(lev[Ti] // k < lev[rows] // k)
    else:
        assert np.all(lev[Ti] < lev[rows])
    # same solution as the original system
    b = np.random.default_rng(3).standard_normal(n)
    A = (S + sp.diags(d)).tocsr()
    ref = spsolve_triangular(A, b, lower=lower)
    x = fused_solve(n, T, R, d, lev, b)
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)


def test_unfused_is_the_original(setup):
    H, n, strict, _ = setup
    sizes, T, R = H.fuse(B.SYS_U, 1)
    Tp, Ti, Tv = T
    U = strict[B.SYS_U]
    assert sizes["nnz_R"] == 0 and sizes["nnz_T"] == U.nnz
    assert np.array_equal(Tp, U.indptr.astype(np.int64)) and np.array_equal(Ti, U.indices)
    assert np.array_equal(Tv, U.data)


def test_fuse_rejects_bad_arguments(setup):
    H, _, _, _ = setup
    with pytest.raises(B.RlsqError):
        H.fuse(7, 2)
    with pytest.raises(B.RlsqError):
        H.fuse(B.SYS_L1, -1)
