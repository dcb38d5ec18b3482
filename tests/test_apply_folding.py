"""The identity behind the GPU apply's CG(k) tail (CPU, from the oracle's
factors with scipy's triangular solves).

Algorithm 3 with k CG steps on S^ w = e ends with f = L2^T w, L1^T y = f,
L1 v = g2 - y.  The CG iteration forms c3_j = L1^{-1} L1^{-T} L2^T p_j for each
direction p_j, and w = sum_j a_j p_j, so v = q1 - sum_j a_j c3_j with
q1 = L1^{-1} g2.  Both orders are computed here step by step and each is held
to the oracle's apply (which runs the printed order) within 1e-13, at two sizes
and for k = 1, 2, 4."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sl

import oracle
from paper_2603_28642_gb300 import synth


def factors(f):
    L1, L2 = f.L1(), f.L2()
    U, ud = f.U()
    n = L1.shape[0]
    L1s = (sp.csr_matrix((L1.val, L1.idx, L1.ptr), shape=L1.shape) + sp.eye(n)).tocsr()
    L2s = sp.csr_matrix((L2.val, L2.idx, L2.ptr), shape=L2.shape).tocsr()
    Us = (sp.csr_matrix((U.val, U.idx, U.ptr), shape=U.shape) + sp.diags(ud)).tocsr()
    return L1s, L2s, Us


def both_orders(f, s, k):
    L1, L2, U = factors(f)
    d = f.scaling()
    lower = lambda M, b: sl.spsolve_triangular(M, b, lower=True)
    upper = lambda M, b: sl.spsolve_triangular(M, b, lower=False)
    L1t, Ut = L1.T.tocsr(), U.T.tocsr()
    g2 = upper(L1t, lower(Ut, d * s))
    q1 = lower(L1, g2)
    r = L2 @ q1
    w = np.zeros_like(r)
    z = np.zeros_like(q1)
    rr = r @ r
    p = r.copy()
    for j in range(k):
        if j > 0:
            p = r + (rr_new / rr) * p
            rr = rr_new
        c3 = lower(L1, upper(L1t, L2.T @ p))
        sp_ = p + L2 @ c3
        a = rr / (p @ sp_)
        w += a * p
        z += a * c3
        r = r - a * sp_
        rr_new = r @ r
    printed = d * upper(U, lower(L1, g2 - upper(L1t, L2.T @ w)))
    folded = d * upper(U, q1 - z)
    return printed, folded


@pytest.mark.parametrize("k", [1, 2, 4])
@pytest.mark.parametrize("which", ["cfg0", "small_cfg1"])
def test_folded_tail_equals_printed_order(which, k):
    prob = synth.config_problem(0) if which == "cfg0" else synth.config_problem(1, scale=0.005)
    f = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, mu=1.0)
    f.set_correction(oracle.CG, k)
    s = np.random.default_rng(k).standard_normal(prob.n)
    ref = f.apply(s)
    printed, folded = both_orders(f, s, k)
    rel = lambda a: np.max(np.abs(a - ref)) / np.max(np.abs(ref))
    assert rel(printed) <= 1e-13  # the restatement is the oracle's apply
    assert rel(folded) <= 1e-13   # and the folded tail is the same operator
