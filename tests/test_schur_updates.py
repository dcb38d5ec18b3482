"""Sec. 3.4 for the dense correction: S = I + Y Y^T (Y = L2 L1^{-1}, eq. 3.9)
changes by a border when rows join A2 and loses rows and columns when rows
leave, and the library updates S^{-1} by block inversion instead of forming it
again.  Pinned against numpy's inverse of S built from the factor, and
against the library's own formation after the update.  No GPU is used."""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import synth


def dense_factor(s, part):
    ptr, idx, val = s.factor_csr(part)
    rows = len(ptr) - 1
    out = np.zeros((rows, s.n))
    for r in range(rows):
        out[r, idx[ptr[r]:ptr[r + 1]]] = val[ptr[r]:ptr[r + 1]]
    return out


def numpy_sinv(s):
    L1 = np.eye(s.n) + dense_factor(s, B.PART_L1)
    L2 = dense_factor(s, B.PART_L2)
    Y = sla.solve_triangular(L1, L2.T, lower=True, trans="T", unit_diagonal=True).T  # L2 L1^{-1}
    return np.linalg.inv(np.eye(L2.shape[0]) + Y @ Y.T)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def new_rows(n, k, d, seed):
    rng = np.random.default_rng(seed)
    rows = [np.sort(rng.choice(n, size=d, replace=False)) for _ in range(k)]
    ptr = np.zeros(k + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rows])
    return ptr, np.concatenate(rows).astype(np.int32), rng.standard_normal(int(ptr[-1]))


@pytest.fixture()
def setup():
    prob = synth.sparse_problem(700, 400, 5, seed=41)
    return prob, B.HostSetup(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, mu=1.0)


def test_formed_inverse_matches_numpy(setup):
    _, s = setup
    X = s.schur_inverse()
    assert X.shape == (300, 300)
    assert rel(X, numpy_sinv(s)) < 1e-11
    assert np.allclose(X, X.T, rtol=0, atol=1e-14)


def test_updates_follow_added_and_removed_rows(setup):
    prob, s = setup
    s.schur_inverse()  # held from here on
    ptr, idx, val = new_rows(prob.n, 9, 6, seed=5)
    s.add_rows(ptr, idx, val)
    X = s.schur_inverse()
    assert X.shape == (309, 309)
    assert rel(X, numpy_sinv(s)) < 1e-11
    # remove old and new rows of A2 (their original ids, ascending)
    _, a2, _, _ = s.split()
    ids = np.sort(np.concatenate([a2[[0, 17, 150]], a2[-4:-1]])).astype(np.int32)
    s.remove_rows(ids)
    X = s.schur_inverse()
    assert X.shape == (303, 303)
    assert rel(X, numpy_sinv(s)) < 1e-11
    # and more rows again: the updated inverse against the library's formation
    ptr, idx, val = new_rows(prob.n, 3, 4, seed=6)
    s.add_rows(ptr, idx, val)
    X = s.schur_inverse()
    assert rel(X, s.schur_inverse(recompute=True)) < 1e-11


def test_update_without_held_inverse_forms_it(setup):
    prob, s = setup
    ptr, idx, val = new_rows(prob.n, 2, 3, seed=7)
    s.add_rows(ptr, idx, val)  # nothing held yet: formed when asked
    assert rel(s.schur_inverse(), numpy_sinv(s)) < 1e-11
