"""The 2M x 1M workload at full size, in the launch configuration bench.py
times (ILUP(p=10, tau=1e-2, mu=1), CG(2), autotuned).  The oracle's ILUP is too
slow at this size, so the checks are properties that hold at any size,
computed independently on the host with scipy:

* the stopping ratio ||A^T r|| / (||A||_2 ||r||) of the returned x, from the
  explicit residual, is below 1e-8 (FP64 apply, FP32 apply, CGLS);
* x agrees with scipy's LSQR solution (unpreconditioned, run to 1e-12);
* the preconditioner is positive (<s, M^{-1} s> > 0) and positively
  homogeneous (CG(k) is not linear in its right-hand side).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import synth

pytestmark = pytest.mark.gpu

FACTOR = dict(p=10, tau=1e-2, mu=1.0, correction=B.CORR_CG, cg_steps=2, autotune=1)


@pytest.fixture(scope="module")
def full():
    prob = synth.config_problem(1)
    A = prob.to_scipy()
    anorm = spla.svds(A, k=1, return_singular_vectors=False, tol=1e-6)[0]
    x_ref = spla.lsqr(A, prob.b, atol=1e-12, btol=1e-12, iter_lim=500)[0]
    P = B.Problem.from_problem(prob)
    P.factor(**FACTOR)
    return prob, A, anorm, x_ref, P


def explicit_ratio(A, anorm, b, x):
    r = b - A @ x
    return np.linalg.norm(A.T @ r) / (anorm * np.linalg.norm(r))


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_fullsize_fp64_solve(full):
    prob, A, anorm, x_ref, P = full
    res = P.solve(prob.b)
    assert res.status == 0
    assert explicit_ratio(A, anorm, prob.b, res.x) < 1.01e-8
    assert rel(res.x, x_ref) < 1e-6
    # the library's ||A|| (50 power steps) bounds the true norm from below, so its
    # own stopping ratio is the more demanding one
    assert 0.95 * anorm <= P.info()["anorm"] <= anorm * (1 + 1e-6)


def test_fullsize_cgls(full):
    prob, A, anorm, x_ref, P = full
    res = P.solve(prob.b, solver=B.SOLVER_CGLS)
    assert res.status == 0
    assert explicit_ratio(A, anorm, prob.b, res.x) < 1.01e-8
    assert rel(res.x, x_ref) < 1e-6


def test_fullsize_apply_positive_and_homogeneous(full):
    # CG(k) from zero is not linear in its right-hand side (its step lengths
    # depend on it), but it is positively homogeneous: M^{-1}(a s) = a M^{-1} s
    prob, _, _, _, P = full
    rng = np.random.default_rng(12)
    s1 = rng.standard_normal(prob.n)
    s2 = rng.standard_normal(prob.n)
    t1, t2 = P.apply(s1), P.apply(s2)
    assert s1 @ t1 > 0 and s2 @ t2 > 0
    assert rel(P.apply(2.5 * s1), 2.5 * t1) < 1e-12


def test_fullsize_fp32_apply(full):
    # last: re-factors the shared handle in float32 (the host ILUP is reused)
    prob, A, anorm, x_ref, P = full
    P.factor(**FACTOR, precision=B.PREC_FP32)
    res = P.solve(prob.b)
    assert res.status == 0
    assert explicit_ratio(A, anorm, prob.b, res.x) < 1.01e-8
    assert rel(res.x, x_ref) < 1e-6
