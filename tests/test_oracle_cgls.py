"""Pins for the oracle's Algorithm 3 on a residual and Algorithm 1 (CGLS).

Algorithm 3 with the exact LU (nothing dropped) and the dense S^ must return
the least-squares correction (A^T A)^{-1} A^T r (Sec. 3.1), with S^ = I dropped
to NONE it must invert A1, CG with m - n steps must reproduce the dense S^;
CGLS with the exact preconditioner must finish in one step, and with the
ILU preconditioners it must reach the lstsq solution.
"""
import numpy as np
import pytest

import oracle
from paper_2603_28642_gb300 import synth


def dense(p):
    return p.to_scipy().toarray()


@pytest.fixture(scope="module")
def exact():
    p = synth.sparse_problem(70, 45, 4, seed=41)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, p=-1, tau=0.0, mu=1.0)
    return p, f


def test_residual_apply_exact_dense_is_least_squares_correction(exact):
    p, f = exact
    f.set_correction(oracle.DENSE)
    A = dense(p)
    r = np.random.default_rng(1).standard_normal(p.m)
    ref = np.linalg.lstsq(A, r, rcond=None)[0]
    np.testing.assert_allclose(f.apply_residual(r), ref, rtol=1e-10, atol=1e-11)


def test_residual_apply_none_inverts_A1(exact):
    p, f = exact
    f.set_correction(oracle.NONE)
    prow, _ = f.perm()
    A1 = dense(p)[prow]
    r = np.random.default_rng(2).standard_normal(p.m)
    np.testing.assert_allclose(f.apply_residual(r), np.linalg.solve(A1, r[prow]), rtol=1e-9, atol=1e-10)


def test_residual_apply_cg_converges_to_dense(exact):
    p, f = exact
    r = np.random.default_rng(3).standard_normal(p.m)
    f.set_correction(oracle.DENSE)
    hd = f.apply_residual(r)
    f.set_correction(oracle.CG, p.m - p.n)  # CG is exact on S^ in m - n steps
    np.testing.assert_allclose(f.apply_residual(r), hd, rtol=1e-7, atol=1e-8)


def test_cgls_exact_preconditioner_one_step(exact):
    p, f = exact
    f.set_correction(oracle.DENSE)
    x_ls = np.linalg.lstsq(dense(p), p.b, rcond=None)[0]
    res = oracle.cgls(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, atol=1e-10, maxit=20)
    assert res.status == 0 and res.its == 1
    np.testing.assert_allclose(res.x, x_ls, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("mode", [oracle.NONE, oracle.CG, oracle.DENSE])
def test_cgls_symmetric_form_reaches_least_squares(mode):
    """Algorithm 1 with h = M^{-1} A^T r (the x-space operator): converges like LSMR."""
    p = synth.config_problem(0)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=1.0)
    f.set_correction(mode, 2)
    A = dense(p)
    x_ls = np.linalg.lstsq(A, p.b, rcond=None)[0]
    res = oracle.cgls(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, atol=1e-8, maxit=2000, form="symmetric")
    assert res.status == 0 and res.its < 60
    rr = p.b - A @ res.x
    ratio = np.linalg.norm(A.T @ rr) / (np.linalg.norm(A, 2) * np.linalg.norm(rr))
    assert ratio < 2e-8
    np.testing.assert_allclose(res.x, x_ls, rtol=1e-6)
    # LSMR with the same preconditioner needs a comparable number of iterations
    ls = oracle.lsmr(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, atol=1e-8, maxit=2000)
    assert abs(ls.its - res.its) <= 3
    # the history starts at ||A^T b|| / (||A|| ||b||)
    assert res.ratio_hist[0] == pytest.approx(
        np.linalg.norm(A.T @ p.b) / (oracle.norm2(p.m, p.n, p.rowptr, p.colidx, p.vals) * np.linalg.norm(p.b)),
        rel=1e-12)


@pytest.mark.parametrize("mode", [oracle.NONE, oracle.CG, oracle.DENSE])
def test_cgls_residual_form_stalls_with_incomplete_factors(mode):
    """With dropped entries Algorithm 3 fed the residual split is no longer
    M^{-1} A^T for any M: at the least-squares residual (A^T r = 0, r != 0) it
    does not vanish, and CGLS stalls far above 1e-8 on the config-0 matrix
    while x stays near the solution.  (Exact factors: one step, pinned above.)"""
    p = synth.config_problem(0)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=1.0)
    f.set_correction(mode, 2)
    A = dense(p)
    x_ls = np.linalg.lstsq(A, p.b, rcond=None)[0]
    res = oracle.cgls(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, atol=1e-8, maxit=300)
    assert res.status == 1 and res.ratio > 1e-3
    # at the least-squares residual the residual-form apply is far from zero
    r_ls = p.b - A @ x_ls
    assert np.linalg.norm(f.apply_residual(r_ls)) > 1e3 * np.linalg.norm(f.apply(A.T @ r_ls))
    assert np.linalg.norm(res.x - x_ls) < 1e-2 * np.linalg.norm(x_ls)
