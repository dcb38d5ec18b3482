"""The sliced layout of the sparse products (A, A^T, L2, L2^T: one lane per
row, rows sorted by length within windows of 1024, slices of 32 rows stored
column-major) against the oracle, through the C ABI.

* the preconditioner application (its L2 and L2^T products) within 1e-12,
  in the 2-norm and element by element, for every correction;
* LSMR solves (the A and A^T products as well) with the oracle's iteration
  counts and x within 1e-6, also unpreconditioned, at n = 50,001 (a ragged
  last slice), in float32, and on a sparse-dense problem whose dense rows are
  empty rows of the sliced A;
* the same iterations and x (1e-10) as the CSR layout;
* the layout reported per product, chosen by the autotuner when asked, and
  a bad option refused."""
import numpy as np
import pytest

import oracle
from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import synth

pytestmark = pytest.mark.gpu

MU = 1.0
MODES = [(B.CORR_NONE, oracle.NONE), (B.CORR_SI, oracle.SI), (B.CORR_CG, oracle.CG),
         (B.CORR_DENSE, oracle.DENSE)]
ALL = 1 | 2 | 4 | 8


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def close(a, b, tol):
    return rel(a, b) <= tol and np.max(np.abs(a - b)) <= tol * np.max(np.abs(b))


def make(prob, mode=B.CORR_CG, **kw):
    P = B.Problem.from_problem(prob)
    P.factor(mu=MU, correction=mode, **kw)
    return P


def oracle_factor(prob, mode, steps=2):
    f = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, mu=MU)
    f.set_correction(mode, steps)
    return f


def check_solve(prob, res, ref):
    assert res.status == 0 and ref.status == 0
    near = abs(ref.ratio_hist[-1] / 1e-8 - 1) < 1e-3 or abs(res.info["ratio"] / 1e-8 - 1) < 1e-3
    assert abs(res.info["iterations"] - ref.its) <= (1 if near else 0)
    assert rel(res.x, ref.x) <= 1e-6
    A = prob.to_scipy()
    r = prob.b - A @ res.x
    assert np.linalg.norm(A.T @ r) / (res.info["anorm"] * np.linalg.norm(r)) < 1.001e-8


@pytest.fixture(scope="module")
def cfg0():
    return synth.config_problem(0)


@pytest.fixture(scope="module")
def mid():
    return synth.sparse_problem(100_003, 50_001, 8, seed=1, hidden_diag=True)


def test_layout_reported_and_option_checked(cfg0):
    assert make(cfg0, sliced=1).info()["sliced_products"] == ALL
    assert make(cfg0, sliced=0).info()["sliced_products"] == 0
    assert make(cfg0).info()["sliced_products"] == 0  # default without autotuning: CSR
    assert make(cfg0, B.CORR_NONE, sliced=1).info()["sliced_products"] == ALL
    with pytest.raises(B.RlsqError) as e:
        make(cfg0, sliced=2)
    assert e.value.code == -1


@pytest.mark.parametrize("modes", MODES, ids=["NONE", "SI", "CG", "DENSE"])
def test_apply_fp64(cfg0, modes):
    bm, om = modes
    P = make(cfg0, bm, sliced=1)
    f = oracle_factor(cfg0, om)
    s = np.random.default_rng(41).standard_normal(cfg0.n)
    assert close(P.apply(s), f.apply(s), 1e-12)


def test_apply_fp32(cfg0):
    P = make(cfg0, B.CORR_CG, sliced=1, precision=B.PREC_FP32)
    f = oracle_factor(cfg0, oracle.CG)
    s = np.random.default_rng(42).standard_normal(cfg0.n)
    assert close(P.apply(s), f.apply(s), 5e-6)


@pytest.mark.parametrize("modes", [MODES[0], MODES[2], MODES[3]], ids=["NONE", "CG", "DENSE"])
def test_solve(cfg0, modes):
    bm, om = modes
    P = make(cfg0, bm, sliced=1)
    ref = oracle.lsmr(oracle_factor(cfg0, om), cfg0.m, cfg0.n, cfg0.rowptr, cfg0.colidx, cfg0.vals, cfg0.b)
    check_solve(cfg0, P.solve(cfg0.b), ref)


def test_solve_plain(cfg0):
    P = make(cfg0, B.CORR_CG, sliced=1)
    ref = oracle.lsmr(None, cfg0.m, cfg0.n, cfg0.rowptr, cfg0.colidx, cfg0.vals, cfg0.b)
    check_solve(cfg0, P.solve(cfg0.b, plain=True), ref)


def test_mid_apply_and_solve(mid):
    P = make(mid, B.CORR_CG, sliced=1)
    f = oracle_factor(mid, oracle.CG)
    s = np.random.default_rng(43).standard_normal(mid.n)
    assert close(P.apply(s), f.apply(s), 1e-12)
    ref = oracle.lsmr(f, mid.m, mid.n, mid.rowptr, mid.colidx, mid.vals, mid.b)
    res = P.solve(mid.b)
    check_solve(mid, res, ref)
    # the CSR layout: the same iterations, x to 1e-10
    csr = make(mid, B.CORR_CG, sliced=0).solve(mid.b)
    assert csr.info["iterations"] == res.info["iterations"] and rel(csr.x, res.x) <= 1e-10


def test_sparse_dense(cfg0):
    prob = synth.sparse_dense_problem(20_000, 10_000, 6, 50, seed=2)
    P = make(prob, B.CORR_CG, sliced=1)
    assert P.info()["n_dense_rows"] == 50 and P.info()["sliced_products"] == ALL
    ref = oracle.lsmr(oracle_factor(prob, oracle.CG), prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, prob.b)
    check_solve(prob, P.solve(prob.b), ref)


def test_autotuned_layout(cfg0):
    P = make(cfg0, B.CORR_CG, autotune=2)
    print("autotuned sliced products:", P.info()["sliced_products"])
    ref = oracle.lsmr(oracle_factor(cfg0, oracle.CG), cfg0.m, cfg0.n, cfg0.rowptr, cfg0.colidx, cfg0.vals, cfg0.b)
    check_solve(cfg0, P.solve(cfg0.b), ref)
    assert make(cfg0, B.CORR_CG, autotune=2, sliced=0).info()["sliced_products"] == 0
