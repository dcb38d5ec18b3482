"""GPU CGLS (Algorithm 1 with h = M^{-1} A^T r) against the oracle's CGLS in
the same form, through the C ABI: equal iteration counts (+-1 when the final
ratio sits near the threshold), x within 1e-6 relative, the stopping ratio
below 1e-8; plain CGLS against the oracle's M = I run; bit-identical repeats;
dense-row problems rejected."""
import numpy as np
import pytest

import oracle
from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import synth

pytestmark = pytest.mark.gpu

MU = 1.0
MODES = [(B.CORR_NONE, oracle.NONE), (B.CORR_SI, oracle.SI), (B.CORR_CG, oracle.CG), (B.CORR_DENSE, oracle.DENSE)]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def cfg0():
    return synth.config_problem(0)


@pytest.mark.parametrize("modes", [MODES[0], MODES[2], MODES[3]], ids=["NONE", "CG", "DENSE"])
def test_cgls_matches_oracle(cfg0, modes):
    bm, om = modes
    p = cfg0
    P = B.Problem.from_problem(p)
    P.factor(mu=MU, correction=bm)
    res = P.solve(p.b, solver=B.SOLVER_CGLS)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=MU)
    f.set_correction(om, 2)
    ref = oracle.cgls(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, form="symmetric")
    assert res.status == 0 and ref.status == 0
    assert abs(res.info["iterations"] - ref.its) <= 1
    assert res.info["ratio"] < 1e-8
    assert rel(res.x, ref.x) <= 1e-6
    # the same x as LSMR to the solution's accuracy
    ls = P.solve(p.b)
    assert rel(res.x, ls.x) <= 1e-6


def test_cgls_mid_problem():
    p = synth.sparse_problem(100_003, 50_001, 8, seed=1, hidden_diag=True)
    P = B.Problem.from_problem(p)
    P.factor(mu=MU, correction=B.CORR_CG)
    res = P.solve(p.b, solver=B.SOLVER_CGLS)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=MU)
    f.set_correction(oracle.CG, 2)
    ref = oracle.cgls(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, form="symmetric")
    assert res.status == 0 and ref.status == 0
    assert abs(res.info["iterations"] - ref.its) <= 1
    assert rel(res.x, ref.x) <= 1e-6


def test_plain_cgls_matches_oracle(cfg0):
    p = cfg0
    P = B.Problem.from_problem(p)
    res = P.solve(p.b, plain=True, solver=B.SOLVER_CGLS)
    ref = oracle.cgls(None, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b)
    assert res.status == 0 and ref.status == 0
    assert abs(res.info["iterations"] - ref.its) <= 1
    assert rel(res.x, ref.x) <= 1e-6


def test_cgls_deterministic_and_maxit(cfg0):
    P = B.Problem.from_problem(cfg0)
    P.factor(mu=MU, correction=B.CORR_CG)
    a = P.solve(cfg0.b, solver=B.SOLVER_CGLS)
    b = P.solve(cfg0.b, solver=B.SOLVER_CGLS)
    assert np.array_equal(a.x, b.x) and a.info["iterations"] == b.info["iterations"]
    c = P.solve(cfg0.b, solver=B.SOLVER_CGLS, maxit=3, allow_fail=True)
    assert c.status == -8 and c.info["iterations"] == 3


def test_cgls_rejects_dense_rows_and_bad_solver(cfg0):
    p = synth.sparse_dense_problem(3000, 1000, 6, 4, seed=9)
    P = B.Problem.from_problem(p)
    P.factor(mu=MU, correction=B.CORR_CG)
    assert P.info()["n_dense_rows"] > 0
    with pytest.raises(B.RlsqError) as e:
        P.solve(p.b, solver=B.SOLVER_CGLS)
    assert e.value.code == -1
    Q = B.Problem.from_problem(cfg0)
    Q.factor(mu=MU)
    with pytest.raises(B.RlsqError):
        Q.solve(cfg0.b, solver=7)
