"""GPU CGLS (Algorithm 1) against the oracle's CGLS, through the C ABI.

x-space form (h = M^{-1} A^T r): equal iteration counts (+-1 when the final
ratio sits near the threshold), x within 1e-6 relative, the stopping ratio
below 1e-8; plain CGLS against the oracle's M = I run; bit-identical repeats;
dense-row problems rejected.

Split form (h = Algorithm 3 on the residual split, the paper's): one
application against the oracle's element by element for every correction,
the exact-factor case against lstsq, and the iterates after K steps against
the oracle's."""
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


# ---- Algorithm 3 fed the residual split (Sec. 3.2: the paper's way of
# combining the preconditioner with A^T in steps 3 and 12 of Algorithm 1) ----

ALL_IDS = ["NONE", "SI", "CG", "DENSE"]


def rel_inf(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def oracle_factor(p, om, steps=2):
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, mu=MU)
    f.set_correction(om, steps)
    return f


@pytest.mark.parametrize("modes", MODES, ids=ALL_IDS)
def test_split_apply_matches_oracle(cfg0, modes):
    bm, om = modes
    p = cfg0
    P = B.Problem.from_problem(p)
    P.factor(mu=MU, correction=bm)
    f = oracle_factor(p, om)
    r = np.random.default_rng(31).standard_normal(p.m)
    t, ref = P.apply_residual(r), f.apply_residual(r)
    assert rel(t, ref) <= 1e-12 and rel_inf(t, ref) <= 1e-12
    # the split apply is not the x-space one (A^T r in, M^{-1} A^T r out)
    assert rel(P.apply(P.matvec(r, trans=True)), t) > 1e-3


@pytest.fixture(scope="module")
def mid():
    return synth.sparse_problem(100_003, 50_001, 8, seed=1, hidden_diag=True)


def test_split_apply_mid_problem_fp64_fp32(mid):
    # many level groups and tiles, a ragged tail (n odd); CG(2) correction
    p = mid
    P = B.Problem.from_problem(p)
    P.factor(mu=MU, correction=B.CORR_CG)
    f = oracle_factor(p, oracle.CG)
    r = np.random.default_rng(32).standard_normal(p.m)
    ref = f.apply_residual(r)
    t = P.apply_residual(r)
    assert rel(t, ref) <= 1e-12 and rel_inf(t, ref) <= 1e-12
    # float32 apply: the same 5e-6 bound as the x-space float32 apply
    P.factor(mu=MU, correction=B.CORR_CG, precision=B.PREC_FP32)
    t32 = P.apply_residual(r)
    print(f"split apply FP32: rel {rel(t32, ref):.2e}, elementwise {rel_inf(t32, ref):.2e}")
    assert rel(t32, ref) <= 5e-6


def test_split_exact_factors_least_squares_one_step():
    """Exact LU (nothing dropped) and the dense S^: the split apply is the
    least-squares correction (A^T A)^{-1} A^T r, and CGLS ends after one step
    at the lstsq solution (Sec. 3.1)."""
    p = synth.sparse_problem(70, 45, 4, seed=41)
    P = B.Problem.from_problem(p)
    P.factor(p=-1, tau=0.0, mu=1.0, correction=B.CORR_DENSE)
    A = p.to_scipy().toarray()
    r = np.random.default_rng(33).standard_normal(p.m)
    np.testing.assert_allclose(P.apply_residual(r), np.linalg.lstsq(A, r, rcond=None)[0], rtol=1e-9, atol=1e-10)
    res = P.solve(p.b, solver=B.SOLVER_CGLS_SPLIT, atol=1e-10, maxit=20)
    assert res.status == 0 and res.info["iterations"] == 1
    np.testing.assert_allclose(res.x, np.linalg.lstsq(A, p.b, rcond=None)[0], rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("modes", [MODES[0], MODES[2], MODES[3]], ids=["NONE", "CG", "DENSE"])
def test_cgls_split_matches_oracle_step_by_step(cfg0, modes):
    """With dropped entries the split form stalls (the oracle's pins); the GPU
    follows the oracle's iterates: after K steps x within 1e-9 and the ratio
    within 1e-9 relative (the oracle moves them by 1e-14 / 1e-12 when b is
    perturbed by 1e-14), both ending on the iteration limit."""
    bm, om = modes
    p = cfg0
    P = B.Problem.from_problem(p)
    P.factor(mu=MU, correction=bm)
    f = oracle_factor(p, om)
    anorm = P.info()["anorm"]
    for K in (1, 3, 10, 30, 100):
        res = P.solve(p.b, solver=B.SOLVER_CGLS_SPLIT, maxit=K, allow_fail=True)
        ref = oracle.cgls(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, anorm=anorm, atol=1e-8, maxit=K)
        assert ref.status == 1 and res.status == -8 and res.info["iterations"] == K, K
        assert abs(res.info["ratio"] - ref.ratio) <= 1e-9 * ref.ratio, K
        assert rel(res.x, ref.x) <= 1e-9, K
    assert res.info["ratio"] > 1e-3  # stalled, as in the oracle


def test_cgls_split_mid_problem(mid):
    p = mid
    P = B.Problem.from_problem(p)
    P.factor(mu=MU, correction=B.CORR_CG)
    f = oracle_factor(p, oracle.CG)
    K = 20
    res = P.solve(p.b, solver=B.SOLVER_CGLS_SPLIT, maxit=K, allow_fail=True)
    ref = oracle.cgls(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, anorm=P.info()["anorm"], atol=1e-8, maxit=K)
    assert res.info["iterations"] == ref.its
    assert abs(res.info["ratio"] - ref.ratio) <= 1e-9 * ref.ratio
    assert rel(res.x, ref.x) <= 1e-9


def test_cgls_split_deterministic_plain_and_rejections(cfg0):
    p = cfg0
    P = B.Problem.from_problem(p)
    P.factor(mu=MU, correction=B.CORR_CG)
    a = P.solve(p.b, solver=B.SOLVER_CGLS_SPLIT, maxit=40, allow_fail=True)
    b = P.solve(p.b, solver=B.SOLVER_CGLS_SPLIT, maxit=40, allow_fail=True)
    assert np.array_equal(a.x, b.x) and a.info["ratio"] == b.info["ratio"]
    # M = I: the split form is plain CGLS
    u = P.solve(p.b, plain=True, solver=B.SOLVER_CGLS_SPLIT)
    v = P.solve(p.b, plain=True, solver=B.SOLVER_CGLS)
    assert np.array_equal(u.x, v.x) and u.info["iterations"] == v.info["iterations"]
    d = synth.sparse_dense_problem(3000, 1000, 6, 4, seed=9)
    Q = B.Problem.from_problem(d)
    Q.factor(mu=MU, correction=B.CORR_CG)
    for call in (lambda: Q.solve(d.b, solver=B.SOLVER_CGLS_SPLIT), lambda: Q.apply_residual(d.b)):
        with pytest.raises(B.RlsqError) as e:
            call()
        assert e.value.code == -1
