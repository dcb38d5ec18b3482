"""Pins for the CPU oracle: each test checks the oracle against something
other than itself -- a closed form, a dense library routine, a brute-force
replica on tiny inputs, or an invariant the mathematics fixes -- so that a
dropped term, a wrong sign or index, or a transposed operand fails one of
them."""

import numpy as np
import pytest

import oracle
from paper_2603_28642_gb300 import synth


def dense(p):
    return p.to_scipy().toarray()


def factors_dense(f):
    n = f.n
    prow, a2 = f.perm()
    L1 = f.L1().to_scipy().toarray() + np.eye(n)
    L2 = f.L2().to_scipy().toarray()
    Uc, ud = f.U()
    U = Uc.to_scipy().toarray() + np.diag(ud)
    return prow, a2, L1, L2, U, f.scaling()


def tiny_problems():
    out = []
    for seed, (m, n, d) in enumerate([(12, 8, 3), (20, 15, 4), (30, 10, 3), (40, 25, 5),
                                      (60, 40, 4), (9, 8, 2)]):
        out.append(synth.sparse_problem(m, n, d, seed=100 + seed))
    return out


# ---------------------------------------------------------------------------
# column scaling (Sec. 5.1)
# ---------------------------------------------------------------------------
def test_column_scaling_unit_norms():
    p = synth.config_problem(0)
    d = oracle.column_scaling(p.m, p.n, p.rowptr, p.colidx, p.vals)
    A = dense(p)
    np.testing.assert_allclose(np.linalg.norm(A * d, axis=0), 1.0, rtol=1e-14)


def test_empty_column_rejected():
    p = synth.sparse_problem(10, 6, 2, seed=3)
    A = dense(p)
    A[:, 2] = 0.0
    import scipy.sparse as sp

    S = sp.csr_matrix(A)
    S.eliminate_zeros()
    with pytest.raises(ValueError):
        oracle.Factor(10, 6, S.indptr, S.indices, S.data)


# ---------------------------------------------------------------------------
# ILUP: no dropping reduces to the exact threshold-pivoted LU (eq. 2.1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prob", tiny_problems(), ids=lambda p: f"{p.m}x{p.n}")
@pytest.mark.parametrize("mu", [0.1, 1.0])
def test_nodrop_is_exact_lu(prob, mu):
    f = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, p=-1, tau=0.0, mu=mu)
    prow, a2, L1, L2, U, d = factors_dense(f)
    Ah = dense(prob) * d
    assert sorted(np.concatenate([prow, a2]).tolist()) == list(range(prob.m))
    assert np.all(np.diff(a2) > 0)
    scale = np.abs(Ah).max()
    np.testing.assert_allclose(L1 @ U, Ah[prow], atol=1e-13 * scale * prob.n)
    np.testing.assert_allclose(L2 @ U, Ah[a2], atol=1e-13 * scale * prob.n)
    # threshold pivoting bounds the multipliers by 1/mu
    assert np.abs(L1).max() <= 1.0 / mu + 1e-12
    assert (np.abs(L2).max() if L2.size else 0.0) <= 1.0 / mu + 1e-12
    assert f.sizes()["nmod"] == 0


# ---------------------------------------------------------------------------
# ILUP with dropping vs a pure-Python dense replica of Algorithms 4-6
# ---------------------------------------------------------------------------
def ilup_dense_reference(Ah, p, tau, mu, small):
    """Algorithm 4 on a small dense matrix, one column at a time, written
    independently of the C oracle (dense arrays, no heap, no stamps)."""
    m, n = Ah.shape
    rc = (Ah != 0).sum(axis=1).astype(np.int64)
    pivpos = -np.ones(m, dtype=np.int64)
    prow = np.zeros(n, dtype=np.int64)
    L = np.zeros((m, n))
    Ucols = []
    udiag = np.zeros(n)
    nmod = 0
    for j in range(n):
        x = Ah[:, j].copy()
        uvals = {}
        for k in range(j):
            ukj = x[prow[k]]
            if ukj == 0.0:
                continue
            uvals[k] = ukj
            for i in range(m):
                if L[i, k] != 0.0:
                    x[i] = x[i] - L[i, k] * ukj
        kept = [(abs(v), k, v) for k, v in uvals.items() if abs(v) >= tau]
        if p >= 0 and len(kept) > p:
            kept.sort(key=lambda t: (-t[0], t[1]))
            kept = kept[:p]
        Ucols.append({k: v for _, k, v in kept})
        beta = 10.0 ** (-2.0 * (1.0 - (j + 1) / n))
        modval = max(beta * np.abs(Ah[:, j]).max(), small)
        cands = [i for i in range(m) if pivpos[i] < 0 and x[i] != 0.0]
        if not cands:
            free = [i for i in range(m) if pivpos[i] < 0]
            r = min(free, key=lambda i: (rc[i], i))
            piv = modval
            nmod += 1
        else:
            mx = max(abs(x[i]) for i in cands)
            R = [i for i in cands if abs(x[i]) >= mu * mx]
            r = min(R, key=lambda i: (rc[i], -abs(x[i]), i))
            piv = x[r]
            if abs(piv) < small:
                piv = -modval if piv < 0 else modval
                nmod += 1
        udiag[j] = piv
        pivpos[r] = j
        prow[j] = r
        lk = [(abs(x[i] / piv), i, x[i] / piv) for i in cands if i != r]
        lk = [t for t in lk if t[0] >= tau and t[2] != 0.0]
        if p >= 0 and len(lk) > p:
            lk.sort(key=lambda t: (-t[0], t[1]))
            lk = lk[:p]
        for _, i, v in lk:
            L[i, j] = v
        for i in range(m):
            if Ah[i, j] != 0.0:
                rc[i] -= 1
    U = np.zeros((n, n))
    for j, col in enumerate(Ucols):
        for k, v in col.items():
            U[k, j] = v
        U[j, j] = udiag[j]
    return prow, L, U, nmod


@pytest.mark.parametrize("prob", tiny_problems(), ids=lambda p: f"{p.m}x{p.n}")
@pytest.mark.parametrize("params", [(2, 0.05, 0.1), (3, 0.0, 1.0), (1, 0.2, 0.5), (2, 0.3, 0.1)])
def test_ilup_matches_dense_replica(prob, params):
    pp, tau, mu = params
    small = 1e-10
    f = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, p=pp, tau=tau, mu=mu,
                      small=small)
    prow, a2, L1, L2, U, d = factors_dense(f)
    Ah = dense(prob) * d
    rprow, rL, rU, rnmod = ilup_dense_reference(Ah, pp, tau, mu, small)
    assert np.array_equal(prow, rprow)
    assert f.sizes()["nmod"] == rnmod
    # bit-exact values: same arithmetic in the same order
    assert np.array_equal(L1 - np.eye(prob.n), rL[prow])
    assert np.array_equal(L2, rL[a2])
    assert np.array_equal(U, rU)


@pytest.mark.parametrize("params", [(2, 0.05, 0.1), (3, 0.01, 1.0)])
def test_drop_rules_hold(params):
    """Per-column rules of Algorithm 4: every kept entry has |.| >= tau and
    each column of L and of U holds at most p off-diagonal entries."""
    pp, tau, mu = params
    prob = synth.sparse_problem(200, 120, 5, seed=7)
    f = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, p=pp, tau=tau, mu=mu)
    prow, a2, L1, L2, U, d = factors_dense(f)
    Lfull = np.vstack([L1 - np.eye(prob.n), L2])
    Uoff = U - np.diag(np.diag(U))
    for M in (Lfull, Uoff):
        nz = M[M != 0]
        assert np.all(np.abs(nz) >= tau)
        assert ((M != 0).sum(axis=0) <= pp).all()


def test_pivot_modification_empty_column():
    """Algorithm 6: a column that is empty after dropping gets the pivot
    max(beta ||A_:,j||_inf, small) with beta = 10^(-2(1 - j/n))."""
    # columns 0 and 1 are identical: with exact elimination column 1 becomes
    # zero, so its pivot must be modified.
    A = np.array([[1.0, 1.0, 0.0],
                  [2.0, 2.0, 1.0],
                  [0.0, 0.0, 3.0],
                  [1.0, 1.0, 1.0]])
    import scipy.sparse as sp

    S = sp.csr_matrix(A)
    f = oracle.Factor(4, 3, S.indptr, S.indices, S.data, p=-1, tau=0.0, mu=1.0, small=1e-10)
    _, _, _, _, U, d = factors_dense(f)
    assert f.sizes()["nmod"] == 1
    beta = 10.0 ** (-2.0 * (1.0 - 2.0 / 3.0))
    colinf = np.abs(A[:, 1] * d[1]).max()
    assert U[1, 1] == pytest.approx(max(beta * colinf, 1e-10), rel=1e-15)


def test_pivot_choice_prefers_sparse_rows():
    """Algorithm 5: among entries within mu of the largest, the row with the
    smallest remaining row count wins."""
    A = np.array([[1.0, 1.0, 1.0],
                  [0.5, 0.0, 0.0],
                  [0.0, 1.0, 0.0],
                  [0.0, 0.0, 1.0]])
    import scipy.sparse as sp

    S = sp.csr_matrix(A)
    f = oracle.Factor(4, 3, S.indptr, S.indices, S.data, p=-1, tau=0.0, mu=0.1)
    prow, _ = f.perm()
    assert prow[0] == 1  # |0.5| >= 0.1 * 1, and row 1 has one entry
    f2 = oracle.Factor(4, 3, S.indptr, S.indices, S.data, p=-1, tau=0.0, mu=1.0)
    assert f2.perm()[0][0] == 0  # mu = 1: only the largest entry qualifies


# ---------------------------------------------------------------------------
# level sets: brute-force longest path
# ---------------------------------------------------------------------------
def _longest_path_levels(M, lower):
    n = M.shape[0]
    memo = {}

    def lev(i):
        if i in memo:
            return memo[i]
        deps = [k for k in range(n) if M[i, k] != 0 and ((k < i) if lower else (k > i))]
        memo[i] = 0 if not deps else 1 + max(lev(k) for k in deps)
        return memo[i]

    return np.array([lev(i) for i in range(n)])


def test_levels_brute_force():
    prob = synth.sparse_problem(90, 60, 4, seed=11)
    f = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, p=10, tau=1e-2, mu=1.0)
    L1 = f.L1()
    U, _ = f.U()
    import scipy.sparse as sp

    for csr, lower in ((L1, True), (U, False)):
        lev, nl = oracle.levels(csr, lower)
        ref = _longest_path_levels(csr.to_scipy().toarray(), lower)
        assert np.array_equal(lev, ref)
        assert nl == ref.max() + 1
        # transposed system
        T = csr.to_scipy().T.tocsr()
        tc = oracle.CSR(T.indptr.astype(np.int64), T.indices.astype(np.int32), T.data, T.shape)
        lev_t, _ = oracle.levels(tc, not lower)
        assert np.array_equal(lev_t, _longest_path_levels(T.toarray(), not lower))
    del sp


# ---------------------------------------------------------------------------
# products, solves and adjointness
# ---------------------------------------------------------------------------
def test_spmv_against_scipy_and_adjoint():
    p = synth.config_problem(0)
    A = p.to_scipy()
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(p.n), rng.standard_normal(p.m)
    ax = oracle.spmv(p.m, p.rowptr, p.colidx, p.vals, x)
    aty = oracle.spmv_t(p.m, p.n, p.rowptr, p.colidx, p.vals, y)
    np.testing.assert_allclose(ax, A @ x, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(aty, A.T @ y, rtol=1e-13, atol=1e-13)
    assert np.dot(ax, y) == pytest.approx(np.dot(x, aty), rel=1e-12)


@pytest.fixture(scope="module")
def cfg0_factor():
    p = synth.config_problem(0)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, p=10, tau=1e-2, mu=1.0)
    return p, f


def test_triangular_solves_and_adjoints(cfg0_factor):
    p, f = cfg0_factor
    prow, a2, L1, L2, U, d = factors_dense(f)
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal(p.n), rng.standard_normal(p.n)
    np.testing.assert_allclose(L1 @ f.solve_L1(a), a, atol=1e-10)
    np.testing.assert_allclose(L1.T @ f.solve_L1t(a), a, atol=1e-10)
    np.testing.assert_allclose(U @ f.solve_U(a), a, atol=1e-10)
    np.testing.assert_allclose(U.T @ f.solve_Ut(a), a, atol=1e-10)
    assert np.dot(f.solve_L1(a), b) == pytest.approx(np.dot(a, f.solve_L1t(b)), rel=1e-11)
    assert np.dot(f.solve_U(a), b) == pytest.approx(np.dot(a, f.solve_Ut(b)), rel=1e-11)


def _dense_minv(f, p, mode, steps=2):
    """M^{-1} from its definition with dense numpy algebra."""
    prow, a2, L1, L2, U, d = factors_dense(f)
    n = p.n
    Y = L2 @ np.linalg.inv(L1)
    if mode == oracle.NONE:
        K = np.eye(n)
    elif mode == oracle.SI:
        K = np.eye(n) - Y.T @ Y
    elif mode == oracle.DENSE:
        K = np.linalg.inv(np.eye(n) + Y.T @ Y)  # Woodbury, Lemma 3.1
    else:
        raise ValueError
    Uinv = np.linalg.inv(U)
    L1inv = np.linalg.inv(L1)
    D = np.diag(d)
    return D @ Uinv @ L1inv @ K @ L1inv.T @ Uinv.T @ D, Y


@pytest.mark.parametrize("mode", [oracle.NONE, oracle.SI, oracle.DENSE])
def test_apply_matches_dense_definition(cfg0_factor, mode):
    p, f = cfg0_factor
    f.set_correction(mode)
    Minv, _ = _dense_minv(f, p, mode)
    rng = np.random.default_rng(2)
    for _ in range(3):
        s = rng.standard_normal(p.n)
        t = f.apply(s)
        np.testing.assert_allclose(t, Minv @ s, rtol=1e-9, atol=1e-9 * np.abs(Minv @ s).max())
    # symmetry of the linear modes
    a, b = rng.standard_normal(p.n), rng.standard_normal(p.n)
    assert np.dot(f.apply(a), b) == pytest.approx(np.dot(a, f.apply(b)), rel=1e-10)


def test_cg_adaptive_steps_match_dense_cg(cfg0_factor):
    """CG on S stopped adaptively (after the step that brings ||r_j|| to at
    most tol ||r_0||, at most k steps): the number of steps and w equal CG
    written on the dense S = I + Y Y^T; tol = 0 keeps k steps; a whole apply
    with the adaptive rule equals the fixed-k apply with the steps it took."""
    p, f = cfg0_factor
    _, Y = _dense_minv(f, p, oracle.NONE)
    S = np.eye(Y.shape[0]) + Y @ Y.T
    kmax = 25
    for tol in (0.5, 0.1, 1e-2, 1e-4, 0.0):
        f.set_correction(oracle.CG, kmax, cg_tol=tol)
        e = np.random.default_rng(int(1000 * tol) + 3).standard_normal(Y.shape[0])
        w = np.zeros_like(e)
        r = e.copy()
        pv = e.copy()
        rr = r @ r
        rr0 = rr
        steps = 0
        for it in range(kmax):
            sp_ = S @ pv
            a = rr / (pv @ sp_)
            w += a * pv
            r -= a * sp_
            steps = it + 1
            rrn = r @ r
            if tol > 0 and rrn <= tol * tol * rr0:
                # not a borderline decision (the oracle's sums are ordered differently)
                assert rrn < (1 - 1e-9) * tol * tol * rr0
                break
            pv = r + rrn / rr * pv
            rr = rrn
        got = f.s_solve(e)
        assert f.cg_last_steps() == steps, (tol, f.cg_last_steps(), steps)
        np.testing.assert_allclose(got, w, rtol=1e-9, atol=1e-11)
        assert (tol > 0 and steps < kmax) or (tol == 0 and steps == kmax)
    # the apply: adaptive == fixed with the same number of steps, bit for bit
    s = np.random.default_rng(77).standard_normal(p.n)
    f.set_correction(oracle.CG, 10, cg_tol=0.05)
    t_adapt = f.apply(s)
    k = f.cg_last_steps()
    assert 1 <= k < 10
    f.set_correction(oracle.CG, k)
    assert np.array_equal(f.apply(s), t_adapt)


def test_cg_mode_matches_dense_cg(cfg0_factor):
    """CG(k) on S = I + Y Y^T from zero: compare with CG written on the dense S."""
    p, f = cfg0_factor
    for k in (1, 2, 3):
        f.set_correction(oracle.CG, k)
        _, Y = _dense_minv(f, p, oracle.NONE)
        S = np.eye(Y.shape[0]) + Y @ Y.T
        e = np.random.default_rng(k).standard_normal(Y.shape[0])
        w = np.zeros_like(e)
        r = e.copy()
        pv = e.copy()
        rr = r @ r
        for _ in range(k):
            sp_ = S @ pv
            a = rr / (pv @ sp_)
            w += a * pv
            r -= a * sp_
            rrn = r @ r
            pv = r + rrn / rr * pv
            rr = rrn
        np.testing.assert_allclose(f.s_solve(e), w, rtol=1e-10, atol=1e-12)
        # positivity of <s, M^{-1} s> under CG(k)
        s = np.random.default_rng(10 + k).standard_normal(p.n)
        assert np.dot(s, f.apply(s)) > 0


def test_dense_mode_cholesky(cfg0_factor):
    p, f = cfg0_factor
    f.set_correction(oracle.DENSE)
    G = f.dense_cholesky()
    _, Y = _dense_minv(f, p, oracle.NONE)
    S = np.eye(Y.shape[0]) + Y @ Y.T
    np.testing.assert_allclose(G @ G.T, S, rtol=1e-12, atol=1e-12)
    assert np.allclose(G, np.tril(G))


def test_nodrop_dense_apply_is_least_squares_solution():
    """Sec. 3.1: with the exact LU and the dense S, one application to A^T b
    gives the least-squares solution."""
    p = synth.sparse_problem(60, 40, 4, seed=21)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, p=-1, tau=0.0, mu=0.1)
    f.set_correction(oracle.DENSE)
    A = dense(p)
    x_ls = np.linalg.lstsq(A, p.b, rcond=None)[0]
    np.testing.assert_allclose(f.apply(A.T @ p.b), x_ls, rtol=1e-10, atol=1e-11)


def test_nodrop_none_mode_inverts_A1():
    """M = A1 exactly when nothing is dropped: (L1 U D^{-1})^{-1} inverts A1."""
    p = synth.sparse_problem(45, 30, 4, seed=22)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, p=-1, tau=0.0, mu=0.5)
    prow, a2, L1, L2, U, d = factors_dense(f)
    A1 = dense(p)[prow]
    MR_inv = np.diag(d) @ np.linalg.inv(U) @ np.linalg.inv(L1)
    np.testing.assert_allclose(A1 @ MR_inv, np.eye(p.n), atol=1e-11)
    # the oracle's NONE apply equals (A1^T A1)^{-1}
    f.set_correction(oracle.NONE)
    s = np.random.default_rng(3).standard_normal(p.n)
    np.testing.assert_allclose(f.apply(s), np.linalg.solve(A1.T @ A1, s), rtol=1e-9, atol=1e-10)


# ---------------------------------------------------------------------------
# power method and LSMR
# ---------------------------------------------------------------------------
def test_power_method_norm():
    p = synth.config_problem(0)
    est = oracle.norm2(p.m, p.n, p.rowptr, p.colidx, p.vals, iters=300)
    ref = np.linalg.norm(dense(p), 2)
    assert est == pytest.approx(ref, rel=1e-6)
    est50 = oracle.norm2(p.m, p.n, p.rowptr, p.colidx, p.vals, iters=50)
    assert est50 <= ref * (1 + 1e-12) and est50 > 0.9 * ref


@pytest.mark.parametrize("prob", tiny_problems()[:5], ids=lambda p: f"{p.m}x{p.n}")
def test_unpreconditioned_lsmr_vs_lstsq(prob):
    A = dense(prob)
    x_ls = np.linalg.lstsq(A, prob.b, rcond=None)[0]
    r = oracle.lsmr(None, prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, prob.b,
                    atol=1e-10, maxit=500)
    # the ratio's attainable floor is about eps ||x|| / ||r||, ~1e-12 here
    assert r.status == 0
    np.testing.assert_allclose(r.x, x_ls, rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("mode", [oracle.NONE, oracle.DENSE, oracle.CG])
def test_preconditioned_lsmr_config0(mode, cfg0_factor):
    p, f = cfg0_factor
    f.set_correction(mode, 2)
    A = dense(p)
    x_ls = np.linalg.lstsq(A, p.b, rcond=None)[0]
    r = oracle.lsmr(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, atol=1e-8, maxit=2000)
    assert r.status == 0 and r.its < 100
    # the stopping ratio recomputed from scratch (normal-equation optimality)
    res = p.b - A @ r.x
    ratio = np.linalg.norm(A.T @ res) / (np.linalg.norm(A, 2) * np.linalg.norm(res))
    assert ratio < 1.001e-8
    np.testing.assert_allclose(r.x, x_ls, rtol=1e-6)


def test_exact_preconditioner_converges_in_one_step():
    p = synth.sparse_problem(80, 50, 4, seed=31)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, p=-1, tau=0.0, mu=1.0)
    f.set_correction(oracle.DENSE)
    r = oracle.lsmr(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, atol=1e-10, maxit=50)
    assert r.status == 0 and r.its == 1


def test_si_mode_reports_breakdown_when_indefinite():
    """With S^ = I, K = I - Y^T Y is indefinite once ||Y|| > 1; LSMR must then
    report a breakdown instead of producing a result."""
    p = synth.config_problem(0)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, p=10, tau=1e-2, mu=0.1)
    f.set_correction(oracle.SI)
    r = oracle.lsmr(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b)
    assert r.status == -2


def test_zero_rhs():
    p = synth.config_problem(0)
    r = oracle.lsmr(None, p.m, p.n, p.rowptr, p.colidx, p.vals, np.zeros(p.m))
    assert r.status == 0 and r.its == 0 and not r.x.any()


def test_ratio_history_is_explicit():
    """ratio_k is the explicitly recomputed ||A^T r_k|| / (||A|| ||r_k||)."""
    p = synth.config_problem(0)
    anorm = oracle.norm2(p.m, p.n, p.rowptr, p.colidx, p.vals)
    r = oracle.lsmr(None, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, anorm=anorm, maxit=5,
                    atol=0.0)
    A = dense(p)
    assert r.status == 1 and r.its == 5
    res = p.b - A @ r.x
    assert r.ratio_hist[-1] == pytest.approx(
        np.linalg.norm(A.T @ res) / (anorm * np.linalg.norm(res)), rel=1e-10)
    assert r.ratio_hist[0] == pytest.approx(
        np.linalg.norm(A.T @ p.b) / (anorm * np.linalg.norm(p.b)), rel=1e-12)
