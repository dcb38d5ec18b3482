"""The pipelined ILUP column loop (several host threads) must give the same
factor, bit for bit, as the one-thread loop, for every parameter choice and
on the degenerate paths: Algorithm 6 pivots (empty columns, tiny pivots),
fewer columns than threads, p = 0 and no entry limit (which always runs on
one thread).  The one-thread loop is itself pinned to the oracle in
test_host_setup.py; one threaded case is compared with the oracle here too."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import synth


def setup_arrays(prob, threads, **kw):
    s = B.HostSetup(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, host_threads=threads, **kw)
    out = {"sizes": s.sizes()}
    out["split"] = s.split()
    for name, part in (("L1", B.PART_L1), ("L2", B.PART_L2), ("U", B.PART_U)):
        out[name] = s.factor_csr(part)
    for name, which in (("lev_L1", B.SYS_L1), ("lev_L1t", B.SYS_L1T), ("lev_U", B.SYS_U), ("lev_Ut", B.SYS_UT)):
        out[name] = s.levels(which)
    return out


def assert_same(a, b):
    assert a["sizes"] == b["sizes"]
    for key in a:
        if key == "sizes":
            continue
        for x, y in zip(a[key], b[key]) if isinstance(a[key], tuple) else [(a[key], b[key])]:
            assert x.dtype == y.dtype and x.shape == y.shape, key
            assert np.array_equal(x.view(np.uint8), y.view(np.uint8)), key  # bits, not values


def assert_oracle(prob, got, **kw):
    okw = {k: v for k, v in kw.items() if k in ("p", "tau", "mu", "small")}
    f = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, scale=kw.get("scale_columns", 1), **okw)
    oprow, oa2 = f.perm()
    assert np.array_equal(got["split"][0], oprow) and np.array_equal(got["split"][1], oa2)
    oU, oud = f.U()
    assert np.array_equal(got["split"][3], oud)
    assert got["sizes"]["nmod"] == f.sizes()["nmod"]
    for name, ref in (("L1", f.L1()), ("L2", f.L2()), ("U", oU)):
        ptr, idx, val = got[name]
        assert np.array_equal(ptr, ref.ptr) and np.array_equal(idx, ref.idx) and np.array_equal(val, ref.val)


def from_dense(A):
    S = sp.csr_matrix(A)
    m, n = A.shape
    return synth.Problem(m, n, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data,
                         np.zeros(m), np.zeros(n), np.zeros(0, dtype=np.int64))


@pytest.mark.parametrize("mu", [0.1, 1.0])
@pytest.mark.parametrize("p,tau", [(10, 1e-2), (3, 0.0), (1, 1e-3), (0, 1e-2), (25, 0.3)])
def test_threads_bitexact_config0(mu, p, tau):
    prob = synth.config_problem(0)
    ref = setup_arrays(prob, 1, p=p, tau=tau, mu=mu)
    for t in (2, 3, 8):
        assert_same(setup_arrays(prob, t, p=p, tau=tau, mu=mu), ref)


@pytest.mark.parametrize("seed", range(12))
def test_threads_bitexact_random(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 300))
    m = n + int(rng.integers(1, 2 * n + 2))
    d = int(rng.integers(1, min(n, 9) + 1))
    prob = synth.sparse_problem(m, n, d, seed=2000 + seed)
    kw = dict(p=int(rng.choice([0, 1, 2, 5, 10, 40])), tau=float(rng.choice([0.0, 1e-3, 1e-2, 0.1])),
              mu=float(rng.choice([0.05, 0.1, 0.5, 1.0])), scale_columns=int(rng.integers(0, 2)))
    ref = setup_arrays(prob, 1, **kw)
    for t in (2, 5, 16):
        assert_same(setup_arrays(prob, t, **kw), ref)


def test_threads_bitexact_modified_pivots():
    """Algorithm 6 on the threaded path.  Column 0 has one entry, so its L
    column is empty; column 1's only entry lies in column 0's pivot row, so
    no unpivoted row has a nonzero there (the empty-column rule); columns 2
    and 3 are equal, so column 3 is left with tiny values or none once
    column 2 is eliminated without dropping."""
    rng = np.random.default_rng(0)
    m, n = 40, 20
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.25)
    A[:, :2] = 0.0
    A[0, :] = 0.0
    A[0, 0], A[0, 1] = 2.0, 3.0
    for j in range(2, n):
        A[j, j] = 1.5 + j / n
    A[:, 3] = A[:, 2]
    prob = from_dense(A)
    for kw, least in ((dict(p=10, tau=0.0, mu=1.0), 2), (dict(p=2, tau=0.05, mu=0.1), 1),
                      (dict(p=0, tau=0.0, mu=1.0), 1)):
        ref = setup_arrays(prob, 1, **kw)
        assert ref["sizes"]["nmod"] >= least, kw
        for t in (2, 3, 7):
            assert_same(setup_arrays(prob, t, **kw), ref)
        assert_oracle(prob, setup_arrays(prob, 3, **kw), **kw)


def test_threads_more_than_columns():
    prob = synth.sparse_problem(9, 3, 2, seed=7)
    ref = setup_arrays(prob, 1, p=10, tau=0.0, mu=1.0)
    for t in (2, 3, 4, 8, 64):
        assert_same(setup_arrays(prob, t, p=10, tau=0.0, mu=1.0), ref)
    one = synth.sparse_problem(4, 1, 1, seed=8)
    ref = setup_arrays(one, 1, p=10, tau=0.0, mu=1.0)
    assert_same(setup_arrays(one, 8, p=10, tau=0.0, mu=1.0), ref)


def test_threads_without_entry_limit_runs_serially():
    prob = synth.sparse_problem(400, 200, 5, seed=9)
    ref = setup_arrays(prob, 1, p=-1, tau=1e-2, mu=1.0)
    assert_same(setup_arrays(prob, 8, p=-1, tau=1e-2, mu=1.0), ref)


def test_threads_config1_recipe_scaled_vs_oracle():
    """The 2M x 1M recipe at 1/80 scale on 8 threads, against the oracle."""
    prob = synth.sparse_problem(25_001, 12_500, 8, seed=1, hidden_diag=True)
    got = setup_arrays(prob, 8, p=10, tau=1e-2, mu=1.0)
    assert_same(setup_arrays(prob, 1, p=10, tau=1e-2, mu=1.0), got)
    assert_oracle(prob, got, p=10, tau=1e-2, mu=1.0)


def test_thread_count_rule():
    lib = B.load()
    assert lib.rlsq_setup_threads(3, 1000, 500) == 3
    assert lib.rlsq_setup_threads(1000, 1000, 500) == 64
    assert 1 <= lib.rlsq_setup_threads(0, 1000, 500) <= 16
    # working arrays of 16 bytes per row: 2 GiB holds one thread's at 2^27 rows
    assert lib.rlsq_setup_threads(8, 1 << 27, 1 << 20) == 1
    assert lib.rlsq_setup_threads(8, 1 << 25, 1 << 20) == 4


def test_threads_bitexact_blocked_transposes():
    """Large enough (about 800k entries in A) that the set-up's transposes
    split into several blocks of rows on several threads."""
    prob = synth.config_problem(1, scale=0.05)
    assert prob.rowptr[-1] > 2 * (1 << 18)  # at least 3 blocks
    ref = setup_arrays(prob, 1, p=10, tau=1e-2, mu=1.0)
    assert_same(setup_arrays(prob, 8, p=10, tau=1e-2, mu=1.0), ref)


@pytest.mark.parametrize("case", ["sparse_dense", "tall", "long_columns"])
def test_threads_bitexact_stress(case):
    """Heavy columns (dense rows in A), tall matrices (m = 40 n) and long L
    columns (no drop tolerance, p = 60)."""
    if case == "sparse_dense":
        prob, kw = synth.sparse_dense_problem(6000, 3000, 6, 20, seed=2), dict(p=10, tau=1e-2, mu=1.0)
    elif case == "tall":
        prob, kw = synth.sparse_problem(40 * 400, 400, 5, seed=31), dict(p=10, tau=1e-3, mu=0.1)
    else:
        prob, kw = synth.sparse_problem(3000, 1500, 7, seed=32), dict(p=60, tau=0.0, mu=0.5)
    ref = setup_arrays(prob, 1, **kw)
    for t in (3, 8):
        assert_same(setup_arrays(prob, t, **kw), ref)


@pytest.mark.slow
def test_fullsize_config1_threaded_setup_matches_oracle():
    """The headline 2M x 1M recipe at full size (p = 10, tau = 1e-2, mu = 1):
    the threaded host set-up (the library's default thread count) against the
    single-threaded oracle, bit for bit: row selection, A2 rows, scaling, the
    L1, L2 and U arrays and U's diagonal, the level sets of L1 and U (both
    from the oracle's level routine).  About two minutes, mostly the oracle."""
    kw = dict(p=10, tau=1e-2, mu=1.0)
    prob = synth.config_problem(1)
    got = setup_arrays(prob, 0, **kw)
    f = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, **kw)
    oprow, oa2 = f.perm()
    assert np.array_equal(got["split"][0], oprow) and np.array_equal(got["split"][1], oa2)
    assert np.array_equal(got["split"][2], f.scaling())
    oU, oud = f.U()
    assert np.array_equal(got["split"][3], oud)
    oL1 = f.L1()
    for name, ref in (("L1", oL1), ("L2", f.L2()), ("U", oU)):
        ptr, idx, val = got[name]
        assert np.array_equal(ptr, ref.ptr) and np.array_equal(idx, ref.idx) and np.array_equal(val, ref.val)
    assert np.array_equal(got["lev_L1"], oracle.levels(oL1, True)[0])
    assert np.array_equal(got["lev_U"], oracle.levels(oU, False)[0])
