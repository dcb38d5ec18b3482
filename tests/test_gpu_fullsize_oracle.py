"""The 2M x 1M workload at full size against the oracle itself, in the launch
configuration bench.py times (ILUP(p=10, tau=1e-2, mu=1), CG(2), level groups
chosen by the cost model, mapping autotuned).

The oracle factors the matrix single-threaded (about two minutes); then:

* the structure the GPU handle holds -- row selection, A2 rows, column
  scaling, the L1, L2 and U arrays (values included) and the level sets of
  L1, L1^T, U, U^T -- equals the oracle's bit for bit;
* one float64 preconditioner application equals the oracle's within 1e-12
  relative, in the 2-norm and element by element (max-norm);
* one float32 application is within 2e-6 relative (2-norm and max-norm),
  about 10x the error measured on GB300 (1.6e-7, elementwise 2.0e-7).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import synth

pytestmark = pytest.mark.gpu

FACTOR = dict(p=10, tau=1e-2, mu=1.0, correction=B.CORR_CG, cg_steps=2, autotune=1)


@pytest.fixture(scope="module")
def full():
    prob = synth.config_problem(1)
    f = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, p=10, tau=1e-2, mu=1.0)
    f.set_correction(oracle.CG, 2)
    P = B.Problem.from_problem(prob)
    P.factor(**FACTOR)
    return prob, f, P


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def rel_inf(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_fullsize_structure_bitexact(full):
    prob, f, P = full
    prow, a2, d, ud = P.split()
    oprow, oa2 = f.perm()
    assert np.array_equal(prow, oprow) and np.array_equal(a2, oa2)
    assert np.array_equal(d, f.scaling())
    oU, oud = f.U()
    assert np.array_equal(ud, oud)
    oL1 = f.L1()
    for part, ref in ((B.PART_L1, oL1), (B.PART_L2, f.L2()), (B.PART_U, oU)):
        ptr, idx, val = P.factor_csr(part)
        assert np.array_equal(ptr, ref.ptr) and np.array_equal(idx, ref.idx) and np.array_equal(val, ref.val)

    def transposed(c):
        t = sp.csr_matrix((c.val, c.idx, c.ptr), shape=c.shape).T.tocsr()
        t.sort_indices()
        return oracle.CSR(t.indptr.astype(np.int64), t.indices.astype(np.int32), t.data, t.shape)

    for sys_id, csr, lower in ((B.SYS_L1, oL1, True), (B.SYS_L1T, transposed(oL1), False),
                               (B.SYS_U, oU, False), (B.SYS_UT, transposed(oU), True)):
        lev, _ = oracle.levels(csr, lower)
        assert np.array_equal(P.levels(sys_id), lev), sys_id


def test_fullsize_apply_fp64(full):
    prob, f, P = full
    s = np.random.default_rng(21).standard_normal(prob.n)
    t = P.apply(s)
    ref = f.apply(s)
    print(f"full-size FP64 apply: rel {rel(t, ref):.2e}, elementwise {rel_inf(t, ref):.2e}")
    assert rel(t, ref) <= 1e-12 and rel_inf(t, ref) <= 1e-12


def test_fullsize_apply_fp32(full):
    # last: re-factors the shared handle in float32 (the host ILUP is reused)
    prob, f, P = full
    P.factor(**FACTOR, precision=B.PREC_FP32)
    s = np.random.default_rng(22).standard_normal(prob.n)
    t = P.apply(s)
    ref = f.apply(s)
    print(f"full-size FP32 apply: rel {rel(t, ref):.2e}, elementwise {rel_inf(t, ref):.2e}")
    assert rel(t, ref) <= 2e-6 and rel_inf(t, ref) <= 2e-6
