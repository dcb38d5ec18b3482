"""CPU tests of the library's host side: the row-selecting ILU set-up must equal
the oracle bit for bit (permutation, factor patterns and values, scaling,
level sets), and the C ABI must load and export every declared symbol with
struct layouts that match the header.  No GPU is used."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def compare(prob, **kw):
    s = B.HostSetup(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, **kw)
    okw = {k: v for k, v in kw.items() if k in ("p", "tau", "mu", "small")}
    f = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals,
                      scale=kw.get("scale_columns", 1), **okw)
    prow, a2, d, ud = s.split()
    oprow, oa2 = f.perm()
    assert np.array_equal(prow, oprow)
    assert np.array_equal(a2, oa2)
    assert np.array_equal(d, f.scaling())
    oU, oud = f.U()
    assert np.array_equal(ud, oud)
    for part, ref in ((B.PART_L1, f.L1()), (B.PART_L2, f.L2()), (B.PART_U, oU)):
        ptr, idx, val = s.factor_csr(part)
        assert np.array_equal(ptr, ref.ptr)
        assert np.array_equal(idx, ref.idx)
        assert np.array_equal(val, ref.val)  # bit-exact values
    sz = s.sizes()
    assert sz["nmod"] == f.sizes()["nmod"]
    L1, (U, _) = f.L1(), f.U()
    import scipy.sparse as sp

    for which, csr, lower in ((B.SYS_L1, L1, True), (B.SYS_U, U, False)):
        lev, nl = oracle.levels(csr, lower)
        assert np.array_equal(s.levels(which), lev)
        T = csr.to_scipy().T.tocsr()
        tc = oracle.CSR(T.indptr.astype(np.int64), T.indices.astype(np.int32), T.data, T.shape)
        lev_t, _ = oracle.levels(tc, not lower)
        assert np.array_equal(s.levels(which + 1), lev_t)
    del sp
    return sz


@pytest.mark.parametrize("mu", [1.0, 0.5, 0.1])
def test_setup_bitexact_config0(mu):
    compare(synth.config_problem(0), mu=mu)


@pytest.mark.parametrize("seed", range(40))
def test_setup_bitexact_random_small(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 60))
    m = n + int(rng.integers(1, 2 * n + 2))
    d = int(rng.integers(1, min(n, 7) + 1))
    prob = synth.sparse_problem(m, n, d, seed=1000 + seed)
    p = int(rng.choice([-1, 1, 2, 5, 10]))
    tau = float(rng.choice([0.0, 1e-3, 1e-2, 0.1, 0.3]))
    mu = float(rng.choice([0.05, 0.1, 0.5, 1.0]))
    compare(prob, p=p, tau=tau, mu=mu, scale_columns=int(rng.integers(0, 2)))


def test_setup_bitexact_with_modified_pivots():
    """Exercise Algorithm 6: heavy dropping on a matrix with dependent
    columns makes columns empty."""
    A = np.zeros((12, 6))
    rng = np.random.default_rng(0)
    A[:, 0] = rng.standard_normal(12)
    A[:, 1] = A[:, 0]
    A[:, 2] = 2 * A[:, 0]
    A[:, 3:] = rng.standard_normal((12, 3))
    import scipy.sparse as sp

    S = sp.csr_matrix(A)
    prob = synth.Problem(12, 6, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data,
                         np.zeros(12), np.zeros(6), np.zeros(0, dtype=np.int64))
    sz = compare(prob, p=-1, tau=0.0, mu=1.0)
    assert sz["nmod"] >= 2


def test_setup_bitexact_config1_recipe_scaled():
    """The 2M x 1M recipe at 1/40 scale (many columns, ragged sizes)."""
    prob = synth.sparse_problem(50_001, 25_000, 8, seed=1, hidden_diag=True)
    sz = compare(prob, mu=1.0)
    assert sz["levels_L1"] < 100


def test_setup_sparse_dense_places_dense_rows_in_A2():
    prob = synth.sparse_dense_problem(6000, 3000, 6, 20, seed=2)
    s = B.HostSetup(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, mu=1.0)
    prow, a2, _, _ = s.split()
    assert set(prob.dense_rows.tolist()) <= set(a2.tolist())
    compare(prob, mu=1.0)


def test_setup_errors():
    prob = synth.config_problem(0)
    with pytest.raises(B.RlsqError) as e:
        B.HostSetup(prob.n, prob.m, prob.rowptr[: prob.n + 1], prob.colidx, prob.vals)
    assert e.value.code == -2
    bad = prob.colidx.copy()
    bad[1] = bad[0]  # duplicate column in row 0
    with pytest.raises(B.RlsqError) as e:
        B.HostSetup(prob.m, prob.n, prob.rowptr, bad, prob.vals)
    assert e.value.code == -3
    # empty column
    keep = prob.colidx != 5
    rp = np.concatenate([[0], np.cumsum([keep[prob.rowptr[i]:prob.rowptr[i + 1]].sum()
                                         for i in range(prob.m)])]).astype(np.int64)
    with pytest.raises(B.RlsqError) as e:
        B.HostSetup(prob.m, prob.n, rp, prob.colidx[keep], prob.vals[keep])
    assert e.value.code == -4
    with pytest.raises(B.RlsqError) as e:
        B.HostSetup(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, mu=0.0)
    assert e.value.code == -1


# ---------------------------------------------------------------------------
# the C ABI itself
# ---------------------------------------------------------------------------
def declared_functions():
    text = open(os.path.join(ROOT, "include", "rlsq.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rlsq_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    lib = B.load()
    names = declared_functions()
    assert len(names) >= 25
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(B.EXPORTS) == names


def test_struct_layouts_match_header(tmp_path):
    """Compile a C program against include/rlsq.h and compare sizes and
    offsets with the ctypes mirrors."""
    structs = {"rlsq_factor_opts": B.FactorOpts, "rlsq_solve_opts": B.SolveOpts,
               "rlsq_info": B.Info, "rlsq_server_opts": B.ServerOpts,
               "rlsq_server_stats": B.ServerStats, "rlsq_profile_out": B.ProfileOut}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rlsq.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'printf("{cname}.{field} %zu\\n", offsetof({cname}, {field}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for field, _ in py._fields_:
            assert int(got[f"{cname}.{field}"]) == getattr(py, field).offset, (cname, field)


def test_defaults_are_the_papers():
    o = B.factor_opts()
    assert (o.p, o.tau, o.mu, o.small) == (10, 1e-2, 0.1, 1e-10)
    s = B.solve_opts()
    assert s.atol == 1e-8 and s.maxit == 2000
