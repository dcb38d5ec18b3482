"""Writes tests/golden/config0_oracle.json from the CPU oracle alone.

The paper prints no worked example, so these fixtures pin the oracle against
its own recorded output on the 1500 x 1000 workload (seed 0; ILUP p = 10,
tau = 1e-2, mu = 1): a later change to the oracle's arithmetic must show up as
a diff here and be justified by the passage of the paper it follows.

    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2603_28642_gb300 import synth  # noqa: E402

MODES = {"NONE": oracle.NONE, "SI": oracle.SI, "CG": oracle.CG, "DENSE": oracle.DENSE}


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def levels_of(L1, U):
    """Level counts of L1 (lower), L1^T, U (upper), U^T."""
    def csr(m):
        m = m.tocsr()
        m.sort_indices()
        return oracle.CSR(m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data, m.shape)
    l1, u = L1.to_scipy(), U.to_scipy()
    systems = [(csr(l1), True), (csr(l1.T), False), (csr(u), False), (csr(u.T), True)]
    return [oracle.levels(c, lower)[1] for c, lower in systems]


def build() -> dict:
    p = synth.config_problem(0)
    f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, p=10, tau=1e-2, mu=1.0)
    prow, a2 = f.perm()
    L1, L2 = f.L1(), f.L2()
    U, ud = f.U()
    out = {
        "problem": "config 0: 1500 x 1000, 6 N(0,1) per row + first-n-rows +-4 diagonal, seed 0",
        "ilup": {"p": 10, "tau": 1e-2, "mu": 1.0},
        "prow": prow.tolist(),
        "a2rows": a2.tolist(),
        "nnz": {"L1": int(L1.ptr[-1]), "L2": int(L2.ptr[-1]), "U": int(U.ptr[-1])},
        "levels": levels_of(L1, U),
        "sha256": {"L1.val": digest(L1.val), "L2.val": digest(L2.val), "U.val": digest(U.val),
                   "Udiag": digest(ud), "scaling": digest(f.scaling())},
        "anorm": oracle.norm2(p.m, p.n, p.rowptr, p.colidx, p.vals),
        "lsmr": {}, "cgls": {},
    }
    for name, mode in MODES.items():
        f.set_correction(mode, 2)
        r = oracle.lsmr(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, atol=1e-8, maxit=2000)
        out["lsmr"][name] = {"status": r.status, "its": r.its, "ratio_hist_first": r.ratio_hist[:5].tolist(),
                             "x_sha256": digest(r.x)}
        c = oracle.cgls(f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, atol=1e-8, maxit=2000, form="symmetric")
        out["cgls"][name] = {"status": c.status, "its": c.its, "x_sha256": digest(c.x)}
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "config0_oracle.json"), "w") as fh:
        json.dump(build(), fh, indent=1)
        fh.write("\n")
