"""Python access to the CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  The oracle is a plain,
single-threaded FP64 C restatement of the paper's method (see oracle.c for
the per-function citations); this module only compiles it and marshals
numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

NONE, SI, CG, DENSE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        i64, i32, dbl, cint = C.c_int64, C.c_int32, C.c_double, C.c_int
        lib.orc_factor_create.restype = P
        lib.orc_factor_create.argtypes = [i64, i64, P, P, P, cint, dbl, dbl, dbl, cint]
        lib.orc_factor_free.argtypes = [P]
        lib.orc_factor_sizes.argtypes = [P, P]
        lib.orc_factor_perm.argtypes = [P, P, P]
        lib.orc_factor_scaling.argtypes = [P, P]
        lib.orc_factor_L1.argtypes = [P, P, P, P]
        lib.orc_factor_L2.argtypes = [P, P, P, P]
        lib.orc_factor_U.argtypes = [P, P, P, P, P]
        lib.orc_levels.restype = i64
        lib.orc_levels.argtypes = [i64, P, P, cint, P]
        lib.orc_correction.restype = cint
        lib.orc_correction.argtypes = [P, cint, cint]
        lib.orc_cg_tolerance.argtypes = [P, dbl]
        lib.orc_cg_last_steps.restype = cint
        lib.orc_cg_last_steps.argtypes = [P]
        lib.orc_correction_dense.restype = cint
        lib.orc_correction_dense.argtypes = [P, P]
        for name in ("orc_apply", "orc_solve_L1", "orc_solve_L1t", "orc_solve_U",
                     "orc_solve_Ut", "orc_s_solve"):
            getattr(lib, name).argtypes = [P, P, P]
        lib.orc_column_scaling.restype = cint
        lib.orc_column_scaling.argtypes = [i64, i64, P, P, P, P]
        lib.orc_spmv.argtypes = [i64, P, P, P, P, P]
        lib.orc_spmv_t.argtypes = [i64, i64, P, P, P, P, P]
        lib.orc_norm2.restype = dbl
        lib.orc_norm2.argtypes = [i64, i64, P, P, P, cint]
        lib.orc_lsmr.restype = cint
        lib.orc_lsmr.argtypes = [P, i64, i64, P, P, P, P, dbl, dbl, cint, P, P, P, P]
        lib.orc_apply_residual.argtypes = [P, P, P]
        lib.orc_factor_add_rows.restype = cint
        lib.orc_factor_add_rows.argtypes = [P, i64, P, P, P, cint, dbl]
        lib.orc_factor_remove_rows.restype = cint
        lib.orc_factor_remove_rows.argtypes = [P, i64, P]
        lib.orc_cgls.restype = cint
        lib.orc_cgls.argtypes = [P, cint, i64, i64, P, P, P, P, dbl, dbl, cint, P, P, P, P]
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _csr_arrays(rowptr, colidx, vals):
    return (np.ascontiguousarray(rowptr, dtype=np.int64),
            np.ascontiguousarray(colidx, dtype=np.int32),
            np.ascontiguousarray(vals, dtype=np.float64))


@dataclass
class CSR:
    ptr: np.ndarray
    idx: np.ndarray
    val: np.ndarray
    shape: tuple

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.idx, self.ptr), shape=self.shape)


class Factor:
    """The oracle's ILUP(p, tau) factorisation of one matrix plus its
    correction set-up.  Arrays are copied out on access."""

    def __init__(self, m, n, rowptr, colidx, vals, p=10, tau=1e-2, mu=0.1, small=1e-10,
                 scale=True):
        lib = _load()
        self._keep = _csr_arrays(rowptr, colidx, vals)
        rp, ci, va = self._keep
        self.m, self.n = int(m), int(n)
        h = lib.orc_factor_create(self.m, self.n, _p(rp), _p(ci), _p(va), int(p), float(tau),
                                  float(mu), float(small), int(bool(scale)))
        if not h:
            raise ValueError("oracle factorisation rejected the input (m <= n or empty column)")
        self._h = h
        self.mode = NONE
        self.cg_steps = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().orc_factor_free(h)
            self._h = None

    # --- structure -------------------------------------------------------
    def sizes(self):
        out = np.zeros(4, dtype=np.int64)
        _load().orc_factor_sizes(self._h, _p(out))
        return dict(nnz_L1=int(out[0]), nnz_L2=int(out[1]), nnz_U=int(out[2]), nmod=int(out[3]))

    def perm(self):
        prow = np.zeros(self.n, dtype=np.int32)
        a2 = np.zeros(max(self.m - self.n, 1), dtype=np.int32)
        _load().orc_factor_perm(self._h, _p(prow), _p(a2))
        return prow, a2[: self.m - self.n]

    def scaling(self):
        d = np.zeros(self.n)
        _load().orc_factor_scaling(self._h, _p(d))
        return d

    def _csr(self, fn, rows, nnz, cols, extra=None):
        ptr = np.zeros(rows + 1, dtype=np.int64)
        idx = np.zeros(max(nnz, 1), dtype=np.int32)
        val = np.zeros(max(nnz, 1))
        args = [self._h, _p(ptr), _p(idx), _p(val)]
        if extra is not None:
            args.append(_p(extra))
        fn(*args)
        return CSR(ptr, idx[:nnz], val[:nnz], (rows, cols))

    def L1(self) -> CSR:
        """strictly lower part of L1 (unit diagonal implied), rows = pivot positions"""
        return self._csr(_load().orc_factor_L1, self.n, self.sizes()["nnz_L1"], self.n)

    def L2(self) -> CSR:
        return self._csr(_load().orc_factor_L2, self.m - self.n, self.sizes()["nnz_L2"], self.n)

    def U(self):
        """(strictly upper CSR of U, diagonal of U)"""
        diag = np.zeros(self.n)
        csr = self._csr(_load().orc_factor_U, self.n, self.sizes()["nnz_U"], self.n, extra=diag)
        return csr, diag

    # --- correction and apply ---------------------------------------------
    def set_correction(self, mode: int, cg_steps: int = 2, cg_tol: float = 0.0):
        """cg_tol > 0 (CG mode): stop the CG steps on S once ||r_j|| <= cg_tol ||r_0||,
        at most cg_steps of them."""
        rc = _load().orc_correction(self._h, int(mode), int(cg_steps))
        if rc != 0:
            raise ValueError("dense S is not positive definite")
        _load().orc_cg_tolerance(self._h, float(cg_tol))
        self.mode, self.cg_steps, self.cg_tol = mode, cg_steps, cg_tol

    def cg_last_steps(self) -> int:
        """CG steps the last S solve (one apply) took."""
        return int(_load().orc_cg_last_steps(self._h))

    def dense_cholesky(self):
        m2 = self.m - self.n
        out = np.zeros((m2, m2))
        ok = _load().orc_correction_dense(self._h, _p(out))
        return out if ok else None

    def _vec(self, fn, v, n_out):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(n_out)
        fn(self._h, _p(v), _p(out))
        return out

    def apply(self, s):
        return self._vec(_load().orc_apply, s, self.n)

    def add_rows(self, rowptr, colidx, vals, p=10, tau=1e-2):
        """Sec. 3.4: append rows (CSR, the user's values) to A2; returns the status."""
        rp, ci, va = _csr_arrays(rowptr, colidx, vals)
        k = len(rp) - 1
        st = _load().orc_factor_add_rows(self._h, k, _p(rp), _p(ci), _p(va), int(p), float(tau))
        self.m += k
        return int(st)

    def remove_rows(self, ids):
        """Sec. 3.4: remove rows of A2 (ascending ids); -1 if one is a pivot row."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        st = _load().orc_factor_remove_rows(self._h, len(ids), _p(ids))
        if st >= 0:
            self.m -= len(ids)
        return int(st)

    def apply_residual(self, r):
        """Algorithm 3 on a residual r (length m): h = M^{-1} A^T r in the paper's form."""
        return self._vec(_load().orc_apply_residual, r, self.n)

    def solve_L1(self, b):
        return self._vec(_load().orc_solve_L1, b, self.n)

    def solve_L1t(self, b):
        return self._vec(_load().orc_solve_L1t, b, self.n)

    def solve_U(self, b):
        return self._vec(_load().orc_solve_U, b, self.n)

    def solve_Ut(self, b):
        return self._vec(_load().orc_solve_Ut, b, self.n)

    def s_solve(self, e):
        return self._vec(_load().orc_s_solve, e, self.m - self.n)


def levels(csr: CSR, lower: bool):
    """Level of every row of a triangular matrix (strictly triangular CSR) and
    the number of levels."""
    n = csr.shape[0]
    lev = np.zeros(n, dtype=np.int32)
    nl = _load().orc_levels(n, _p(csr.ptr), _p(csr.idx), int(bool(lower)), _p(lev))
    return lev, int(nl)


def column_scaling(m, n, rowptr, colidx, vals):
    rp, ci, va = _csr_arrays(rowptr, colidx, vals)
    d = np.zeros(n)
    rc = _load().orc_column_scaling(m, n, _p(rp), _p(ci), _p(va), _p(d))
    if rc != 0:
        raise ValueError("empty column")
    return d


def spmv(m, rowptr, colidx, vals, x):
    rp, ci, va = _csr_arrays(rowptr, colidx, vals)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(m)
    _load().orc_spmv(m, _p(rp), _p(ci), _p(va), _p(x), _p(y))
    return y


def spmv_t(m, n, rowptr, colidx, vals, x):
    rp, ci, va = _csr_arrays(rowptr, colidx, vals)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(n)
    _load().orc_spmv_t(m, n, _p(rp), _p(ci), _p(va), _p(x), _p(y))
    return y


def norm2(m, n, rowptr, colidx, vals, iters=50):
    rp, ci, va = _csr_arrays(rowptr, colidx, vals)
    return float(_load().orc_norm2(m, n, _p(rp), _p(ci), _p(va), int(iters)))


@dataclass
class LsmrResult:
    x: np.ndarray
    its: int
    status: int  # 0 converged, 1 iteration limit, -2 breakdown
    ratio: float
    ratio_hist: np.ndarray


def lsmr(factor, m, n, rowptr, colidx, vals, b, anorm=None, atol=1e-8, maxit=2000):
    """Preconditioned LSMR (factor=None: unpreconditioned)."""
    lib = _load()
    rp, ci, va = _csr_arrays(rowptr, colidx, vals)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if anorm is None:
        anorm = norm2(m, n, rp, ci, va)
    x = np.zeros(n)
    its = C.c_int(0)
    fr = C.c_double(0.0)
    hist = np.zeros(maxit + 1)
    st = lib.orc_lsmr(factor._h if factor is not None else None, m, n, _p(rp), _p(ci), _p(va),
                      _p(b), float(anorm), float(atol), int(maxit), _p(x), C.byref(its),
                      _p(hist), C.byref(fr))
    return LsmrResult(x, its.value, int(st), fr.value, hist[: its.value + 1])


def cgls(factor, m, n, rowptr, colidx, vals, b, anorm=None, atol=1e-8, maxit=2000, form="residual"):
    """Algorithm 1 (left preconditioned CGLS).  form "residual": h from
    Algorithm 3 fed the residual split (the paper's combination of M^{-1} with
    A^T); "symmetric": h = M^{-1} A^T r with the x-space operator."""
    lib = _load()
    rp, ci, va = _csr_arrays(rowptr, colidx, vals)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if anorm is None:
        anorm = norm2(m, n, rp, ci, va)
    x = np.zeros(n)
    its = C.c_int(0)
    fr = C.c_double(0.0)
    hist = np.zeros(maxit + 1)
    st = lib.orc_cgls(factor._h if factor is not None else None, 0 if form == "residual" else 1, m, n,
                      _p(rp), _p(ci), _p(va), _p(b),
                      float(anorm), float(atol), int(maxit),
                      _p(x), C.byref(its), _p(hist), C.byref(fr))
    return LsmrResult(x, its.value, int(st), fr.value, hist[: its.value + 1])
