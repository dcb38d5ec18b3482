"""ctypes binding of the rlsq C ABI (include/rlsq.h).

Argument marshalling only: every step of the factorisation set-up and of the
solve runs inside librlsq.so.  Host arrays are numpy arrays; device arrays
are CUDA torch tensors (torch supplies device memory and streams).  There is
no fallback: if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

# status codes (rlsq.h)
OK, PENDING = 0, 1
ERR = {
    -1: "ARG", -2: "SHAPE", -3: "CSR", -4: "RANK", -5: "NOT_FACTORED", -6: "OOM",
    -7: "BREAKDOWN", -8: "MAXIT", -9: "DEVICE_TIMEOUT", -10: "CUDA", -11: "ADMISSION",
    -12: "NOT_FOUND", -13: "NUMERIC",
}
ERR_BREAKDOWN, ERR_MAXIT, ERR_DEVICE_TIMEOUT = -7, -8, -9
HOST_PTRS, DEVICE_PTRS = 0, 1
CORR_NONE, CORR_SI, CORR_CG, CORR_DENSE, CORR_AUTO = 0, 1, 2, 3, 4
PREC_FP64, PREC_FP32 = 0, 1
TRSV_AUTO, TRSV_LEVEL, TRSV_SYNCFREE, TRSV_COOP, TRSV_WAVE, TRSV_BINNED = 0, 1, 2, 3, 4, 5
SOLVER_LSMR, SOLVER_CGLS, SOLVER_CGLS_SPLIT = 0, 1, 2
SYS_L1, SYS_L1T, SYS_U, SYS_UT = 0, 1, 2, 3
PART_L1, PART_L2, PART_U = 0, 1, 2


class RlsqError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rlsq error {code} ({ERR.get(code, '?')}): {msg}")
        self.code = code


class FactorOpts(C.Structure):
    _fields_ = [
        ("p", C.c_int32), ("tau", C.c_double), ("mu", C.c_double), ("small", C.c_double),
        ("scale_columns", C.c_int32), ("correction", C.c_int32), ("cg_steps", C.c_int32),
        ("dense_cap", C.c_int64), ("precision", C.c_int32), ("trsv_schedule", C.c_int32),
        ("autotune", C.c_int32), ("dense_row_min", C.c_int64), ("host_threads", C.c_int32),
        ("level_merge", C.c_int32), ("trsv_rows", C.c_int32), ("cg_tol", C.c_double),
        ("dense_host", C.c_int32),
        ("sliced", C.c_int32),
    ]


class SolveOpts(C.Structure):
    _fields_ = [
        ("atol", C.c_double), ("maxit", C.c_int32), ("ptr_mode", C.c_int32),
        ("stream", C.c_void_p), ("check_every", C.c_int32), ("solver", C.c_int32),
    ]


class Info(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("iterations", C.c_int32), ("ratio", C.c_double),
        ("rnorm", C.c_double), ("arnorm", C.c_double), ("anorm", C.c_double),
        ("factor_seconds", C.c_double), ("solve_seconds", C.c_double),
        ("m", C.c_int64), ("n", C.c_int64), ("nnz_A", C.c_int64), ("nnz_L1", C.c_int64),
        ("nnz_L2", C.c_int64), ("nnz_U", C.c_int64), ("nmod", C.c_int64),
        ("n_dense_rows", C.c_int64),
        ("levels_L1", C.c_int32), ("levels_L1t", C.c_int32), ("levels_U", C.c_int32),
        ("levels_Ut", C.c_int32), ("correction", C.c_int32), ("precision", C.c_int32),
        ("bytes_per_iter", C.c_double), ("solve_levels", C.c_int32 * 4), ("level_merge", C.c_int32 * 4),
        ("trsv_schedule", C.c_int32 * 4), ("ilup_seconds", C.c_double), ("ilup_threads", C.c_int32),
        ("solve_entries", C.c_int64 * 4),
        ("sliced_products", C.c_int32),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") and not isinstance(v, (bytes, str)) else v
        return out


class ServerOpts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_slots", C.c_int32), ("atol", C.c_double),
                ("maxit", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [
        ("submitted", C.c_int64), ("completed", C.c_int64), ("queued", C.c_int64),
        ("active", C.c_int64), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
        ("mean_ms", C.c_double), ("solves_per_s", C.c_double), ("ticks", C.c_int64),
        ("peak_bytes", C.c_int64), ("tick_ms", C.c_double), ("tick_device_ms", C.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


# every symbol declared in include/rlsq.h
EXPORTS = [
    "rlsq_factor_opts_default", "rlsq_solve_opts_default", "rlsq_create", "rlsq_factor",
    "rlsq_solve", "rlsq_solve_plain", "rlsq_batch_solve", "rlsq_apply", "rlsq_apply_residual", "rlsq_matvec",
    "rlsq_trsv", "rlsq_get_info", "rlsq_get_split", "rlsq_get_factor", "rlsq_get_levels",
    "rlsq_destroy", "rlsq_server_create", "rlsq_server_register", "rlsq_server_submit",
    "rlsq_server_poll", "rlsq_server_get_stats", "rlsq_server_destroy", "rlsq_last_error",
    "rlsq_setup_create", "rlsq_setup_threads", "rlsq_setup_schur_inverse", "rlsq_setup_sizes", "rlsq_setup_split", "rlsq_setup_factor",
    "rlsq_setup_levels", "rlsq_setup_destroy", "rlsq_profile", "rlsq_trsv_noalloc",
    "rlsq_setup_fuse", "rlsq_setup_fused", "rlsq_setup_add_rows", "rlsq_setup_remove_rows",
    "rlsq_add_rows", "rlsq_remove_rows",
]

KCLASS = ["spmv", "spmvt", "trsv_L1", "trsv_L1t", "trsv_U", "trsv_Ut", "l2", "l2t", "vec",
          "finish", "update", "dense"]


class ProfileOut(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("total_ms", C.c_double),
                ("class_ms", C.c_double * 12), ("class_launches", C.c_int32 * 12),
                ("class_bytes", C.c_double * 12), ("bytes_per_iter", C.c_double)]

_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True):
    """Load librlsq.so (building it first if needed); raises if impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        lib = C.CDLL(path)
        P, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "rlsq_factor_opts_default": (None, [P]),
            "rlsq_solve_opts_default": (None, [P]),
            "rlsq_create": (C.c_int, [i64, i64, P, P, P, i32, P, P]),
            "rlsq_factor": (C.c_int, [P, P]),
            "rlsq_solve": (C.c_int, [P, P, P, P, P]),
            "rlsq_solve_plain": (C.c_int, [P, P, P, P, P]),
            "rlsq_batch_solve": (C.c_int, [P, P, P, i32, P, P]),
            "rlsq_apply": (C.c_int, [P, P, P, i32, P]),
            "rlsq_apply_residual": (C.c_int, [P, P, P, i32, P]),
            "rlsq_matvec": (C.c_int, [P, i32, P, P, i32, P]),
            "rlsq_trsv": (C.c_int, [P, i32, P, P, i32, P]),
            "rlsq_get_info": (C.c_int, [P, P]),
            "rlsq_get_split": (C.c_int, [P, P, P, P, P]),
            "rlsq_get_factor": (C.c_int, [P, i32, P, P, P]),
            "rlsq_get_levels": (C.c_int, [P, i32, P]),
            "rlsq_destroy": (None, [P]),
            "rlsq_server_create": (C.c_int, [P, P]),
            "rlsq_server_register": (C.c_int, [P, P, P]),
            "rlsq_server_submit": (C.c_int, [P, i32, P, P]),
            "rlsq_server_poll": (C.c_int, [P, i64, P, P]),
            "rlsq_server_get_stats": (C.c_int, [P, P]),
            "rlsq_server_destroy": (None, [P]),
            "rlsq_last_error": (C.c_char_p, []),
            "rlsq_setup_create": (C.c_int, [i64, i64, P, P, P, P, P]),
            "rlsq_setup_threads": (C.c_int32, [C.c_int32, C.c_int64, C.c_int64]),
            "rlsq_setup_schur_inverse": (C.c_int, [P, C.c_int32, P]),
            "rlsq_setup_sizes": (C.c_int, [P, P]),
            "rlsq_setup_split": (C.c_int, [P, P, P, P, P]),
            "rlsq_setup_factor": (C.c_int, [P, i32, P, P, P]),
            "rlsq_setup_levels": (C.c_int, [P, i32, P]),
            "rlsq_setup_destroy": (None, [P]),
            "rlsq_profile": (C.c_int, [P, P, i32, i32, i32, P]),
            "rlsq_trsv_noalloc": (C.c_int, [P, i32, P, P, P]),
            "rlsq_setup_fuse": (C.c_int, [P, i32, i32, P]),
            "rlsq_setup_fused": (C.c_int, [P, i32, P, P, P]),
            "rlsq_setup_add_rows": (C.c_int, [P, i64, P, P, P]),
            "rlsq_setup_remove_rows": (C.c_int, [P, i64, P]),
            "rlsq_add_rows": (C.c_int, [P, i64, P, P, P]),
            "rlsq_remove_rows": (C.c_int, [P, i64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(code: int, allow=(OK,)):
    if code in allow:
        return code
    msg = load().rlsq_last_error().decode(errors="replace")
    raise RlsqError(code, msg)


def _ptr(a):
    """Host numpy array -> (pointer, HOST_PTRS); CUDA torch tensor -> (pointer, DEVICE_PTRS)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p), HOST_PTRS
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        return C.c_void_p(a.data_ptr()), DEVICE_PTRS
    raise TypeError("expected a numpy array or a CUDA torch tensor")


def _stream_of(a):
    if isinstance(a, np.ndarray):
        return None
    import torch

    return C.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)


def factor_opts(**kw) -> FactorOpts:
    o = FactorOpts()
    load().rlsq_factor_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown factor option {k}")
        setattr(o, k, v)
    return o


def solve_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    load().rlsq_solve_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown solve option {k}")
        setattr(o, k, v)
    return o


@dataclass
class SolveResult:
    x: object
    info: dict
    status: int


class Problem:
    """One least-squares problem min ||b - A x|| resident on the GPU."""

    def __init__(self, m, n, rowptr, colidx, vals):
        lib = load()
        if isinstance(rowptr, np.ndarray):
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
            colidx = np.ascontiguousarray(colidx, dtype=np.int32)
            vals = np.ascontiguousarray(vals, dtype=np.float64)
        p0, mode = _ptr(rowptr)
        p1, _ = _ptr(colidx)
        p2, _ = _ptr(vals)
        h = C.c_void_p()
        _check(lib.rlsq_create(int(m), int(n), p0, p1, p2, mode, _stream_of(rowptr), C.byref(h)))
        self._h = h
        self.m, self.n = int(m), int(n)

    @classmethod
    def from_problem(cls, prob):
        return cls(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().rlsq_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def factor(self, **kw):
        o = factor_opts(**kw)
        _check(load().rlsq_factor(self._h, C.byref(o)))
        return self.info()

    def add_rows(self, rowptr, colidx, vals):
        """Sec. 3.4: append rows (host CSR over the n columns) without refactorising."""
        rp = np.ascontiguousarray(rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(colidx, dtype=np.int32)
        va = np.ascontiguousarray(vals, dtype=np.float64)
        k = len(rp) - 1
        _check(load().rlsq_add_rows(self._h, k, _ptr(rp)[0], _ptr(ci if len(ci) else np.zeros(1, np.int32))[0],
                                    _ptr(va if len(va) else np.zeros(1))[0]))
        self.m += k
        return self.info()

    def remove_rows(self, ids):
        """Sec. 3.4: remove rows of A2 (ascending ids) without refactorising."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        _check(load().rlsq_remove_rows(self._h, len(ids), _ptr(ids if len(ids) else np.zeros(1, np.int32))[0]))
        self.m -= len(ids)
        return self.info()

    def info(self) -> dict:
        inf = Info()
        _check(load().rlsq_get_info(self._h, C.byref(inf)))
        return inf.as_dict()

    def _out_like(self, ref, size):
        if isinstance(ref, np.ndarray):
            return np.zeros(size)
        import torch

        return torch.empty(size, dtype=torch.float64, device=ref.device)

    def solve(self, b, plain: bool = False, allow_fail: bool = False, **kw) -> SolveResult:
        if isinstance(b, np.ndarray):
            b = np.ascontiguousarray(b, dtype=np.float64)
        pb, mode = _ptr(b)
        x = self._out_like(b, self.n)
        px, _ = _ptr(x)
        o = solve_opts(ptr_mode=mode, stream=_stream_of(b), **kw)
        inf = Info()
        fn = load().rlsq_solve_plain if plain else load().rlsq_solve
        code = fn(self._h, pb, px, C.byref(o), C.byref(inf))
        if not allow_fail:
            _check(code, allow=(OK, ERR_MAXIT))
        return SolveResult(x, inf.as_dict(), code)

    def apply(self, s):
        if isinstance(s, np.ndarray):
            s = np.ascontiguousarray(s, dtype=np.float64)
        ps, mode = _ptr(s)
        t = self._out_like(s, self.n)
        pt, _ = _ptr(t)
        _check(load().rlsq_apply(self._h, ps, pt, mode, _stream_of(s)))
        return t

    def apply_residual(self, r):
        """Algorithm 3 fed the residual split of r (length m): t (length n)."""
        if isinstance(r, np.ndarray):
            r = np.ascontiguousarray(r, dtype=np.float64)
        pr, mode = _ptr(r)
        t = self._out_like(r, self.n)
        pt, _ = _ptr(t)
        _check(load().rlsq_apply_residual(self._h, pr, pt, mode, _stream_of(r)))
        return t

    def matvec(self, x, trans: bool = False):
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float64)
        px, mode = _ptr(x)
        y = self._out_like(x, self.n if trans else self.m)
        py, _ = _ptr(y)
        _check(load().rlsq_matvec(self._h, int(bool(trans)), px, py, mode, _stream_of(x)))
        return y

    def trsv(self, which: int, b):
        if isinstance(b, np.ndarray):
            b = np.ascontiguousarray(b, dtype=np.float64)
        pb, mode = _ptr(b)
        x = self._out_like(b, self.n)
        px, _ = _ptr(x)
        _check(load().rlsq_trsv(self._h, int(which), pb, px, mode, _stream_of(b)))
        return x

    def split(self):
        prow = np.zeros(self.n, dtype=np.int32)
        a2 = np.zeros(max(self.m - self.n, 1), dtype=np.int32)
        d = np.zeros(self.n)
        ud = np.zeros(self.n)
        _check(load().rlsq_get_split(self._h, _ptr(prow)[0], _ptr(a2)[0], _ptr(d)[0], _ptr(ud)[0]))
        return prow, a2[: self.m - self.n], d, ud

    def factor_csr(self, part: int):
        inf = self.info()
        rows = self.n if part in (PART_L1, PART_U) else self.m - self.n
        nnz = {PART_L1: inf["nnz_L1"], PART_L2: inf["nnz_L2"], PART_U: inf["nnz_U"] - self.n}[part]
        ptr = np.zeros(rows + 1, dtype=np.int64)
        idx = np.zeros(max(nnz, 1), dtype=np.int32)
        val = np.zeros(max(nnz, 1))
        _check(load().rlsq_get_factor(self._h, int(part), _ptr(ptr)[0], _ptr(idx)[0], _ptr(val)[0]))
        return ptr, idx[:nnz], val[:nnz]

    def levels(self, which: int):
        lev = np.zeros(self.n, dtype=np.int32)
        _check(load().rlsq_get_levels(self._h, int(which), _ptr(lev)[0]))
        return lev

    def profile(self, b, warmup=3, iters=20, plain=False) -> dict:
        """Device-timed LSMR iterations (graph replay) plus a per-kernel-class
        breakdown of one eager iteration."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        o = ProfileOut()
        _check(load().rlsq_profile(self._h, _ptr(b)[0], int(warmup), int(iters), int(bool(plain)),
                                   C.byref(o)))
        classes = {}
        for i, name in enumerate(KCLASS):
            if o.class_launches[i]:
                classes[name] = dict(ms=o.class_ms[i], launches=o.class_launches[i],
                                     bytes=o.class_bytes[i])
        return dict(status=o.status, iters=o.iters, total_ms=o.total_ms,
                    ms_per_iter=o.total_ms / o.iters, bytes_per_iter=o.bytes_per_iter,
                    classes=classes)


def trsv_noalloc(problem, which: int, b, x):
    """rlsq_trsv_noalloc: triangular solve whose working memory is a static
    device array, for callers that cannot allocate device memory.  b and x
    are CUDA float64 tensors of length n; x is written in place."""
    pb, mb = _ptr(b)
    px, mx = _ptr(x)
    if mb != DEVICE_PTRS or mx != DEVICE_PTRS:
        raise TypeError("rlsq_trsv_noalloc takes device arrays")
    _check(load().rlsq_trsv_noalloc(problem.handle, int(which), pb, px, _stream_of(b)))
    return x


def batch_solve(problems, bs, **kw):
    """Solve several factored problems together; returns (xs, infos, status)."""
    lib = load()
    count = len(problems)
    hs = (C.c_void_p * count)(*[p.handle.value for p in problems])
    bs = [np.ascontiguousarray(b, dtype=np.float64) if isinstance(b, np.ndarray) else b for b in bs]
    mode = _ptr(bs[0])[1]
    xs = [p._out_like(b, p.n) for p, b in zip(problems, bs)]
    bp = (C.c_void_p * count)(*[_ptr(b)[0].value for b in bs])
    xp = (C.c_void_p * count)(*[_ptr(x)[0].value for x in xs])
    infos = (Info * count)()
    o = solve_opts(ptr_mode=mode, stream=_stream_of(bs[0]), **kw)
    code = lib.rlsq_batch_solve(hs, bp, xp, count, C.byref(o), infos)
    _check(code, allow=(OK, ERR_MAXIT, ERR_BREAKDOWN))
    return xs, [infos[i].as_dict() for i in range(count)], code


class Server:
    """Continuous-batching solve server over resident factored problems."""

    def __init__(self, hbm_budget_bytes=150 * 2**30, max_slots=64, atol=1e-8, maxit=2000):
        lib = load()
        o = ServerOpts(int(hbm_budget_bytes), int(max_slots), float(atol), int(maxit))
        h = C.c_void_p()
        _check(lib.rlsq_server_create(C.byref(o), C.byref(h)))
        self._h = h
        self._problems = {}

    def register(self, problem: Problem) -> int:
        mid = C.c_int32()
        _check(load().rlsq_server_register(self._h, problem.handle, C.byref(mid)))
        self._problems[mid.value] = problem
        return mid.value

    def submit(self, matrix_id: int, b) -> int:
        b = np.ascontiguousarray(b, dtype=np.float64)
        t = C.c_int64()
        _check(load().rlsq_server_submit(self._h, int(matrix_id), _ptr(b)[0], C.byref(t)))
        return t.value

    def poll(self, ticket: int, n: int):
        """None while pending; else (x, info dict, status)."""
        x = np.zeros(n)
        inf = Info()
        code = load().rlsq_server_poll(self._h, int(ticket), _ptr(x)[0], C.byref(inf))
        if code == PENDING:
            return None
        _check(code, allow=(OK, ERR_MAXIT, ERR_BREAKDOWN))
        return x, inf.as_dict(), code

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().rlsq_server_get_stats(self._h, C.byref(s)))
        return s.as_dict()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().rlsq_server_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostSetup:
    """The host-side ILUP set-up alone (rlsq_setup_*); needs no GPU."""

    def __init__(self, m, n, rowptr, colidx, vals, **kw):
        lib = load()
        self._keep = (np.ascontiguousarray(rowptr, dtype=np.int64),
                      np.ascontiguousarray(colidx, dtype=np.int32),
                      np.ascontiguousarray(vals, dtype=np.float64))
        o = factor_opts(**kw)
        h = C.c_void_p()
        _check(lib.rlsq_setup_create(int(m), int(n), *[_ptr(a)[0] for a in self._keep],
                                     C.byref(o), C.byref(h)))
        self._h = h
        self.m, self.n = int(m), int(n)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().rlsq_setup_destroy(h)
            self._h = None

    def sizes(self):
        s = np.zeros(8, dtype=np.int64)
        _check(load().rlsq_setup_sizes(self._h, _ptr(s)[0]))
        keys = ["nnz_L1", "nnz_L2", "nnz_U", "nmod", "levels_L1", "levels_L1t", "levels_U",
                "levels_Ut"]
        return {k: int(v) for k, v in zip(keys, s)}

    def split(self):
        prow = np.zeros(self.n, dtype=np.int32)
        a2 = np.zeros(max(self.m - self.n, 1), dtype=np.int32)
        d = np.zeros(self.n)
        ud = np.zeros(self.n)
        _check(load().rlsq_setup_split(self._h, _ptr(prow)[0], _ptr(a2)[0], _ptr(d)[0], _ptr(ud)[0]))
        return prow, a2[: self.m - self.n], d, ud

    def factor_csr(self, part: int):
        s = self.sizes()
        rows = self.n if part in (PART_L1, PART_U) else self.m - self.n
        nnz = {PART_L1: s["nnz_L1"], PART_L2: s["nnz_L2"], PART_U: s["nnz_U"]}[part]
        ptr = np.zeros(rows + 1, dtype=np.int64)
        idx = np.zeros(max(nnz, 1), dtype=np.int32)
        val = np.zeros(max(nnz, 1))
        _check(load().rlsq_setup_factor(self._h, int(part), _ptr(ptr)[0], _ptr(idx)[0], _ptr(val)[0]))
        return ptr, idx[:nnz], val[:nnz]

    def levels(self, which: int):
        lev = np.zeros(self.n, dtype=np.int32)
        _check(load().rlsq_setup_levels(self._h, int(which), _ptr(lev)[0]))
        return lev

    def add_rows(self, rowptr, colidx, vals):
        """Sec. 3.4: append rows (host CSR over the n columns) to A2."""
        rp = np.ascontiguousarray(rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(colidx, dtype=np.int32)
        va = np.ascontiguousarray(vals, dtype=np.float64)
        k = len(rp) - 1
        _check(load().rlsq_setup_add_rows(self._h, k, _ptr(rp)[0], _ptr(ci if len(ci) else np.zeros(1, np.int32))[0],
                                          _ptr(va if len(va) else np.zeros(1))[0]))
        self.m += k

    def schur_inverse(self, recompute: bool = False):
        """S^{-1} of the dense correction ((m-n) x (m-n)); kept and updated by row changes."""
        m2 = self.m - self.n
        out = np.zeros((m2, m2))
        _check(load().rlsq_setup_schur_inverse(self._h, int(bool(recompute)), _ptr(out if m2 else np.zeros(1))[0]))
        return out

    def remove_rows(self, ids):
        """Sec. 3.4: remove rows of A2 (ascending ids); raises for a pivot row."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        _check(load().rlsq_setup_remove_rows(self._h, len(ids), _ptr(ids if len(ids) else np.zeros(1, np.int32))[0]))
        self.m -= len(ids)

    def fuse(self, which: int, k: int):
        """Level fusion of one system (k >= 1 fixed groups, 0 chosen level by
        level); returns sizes and the CSR of T and R (unknown ids)."""
        out = np.zeros(4, dtype=np.int64)
        _check(load().rlsq_setup_fuse(self._h, int(which), int(k), _ptr(out)[0]))
        parts = []
        for part, nnz in ((0, int(out[0])), (1, int(out[1]))):
            ptr = np.zeros(self.n + 1, dtype=np.int64)
            idx = np.zeros(max(nnz, 1), dtype=np.int32)
            val = np.zeros(max(nnz, 1))
            _check(load().rlsq_setup_fused(self._h, part, _ptr(ptr)[0], _ptr(idx)[0], _ptr(val)[0]))
            parts.append((ptr, idx[:nnz], val[:nnz]))
        sizes = {"nnz_T": int(out[0]), "nnz_R": int(out[1]), "levels": int(out[2]), "max_group": int(out[3])}
        return sizes, parts[0], parts[1]
