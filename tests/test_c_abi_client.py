"""The boundary is a plain C ABI.  A C program (tests/c_client/setup_client.c)
compiled with gcc against include/rlsq.h and linked to the library runs the
host-only set-up and gets, bit for bit, what the Python binding and the
oracle get; error statuses and messages reach C too (no GPU used).  A second
C program (tests/c_client/solve_client.c, GPU test) runs rlsq_create,
rlsq_factor, rlsq_solve, rlsq_batch_solve and the server calls and is checked
against the oracle's solution."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import build as _build
from paper_2603_28642_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    B.load()  # builds the library if needed
    lib = _build.LIB
    exe = tmp_path_factory.mktemp("c_client") / "setup_client"
    subprocess.run(["gcc", "-std=c99", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_client", "setup_client.c"), "-o", str(exe),
                    lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    return exe


def run_client(exe, prob, threads, tmp_path):
    path = tmp_path / "a.bin"
    with open(path, "wb") as f:
        np.array([prob.m, prob.n, prob.rowptr[-1]], dtype=np.int64).tofile(f)
        np.asarray(prob.rowptr, np.int64).tofile(f)
        np.asarray(prob.colidx, np.int32).tofile(f)
        np.asarray(prob.vals, np.float64).tofile(f)
    out = subprocess.run([str(exe), str(path), str(threads)], capture_output=True, text=True, check=True).stdout
    rows = {}
    for line in out.splitlines():
        key, *vals = line.split(" ")
        rows[key] = vals
    return rows


def ints(v):
    return np.array([int(t) for t in v], dtype=np.int64)


def floats(v):
    return np.array([float.fromhex(t) for t in v], dtype=np.float64)


@pytest.mark.parametrize("which,threads", [("config0", 1), ("config0", 4), ("random", 3)])
def test_c_client_matches_binding_and_oracle(client, tmp_path, which, threads):
    prob = synth.config_problem(0) if which == "config0" else synth.sparse_problem(700, 300, 4, seed=77)
    got = run_client(client, prob, threads, tmp_path)
    assert got["bad_shape"] == ["-2", "1"]  # RLSQ_ERR_SHAPE with a message
    assert int(got["threads"][0]) == threads
    s = B.HostSetup(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, mu=1.0, host_threads=threads)
    sizes = s.sizes()
    assert list(ints(got["sizes"])) == list(sizes.values())
    prow, a2, d, ud = s.split()
    assert np.array_equal(ints(got["prow"]), prow) and np.array_equal(ints(got["a2"]), a2)
    assert np.array_equal(floats(got["d"]).view(np.uint64), d.view(np.uint64))
    assert np.array_equal(floats(got["udiag"]).view(np.uint64), ud.view(np.uint64))
    for name, part in (("L1", B.PART_L1), ("L2", B.PART_L2), ("U", B.PART_U)):
        ptr, idx, val = s.factor_csr(part)
        assert np.array_equal(ints(got[name]), ptr)
        assert np.array_equal(ints(got[name + ".idx"]), idx)
        assert np.array_equal(floats(got[name + ".val"]).view(np.uint64), val.view(np.uint64))
    f = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, mu=1.0)
    oprow, oa2 = f.perm()
    assert np.array_equal(ints(got["prow"]), oprow) and np.array_equal(ints(got["a2"]), oa2)
    L2 = f.L2()
    assert np.array_equal(floats(got["L2.val"]), L2.val)
    # statuses reach C (ARG, SHAPE, ARG, CSR) and nothing changed on error
    assert got["errors"] == ["-1", "-2", "-1", "-3"]
    X = floats(got["sinv"]).reshape(prob.m - prob.n, prob.m - prob.n)
    assert np.array_equal(X.view(np.uint64), s.schur_inverse().view(np.uint64))


# ---------------------------------------------------------------------------
# the GPU calls from C
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def solve_client(tmp_path_factory):
    B.load()
    lib = _build.LIB
    exe = tmp_path_factory.mktemp("c_client") / "solve_client"
    subprocess.run(["gcc", "-std=c99", "-D_POSIX_C_SOURCE=199309L", "-O1", "-Wall", "-Werror", "-I",
                    os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_client", "solve_client.c"),
                    "-o", str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib),
                    "-Wl,-rpath,/usr/local/cuda/lib64"], check=True)
    return exe


@pytest.mark.gpu
def test_c_client_gpu_calls_match_oracle(solve_client, tmp_path):
    """rlsq_create / rlsq_factor / rlsq_solve / rlsq_batch_solve and the
    server calls, driven from C through include/rlsq.h alone on config 0:
    every x within 1e-6 of the oracle's LSMR solution (CG(2) correction),
    the batch's second system (2 b) gives 2 x, and an unfactored solve
    reports RLSQ_ERR_NOT_FACTORED."""
    prob = synth.config_problem(0)
    path = tmp_path / "ab.bin"
    with open(path, "wb") as f:
        np.array([prob.m, prob.n, prob.rowptr[-1]], dtype=np.int64).tofile(f)
        np.asarray(prob.rowptr, np.int64).tofile(f)
        np.asarray(prob.colidx, np.int32).tofile(f)
        np.asarray(prob.vals, np.float64).tofile(f)
        np.asarray(prob.b, np.float64).tofile(f)
    out = subprocess.run([str(solve_client), str(path)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    rows = {}
    for line in out.stdout.splitlines():
        key, *vals = line.split(" ")
        rows[key] = vals
    fo = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, mu=1.0)
    fo.set_correction(oracle.CG, 2)
    ref = oracle.lsmr(fo, prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, prob.b)

    def result(key):
        v = rows[key]
        return int(v[0]), int(v[1]), float.fromhex(v[2]), floats(v[3:])

    for key, scale in (("solve", 1.0), ("batch0", 1.0), ("batch1", 2.0), ("server", 1.0)):
        status, its, ratio, x = result(key)
        assert status == 0 and ratio < 1e-8, (key, status, ratio)
        assert abs(its - ref.its) <= 1, (key, its, ref.its)
        assert np.linalg.norm(x - scale * ref.x) <= 1e-6 * scale * np.linalg.norm(ref.x), key
    _, _, _, x0 = result("batch0")
    _, _, _, x1 = result("batch1")
    assert np.linalg.norm(x1 - 2.0 * x0) <= 1e-12 * np.linalg.norm(x1)
    assert rows["stats"] == ["1", "1"]
    assert rows["unfactored"] == ["-5"]  # RLSQ_ERR_NOT_FACTORED
