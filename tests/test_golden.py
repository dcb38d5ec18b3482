"""The oracle against its recorded output (tests/golden/config0_oracle.json,
written by tests/golden/make_golden.py from the oracle alone): structure and
iteration counts exactly, float checksums bit for bit, norms to 1e-13."""
import json
import os
import sys

import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)

import make_golden  # noqa: E402


@pytest.fixture(scope="module")
def pair():
    with open(os.path.join(HERE, "config0_oracle.json")) as fh:
        stored = json.load(fh)
    return stored, make_golden.build()


def test_structure(pair):
    stored, now = pair
    for key in ("prow", "a2rows", "nnz", "levels", "sha256"):
        assert now[key] == stored[key], key


def test_solvers(pair):
    stored, now = pair
    assert now["anorm"] == pytest.approx(stored["anorm"], rel=1e-13)
    for solver in ("lsmr", "cgls"):
        for mode, rec in stored[solver].items():
            got = now[solver][mode]
            assert got["status"] == rec["status"] and got["its"] == rec["its"], (solver, mode)
            assert got["x_sha256"] == rec["x_sha256"], (solver, mode)
    for mode, rec in stored["lsmr"].items():
        assert now["lsmr"][mode]["ratio_hist_first"] == pytest.approx(rec["ratio_hist_first"], rel=1e-13)
