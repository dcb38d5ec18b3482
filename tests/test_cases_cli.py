"""The profiling entry points (python -m paper_2603_28642_gb300.cases), CPU
side: the host-only `setup` case runs and reports the same factor checksum
for any thread count, and every subcommand parses the arguments the committed
profile summaries use (the GPU cases themselves run under the GPU tests'
conditions only)."""
import re

import pytest

from paper_2603_28642_gb300 import cases


def test_setup_case_same_factor_for_any_thread_count(capsys):
    sums = []
    for threads in (1, 2):
        assert cases.main(["setup", "--scale", "0.01", "--threads", str(threads)]) == 0
        out = capsys.readouterr().out
        m = re.search(r"factor sha1 ([0-9a-f]{16})", out)
        assert m, out
        sums.append(m.group(1))
    assert sums[0] == sums[1]


@pytest.mark.parametrize("argv", [
    ["trsv", "--system", "L1", "--schedule", "binned", "--merge", "0", "--scale", "0.5", "--repeat", "2"],
    ["trsv", "--system", "U", "--schedule", "coop", "--scale", "0.25"],
    ["iteration", "--scale", "0.5"],
    ["products", "--scale", "0.5"],
])
def test_gpu_case_arguments_parse(argv, monkeypatch):
    # stop right after parsing: the problem generator is the first call after it
    def stop(*a, **k):
        raise RuntimeError("parsed")

    monkeypatch.setattr(cases.synth, "config_problem", stop)
    with pytest.raises(RuntimeError, match="parsed"):
        cases.main(argv)
