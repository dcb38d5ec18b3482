"""The bench's reference arm (the oracle on the host cores) runs without a GPU
and prints one JSON line with the keys the benchmark contract asks for: the
same metric and unit as the GPU arm, the requested steps and warm-up, a
cpu_baseline and an e2e object.  Under several ranks only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=e,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [line for line in out.stdout.splitlines() if line.startswith("{")]


def test_reference_arm_contract():
    lines = run_bench(["--impl", "reference", "--steps", "3", "--warmup", "1"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "preconditioned LSMR iterations/s" and d["unit"] == "iter/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 3 and d["warmup"] == 1
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1000.0 / d["value"]) < 1e-9 * d["ms_per_step"]
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["unit"] == "iter/s" and cb["value"] == d["value"]
    assert "3 runs of" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    assert run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"],
                     env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_gpu_arm_cpu_baseline_helper():
    """The GPU arm's cpu_baseline object comes from the same oracle sample."""
    sys.path.insert(0, ROOT)
    import bench

    cb = bench.cpu_oracle_sample(0.02, bench.full_nnz_estimate(1.0), iters_target_s=1.0)
    assert set(cb) == {"value", "unit", "cores", "kind", "sample", "time_to_tol"}
    assert cb["value"] > 0 and cb["unit"] == "iter/s" and cb["cores"] == 1 and cb["kind"] == "oracle"
    assert "scale 0.02" in cb["sample"]
    tt = cb["time_to_tol"]
    assert set(tt) >= {"config0_dense", "config1_scale0.02_cg2"} and len(tt) == 3
    for v in tt.values():
        assert v["factor_seconds"] > 0 and v["seconds_to_tol"] > 0 and v["ratio"] < 1e-8
        assert 0 < v["iterations"] < 2000
