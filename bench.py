#!/usr/bin/env python
"""Benchmark of the preconditioned LSMR hot path on one GB300.

Workload (default): the single large sparse problem -- A is 2,000,000 x
1,000,000 with 8 random N(0,1) nonzeros per row plus a +-4 entry on a hidden
n-row subset (seed 1), b = A x_true + 1e-3 noise -- preconditioned by the
row-splitting ILUP(p=10, tau=1e-2, mu=1) with the CG(2) correction.

One step = one preconditioned LSMR iteration (A and A^T products, the full
preconditioner application, the scalar recurrences and vector updates).
`value` = iterations per second over K device-timed steps (CUDA events on the
library's stream, inputs resident in HBM, working set ~1.5 GB >> 129 MB L2).
`e2e` = the same metric through rlsq_solve with host buffers (b in, x out).
Also reported: time to ||A^T r|| / (||A|| ||r||) < 1e-8 in float64 and with
the float32 apply, the per-kernel-class breakdown, the roofline of the
dominant kernel class against the measured HBM copy bandwidth, and the CPU
oracle timed on a bounded sample.

`--impl reference` times the CPU oracle alone on the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

def host_threads():
    """Host threads for one rank's set-up: this process's CPUs shared among
    the ranks on the node."""
    try:
        cpus = len(os.sched_getaffinity(0))
    except AttributeError:
        cpus = os.cpu_count() or 1
    return max(1, cpus // max(1, int(os.environ.get("LOCAL_WORLD_SIZE", "1"))))


FACTOR = dict(p=10, tau=1e-2, mu=1.0, small=1e-10, correction=2, cg_steps=2, host_threads=host_threads())
# steps of the split-form CGLS run timed beside LSMR (it stalls above 1e-8)
CGLS_SPLIT_STEPS = 200
WORKLOAD = ("sparse LS m=2,000,000 n=1,000,000, 8 N(0,1) nnz/row + hidden +-4 diagonal (seed 1); "
            "ILUP(p=10, tau=1e-2, mu=1) row split, CG(2) correction; LSMR, atol 1e-8")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (testing only)")
    ap.add_argument("--cpu-scale", type=float, default=0.1, help="oracle sample size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the sampled sparse-dense, batched and served measurements")
    ap.add_argument("--workload", default="cfg1", choices=["cfg1", "sparse-dense", "batched", "served"],
                    help="cfg1: the headline line; the others print one line of their own at full size")
    ap.add_argument("--count", type=int, default=0, help="batched/served: problems or matrices (0 = recipe)")
    ap.add_argument("--requests", type=int, default=0, help="served: requests per arrival rate")
    return ap.parse_args()


# DRAM bytes (read + write) of ONE launch of a kernel class's solve kernel,
# from an ncu capture of the same kernel on the same recipe, keyed by (class,
# schedule the class ran with).  The bench reports it only when its dominant
# class ran that way.  The binned L1 solve was captured at half size
# (1M x 500k: 52.80 MB); its traffic grows with the rows and entries, so a
# full-size launch moves twice that.
MEASURED_TRAFFIC = {("trsv_L1", 5): 2 * 52.80e6}
CLASS_SYSTEM = {"trsv_L1": 0, "trsv_L1t": 1, "trsv_U": 2, "trsv_Ut": 3}
# solves per iteration of each triangular-solve class with CG(k): L1 and L1^T
# once each around the correction and once per CG step; U and U^T once
CLASS_SOLVES = {"trsv_L1": FACTOR["cg_steps"] + 1, "trsv_L1t": FACTOR["cg_steps"] + 1, "trsv_U": 1, "trsv_Ut": 1}


def finfo_ms_per_iter(P, prob):
    """A short untimed estimate of one iteration's time (for the clock soak)."""
    return P.profile(prob.b, warmup=1, iters=3)["ms_per_iter"] / 1000.0


# ---------------------------------------------------------------------------
def max_over_ranks(value: float, dist) -> float:
    """The largest `value` over all ranks (every rank gets it); `dist` is
    torch.distributed or None for one process."""
    if dist is None:
        return float(value)
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist) -> float:
    """The sum of `value` over all ranks (every rank gets it)."""
    if dist is None:
        return float(value)
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(items, rank: int, world: int):
    """The independent problems one rank solves: every world-th, from its rank
    on (sizes are drawn per problem, so the shares stay balanced)."""
    return list(items[rank::world])


def whole_job_rate(steps_per_rank: int, world: int, max_ms: float) -> float:
    """Iterations per second of the whole job: every rank runs its own replica
    for `steps_per_rank` iterations, timed by the slowest rank."""
    return world * steps_per_rank / (max_ms / 1000.0)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
class OracleSample:
    """The oracle as it stands (single thread) on the same recipe at a smaller
    size, factored once; run(its) times `its` LSMR+CG(2) iterations from x = 0
    and gives iterations/s scaled to the full workload by the nonzero ratio."""

    def __init__(self, cpu_scale: float, full_nnz: int):
        import oracle
        from paper_2603_28642_gb300 import synth

        self.oracle = oracle
        self.scale = cpu_scale
        self.prob = synth.config_problem(1, scale=cpu_scale)
        p = self.prob
        t0 = time.perf_counter()
        self.f = oracle.Factor(p.m, p.n, p.rowptr, p.colidx, p.vals, p=FACTOR["p"], tau=FACTOR["tau"],
                               mu=FACTOR["mu"], small=FACTOR["small"])
        self.f.set_correction(oracle.CG, FACTOR["cg_steps"])
        self.factor_seconds = time.perf_counter() - t0
        self.anorm = oracle.norm2(p.m, p.n, p.rowptr, p.colidx, p.vals)
        self.factor = p.nnz / full_nnz

    def run(self, its: int):
        p = self.prob
        t0 = time.perf_counter()
        r = self.oracle.lsmr(self.f, p.m, p.n, p.rowptr, p.colidx, p.vals, p.b, anorm=self.anorm, atol=0.0,
                             maxit=its)
        return r.its, time.perf_counter() - t0

    def seconds_per_iteration(self):
        its, dt = self.run(2)
        return dt / max(its, 1)

    def describe(self, its: int, dt: float, runs: int = 1):
        p = self.prob
        what = f"{its} LSMR+CG(2) iterations in {dt:.1f}s" if runs == 1 else \
            f"{runs} runs of {its // runs} LSMR+CG(2) iterations in {dt:.1f}s"
        return (f"config-1 recipe at scale {self.scale} (m={p.m:,}, n={p.n:,}, nnz={p.nnz:,}); {what} on 1 of "
                f"{os.cpu_count()} host cores; iter/s scaled by nnz ratio {self.factor:.4f}")

    def baseline(self, its: int, dt: float, runs: int = 1):
        return {"value": its / dt * self.factor, "unit": "iter/s", "cores": 1, "kind": "oracle",
                "sample": self.describe(its, dt, runs)}


def oracle_time_to_tol(prob, correction, cg_steps=2):
    """The oracle's factor time and LSMR time to ratio < 1e-8 on one problem
    (ILUP(p=10, tau=1e-2, mu=1), single thread)."""
    import oracle

    t0 = time.perf_counter()
    f = oracle.Factor(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, p=FACTOR["p"], tau=FACTOR["tau"],
                      mu=FACTOR["mu"], small=FACTOR["small"])
    f.set_correction(correction, cg_steps)
    t_factor = time.perf_counter() - t0
    t1 = time.perf_counter()
    r = oracle.lsmr(f, prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, prob.b)
    t_solve = time.perf_counter() - t1
    return {"m": prob.m, "n": prob.n, "nnz": prob.nnz, "factor_seconds": t_factor, "iterations": r.its,
            "seconds_to_tol": t_solve, "seconds_per_iteration": t_solve / max(r.its, 1), "ratio": r.ratio}


def cpu_oracle_sample(cpu_scale: float, full_nnz: int, iters_target_s: float = 12.0):
    """One bounded run of the oracle on the scaled recipe (about iters_target_s),
    then its factor time and time to tolerance on config 0 (dense S, as the
    recipe gives), on that sample (CG(2)) and on a mid-size problem of the
    batched recipe (CG(2))."""
    import oracle
    from paper_2603_28642_gb300 import synth

    o = OracleSample(cpu_scale, full_nnz)
    its = max(3, int(iters_target_s / max(o.seconds_per_iteration(), 1e-6)))
    done, dt = o.run(its)
    out = o.baseline(done, dt)
    t0 = time.perf_counter()
    r = o.oracle.lsmr(o.f, o.prob.m, o.prob.n, o.prob.rowptr, o.prob.colidx, o.prob.vals, o.prob.b,
                      anorm=o.anorm)
    sample_tol = {"m": o.prob.m, "n": o.prob.n, "nnz": o.prob.nnz, "factor_seconds": o.factor_seconds,
                  "iterations": r.its, "seconds_to_tol": time.perf_counter() - t0, "ratio": r.ratio}
    sample_tol["seconds_per_iteration"] = sample_tol["seconds_to_tol"] / max(r.its, 1)
    import numpy as np

    bn, bm, bd = synth.batch_problem_sizes(512)
    mid = int(np.argsort(bn)[len(bn) // 2])  # the median-size problem of the batched recipe
    mid_prob = synth.sparse_problem(int(bm[mid]), int(bn[mid]), int(bd[mid]), seed=3000 + mid)
    out["time_to_tol"] = {
        "config0_dense": oracle_time_to_tol(synth.config_problem(0), oracle.DENSE),
        f"config1_scale{cpu_scale}_cg2": sample_tol,
        f"batched_problem{mid}_cg2": oracle_time_to_tol(mid_prob, oracle.CG),
    }
    return out


def full_nnz_estimate(scale):
    # nnz of the full workload (computed once, cheap relative to the factor)
    from paper_2603_28642_gb300 import synth

    return synth.config_problem(1, scale=scale).nnz


# ---------------------------------------------------------------------------
def run_reference(args):
    """The oracle arm: the same metric on the host cores.  The sample is factored
    once (untimed, as the GPU arm's set-up is), then `warmup` untimed and
    `steps` timed steps of a fixed iteration count, sized so that all of them
    take about two minutes (at most 3 s a step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    o = OracleSample(args.cpu_scale, full_nnz_estimate(args.scale))
    per = o.seconds_per_iteration()
    k, w = max(1, args.steps), max(0, args.warmup)
    step_s = min(3.0, 120.0 / (k + w))
    its = max(2, int(step_s / max(per, 1e-6)))
    for _ in range(w):
        o.run(its)
    total_its, total_s = 0, 0.0
    for _ in range(k):
        done, dt = o.run(its)
        total_its += done
        total_s += dt
    cb = o.baseline(total_its, total_s, runs=k)
    v = cb["value"]
    out = {
        "impl": "reference", "metric": "preconditioned LSMR iterations/s", "value": v,
        "unit": "iter/s", "n_gpus": args.gpus, "steps": k, "warmup": w,
        "ms_per_step": 1000.0 / v if v else None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "scale": args.scale},
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def run_ours(args):
    import numpy as np
    import torch

    from paper_2603_28642_gb300 import binding as B
    from paper_2603_28642_gb300 import synth

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    B.load()

    # the single-problem path does not shard: every rank runs its own replica
    prob = synth.config_problem(1, scale=args.scale)
    P = B.Problem.from_problem(prob)
    finfo = P.factor(**FACTOR, precision=B.PREC_FP64, autotune=1)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    clk = Clocks(local)
    # about one second of the same iteration first, so that the clock sampler
    # (10 samples a second) sees this load; then W warm-up and K timed steps
    soak_t0 = time.perf_counter()
    P.profile(prob.b, warmup=0, iters=max(1, int(1.0 / max(finfo_ms_per_iter(P, prob), 1e-4))))
    soak_s = time.perf_counter() - soak_t0
    torch.cuda.nvtx.range_push("timed")
    prof = P.profile(prob.b, warmup=max(3, args.warmup), iters=args.steps)
    torch.cuda.nvtx.range_pop()
    clocks = clk.stop()
    clocks["window"] = f"{soak_s:.2f} s of the same iteration before the timed steps, and the timed steps"
    barrier()
    total_ms = max_over_ranks(prof["total_ms"], dist)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(args.steps, world, total_ms)

    # end to end through the public call with host buffers (b in, x out)
    barrier()
    t0 = time.perf_counter()
    e2e_res = P.solve(prob.b, atol=0.0, maxit=args.steps, check_every=8)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * e2e_res.info["iterations"] / e2e_s

    # time to tolerance: float64, unpreconditioned, then float32 apply (the
    # host factor is reused; only the device copy changes precision)
    tol64 = P.solve(prob.b)
    plain = P.solve(prob.b, plain=True)
    cgls = P.solve(prob.b, solver=B.SOLVER_CGLS, allow_fail=True)  # Algorithm 1, same preconditioner
    # Algorithm 1 with Algorithm 3 fed the residual split (the paper's form):
    # it stalls once entries are dropped, so a fixed number of steps is timed
    cgls_split = P.solve(prob.b, solver=B.SOLVER_CGLS_SPLIT, maxit=CGLS_SPLIT_STEPS, allow_fail=True)
    P.factor(**FACTOR, precision=B.PREC_FP32, autotune=1)
    tol32 = P.solve(prob.b)
    prof32 = P.profile(prob.b, warmup=3, iters=args.steps)
    x64 = tol64.x
    err32 = float(np.linalg.norm(tol32.x - x64) / np.linalg.norm(x64))

    # roofline of the dominant kernel class: the method's algorithmic bytes
    # (each stored entry of the factor system once, row pointers, vector in
    # and out) over the class's device time; the entries that level fusion
    # adds are reported beside it as overhead, not counted as achieved bytes
    hbm, src = peaks()
    cls = prof["classes"]
    dom = max(cls, key=lambda k: cls[k]["ms"])
    d = cls[dom]
    achieved = d["bytes"] / (d["ms"] / 1000.0) / 1e9
    sched = finfo["trsv_schedule"][CLASS_SYSTEM[dom]] if dom in CLASS_SYSTEM else None
    per_launch = d["bytes"] / max(1, CLASS_SOLVES.get(dom, d["launches"]))
    traffic = MEASURED_TRAFFIC.get((dom, sched))
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "peak_source": src,
            "algorithmic_bytes_per_launch": per_launch,
            "traffic": traffic, "traffic_over_algorithmic": traffic / per_launch if traffic else None,
            "iteration_achieved": prof["bytes_per_iter"] / (ms_per_step / 1000.0) / 1e9,
            "iteration_frac": prof["bytes_per_iter"] / (ms_per_step / 1000.0) / 1e9 / hbm,
            "bytes_per_iteration": prof["bytes_per_iter"]}
    if dom in CLASS_SYSTEM:
        w = CLASS_SYSTEM[dom]
        own = finfo["nnz_L1"] if w < 2 else finfo["nnz_U"]
        roof["schedule_entries_over_factor_entries"] = finfo["solve_entries"][w] / max(1, own)
    launches = sum(c["launches"] for c in cls.values())

    out = {
        "metric": "preconditioned LSMR iterations/s", "value": value, "unit": "iter/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "scale": args.scale, "l2": "inputs larger than L2",
                   "m": prob.m, "n": prob.n, "nnz_A": prob.nnz,
                   "nnz_L1": finfo["nnz_L1"], "nnz_L2": finfo["nnz_L2"], "nnz_U": finfo["nnz_U"],
                   "levels": [finfo["levels_L1"], finfo["levels_L1t"], finfo["levels_U"],
                              finfo["levels_Ut"]],
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": e2e_value, "unit": "iter/s", "h2d_bytes_per_step": 8 * prob.m / args.steps,
                "d2h_bytes_per_step": 8 * prob.n / args.steps, "wall_s": e2e_s},
        "time_to_tol": {
            "fp64": {"iterations": tol64.info["iterations"], "seconds": tol64.info["solve_seconds"],
                     "ratio": tol64.info["ratio"], "status": tol64.status},
            "fp32_apply": {"iterations": tol32.info["iterations"],
                           "seconds": tol32.info["solve_seconds"], "ratio": tol32.info["ratio"],
                           "x_rel_diff_vs_fp64": err32, "status": tol32.status,
                           "iter_per_s": 1000.0 / prof32["ms_per_iter"]},
            "unpreconditioned": {"iterations": plain.info["iterations"],
                                 "seconds": plain.info["solve_seconds"], "status": plain.status},
            "cgls_fp64": {"iterations": cgls.info["iterations"], "seconds": cgls.info["solve_seconds"],
                          "ratio": cgls.info["ratio"], "status": cgls.status,
                          "x_rel_diff_vs_lsmr": float(np.linalg.norm(cgls.x - tol64.x) / np.linalg.norm(tol64.x))},
            "cgls_split_fp64": {"iterations": cgls_split.info["iterations"],
                                "seconds": cgls_split.info["solve_seconds"],
                                "ms_per_iter": 1000.0 * cgls_split.info["solve_seconds"]
                                / max(1, cgls_split.info["iterations"]),
                                "ratio": cgls_split.info["ratio"], "status": cgls_split.status,
                                "x_rel_diff_vs_lsmr": float(np.linalg.norm(cgls_split.x - tol64.x)
                                                            / np.linalg.norm(tol64.x))},
        },
        "factor_seconds": finfo["factor_seconds"],
        "ilup_seconds": finfo["ilup_seconds"], "ilup_threads": finfo["ilup_threads"],
        "roofline": roof,
        "kernel_classes": {k: {"ms": v["ms"], "launches": v["launches"],
                               "GBps": v["bytes"] / (v["ms"] / 1000.0) / 1e9} for k, v in cls.items()},
        "gpu_launches": launches * args.steps,
        # products in the sliced layout (bits: 1 A, 2 A^T, 4 L2, 8 L2^T), as the autotuner chose
        "sliced_products": finfo["sliced_products"],
        "clocks": clocks,
    }
    if rank == 0 and not args.no_extras:
        # CG steps on the implicit S (Algorithm 3, step 2; the paper uses 2): time
        # to tolerance with 3 and 4 steps, float64, on the same host factor
        more = {}
        for k in (3, 4):
            try:
                P.factor(**{**FACTOR, "cg_steps": k}, precision=B.PREC_FP64, autotune=1)
                r = P.solve(prob.b, allow_fail=True)
                more[f"cg{k}"] = {"iterations": r.info["iterations"], "seconds": r.info["solve_seconds"],
                                  "ratio": r.info["ratio"], "status": r.status,
                                  "x_rel_diff_vs_cg2": float(np.linalg.norm(r.x - x64) / np.linalg.norm(x64))}
            except Exception as e:  # recorded, so the headline line still prints
                more[f"cg{k}"] = {"error": f"{type(e).__name__}: {e}"}
        out["time_to_tol"]["fp64_more_cg_steps"] = more
        # CG steps on S stopped adaptively: once ||r_j|| <= eta ||r_0||, at most 8
        adaptive = {}
        for eta in (0.3, 0.1):
            try:
                P.factor(**{**FACTOR, "cg_steps": 8}, cg_tol=eta, precision=B.PREC_FP64, autotune=1)
                r = P.solve(prob.b, allow_fail=True)
                adaptive[f"eta{eta}"] = {"iterations": r.info["iterations"], "seconds": r.info["solve_seconds"],
                                         "ratio": r.info["ratio"], "status": r.status,
                                         "x_rel_diff_vs_cg2": float(np.linalg.norm(r.x - x64) / np.linalg.norm(x64))}
            except Exception as e:  # recorded, so the headline line still prints
                adaptive[f"eta{eta}"] = {"error": f"{type(e).__name__}: {e}"}
        out["time_to_tol"]["fp64_adaptive_cg_steps"] = adaptive
        try:
            out["dense_correction"] = measure_dense_correction()
        except Exception as e:  # recorded, so the headline line still prints
            out["dense_correction"] = {"error": f"{type(e).__name__}: {e}"}
    del P
    if rank == 0 and not args.no_extras:
        # the other forms, sampled so the default run stays within minutes
        for key, fn in (("sparse_dense", lambda: measure_sparse_dense(args.scale)),
                        ("batched_sample", lambda: measure_batched(512, first=64, sample=8)),
                        ("served_sample", lambda: measure_served(16, n_hi=20000, rates=(100, 1000, 5000),
                                                                 requests=200))):
            try:
                out[key] = fn()
            except Exception as e:  # recorded, so the headline line still prints
                out[key] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_oracle_sample(args.cpu_scale, prob.nnz)
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the other forms: sparse-dense, batched, served
# ---------------------------------------------------------------------------
def factor_all(problems, threads=None, tune=True, **kw):
    """Creates and factors problems concurrently (the host set-up releases the
    GIL); then, one problem at a time so that the timings do not disturb each
    other, tunes each problem's own product lanes (autotune = 2; the host
    factor is reused), which is what its slot in a batch runs with."""
    from concurrent.futures import ThreadPoolExecutor

    from paper_2603_28642_gb300 import binding as B

    def one(p):
        P = B.Problem.from_problem(p)
        # the pool already runs one set-up per CPU
        P.factor(**{"host_threads": 1, **kw})
        return P

    with ThreadPoolExecutor(threads or host_threads()) as ex:
        hs = list(ex.map(one, problems))
    if tune:
        for P in hs:
            P.factor(**{"host_threads": 1, **kw}, autotune=2)
    return hs


def measure_sparse_dense(scale=1.0):
    """Sparse-dense problem (n = 500,000, 1,000,000 sparse rows, 200 dense rows):
    float32 apply, float64 recurrences, CG(2)."""
    from paper_2603_28642_gb300 import binding as B
    from paper_2603_28642_gb300 import synth

    prob = synth.config_problem(2, scale=scale)
    P = B.Problem.from_problem(prob)
    info = P.factor(**FACTOR, precision=B.PREC_FP32, autotune=1)
    prow, a2, _, _ = P.split()
    in_a2 = bool(set(prob.dense_rows.tolist()) <= set(a2.tolist()))
    prof = P.profile(prob.b, warmup=3, iters=20)
    tol = P.solve(prob.b)
    cls = prof["classes"]
    dense = cls.get("dense", {"ms": 0.0, "bytes": 0.0})
    return {
        "m": prob.m, "n": prob.n, "dense_rows": info["n_dense_rows"], "dense_rows_in_A2": in_a2,
        "iter_per_s": 1000.0 / prof["ms_per_iter"], "ms_per_iter": prof["ms_per_iter"],
        "time_to_tol_s": tol.info["solve_seconds"], "iterations": tol.info["iterations"],
        "ratio": tol.info["ratio"], "status": tol.status,
        "dense_gemv_GBps": dense["bytes"] / (dense["ms"] / 1000.0) / 1e9 if dense["ms"] else None,
        "iteration_GBps": prof["bytes_per_iter"] / (prof["ms_per_iter"] / 1000.0) / 1e9,
    }


def measure_dense_correction(n=100_000, m2=512):
    """The dense correction on a quasi-square problem (n = 100,000, m - n =
    512, 8 per row, hidden +-4 diagonal): the set-up with S^{-1} formed on the
    GPU against the same set-up on the host threads (fresh handles; the ILUP
    time is reported beside each), and the time to tolerance in float64."""
    from paper_2603_28642_gb300 import binding as B
    from paper_2603_28642_gb300 import synth

    prob = synth.sparse_problem(n + m2, n, 8, seed=5, hidden_diag=True)
    kw = dict(p=10, tau=1e-2, mu=1.0, correction=B.CORR_DENSE)
    # first use of the device formation (library handles, lazy module loads) kept out of the timing
    small = synth.config_problem(0)
    B.Problem.from_problem(small).factor(**kw)
    out = {"m": prob.m, "n": prob.n, "m_minus_n": m2}
    for name, host in (("device", 0), ("host", 1)):
        P = B.Problem.from_problem(prob)
        info = P.factor(**kw, dense_host=host)
        out[f"factor_s_sinv_on_{name}"] = info["factor_seconds"]
        out[f"ilup_s_{name}_run"] = info["ilup_seconds"]
        if host == 0:
            r = P.solve(prob.b)
            out.update(iterations=r.info["iterations"], seconds_to_tol=r.info["solve_seconds"], status=r.status)
        del P
    return out


def measure_batched(count=512, first=None, sample=16, rank=0, world=1, dist=None):
    """Batched form: the first `first` problems of the 512-problem recipe solved
    together (float32 apply, float64 recurrences), against the same problems
    solved one at a time in float64 (timed on `sample` of them; all of them
    in the full `--workload batched` run).  With several
    ranks every rank solves its shard of the problems (no collective on the
    data path); the job's time is the slowest rank's and its iterations are all
    ranks' iterations."""
    from paper_2603_28642_gb300 import binding as B
    from paper_2603_28642_gb300 import synth

    every = synth.batch_problems(count, first=first)
    probs = shard(every, rank, world)
    hs = factor_all(probs, mu=1.0, p=10, tau=1e-2, correction=B.CORR_AUTO, cg_steps=2,
                    precision=B.PREC_FP32)
    B.batch_solve(hs[:2], [p.b for p in probs[:2]])  # warm-up (graph capture, lazy loading)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    xs, infos, code = B.batch_solve(hs, [p.b for p in probs])
    wall = max_over_ranks(time.perf_counter() - t0, dist)
    its = sum_over_ranks(sum(i["iterations"] for i in infos), dist)
    code = -int(max_over_ranks(abs(code), dist))  # the worst status (0 or a negative error)
    worst = max_over_ranks(max(i["ratio"] for i in infos), dist)
    # one at a time, float64 apply, the same problems (a sample of each shard)
    step = max(1, len(probs) // max(1, sample // world))
    idx = list(range(0, len(probs), step))[:max(1, sample // world)]
    t_one, its_one = 0.0, 0
    for k in idx:
        hs[k].factor(mu=1.0, p=10, tau=1e-2, correction=B.CORR_AUTO, cg_steps=2, precision=B.PREC_FP64)
        hs[k].solve(probs[k].b)  # warm-up of this handle's graph
        t1 = time.perf_counter()
        r = hs[k].solve(probs[k].b)
        t_one += time.perf_counter() - t1
        its_one += r.info["iterations"]
    t_one = sum_over_ranks(t_one, dist)
    its_one = sum_over_ranks(its_one, dist)
    n_one = sum_over_ranks(len(idx), dist)
    # all problems one at a time on one GPU: measured when every problem was
    # timed, else the sample's mean time per problem times the count
    one_total = t_one if int(n_one) == len(every) else t_one / n_one * len(every)
    return {
        "problems": len(every), "ranks": world, "sum_n": int(sum(p.n for p in every)),
        "sum_nnz": int(sum(p.nnz for p in every)),
        "status": code, "iterations_total": int(its), "batched_wall_s": wall,
        "aggregate_iter_per_s": its / wall,
        "one_at_a_time_fp64_s": one_total, "one_at_a_time_timed": int(n_one),
        "one_at_a_time_measured": int(n_one) == len(every),
        "one_at_a_time_iter_per_s": its_one / t_one if t_one else None,
        "speedup_time_to_tol": one_total / wall if wall else None,
        "max_ratio": worst,
    }


def measure_served(nmat=64, n_hi=200000, rates=(100, 1000, 5000), requests=500, rank=0, world=1, dist=None):
    """Served form: Poisson arrivals of new right-hand sides for resident
    matrices (m = 1.5 n), float32 apply, float64 recurrences, 150 GB budget.
    With several ranks, each rank owns whole matrices (balanced by nonzeros)
    and serves the requests for them on its own GPU; the request stream is
    the same on every rank, and the job's p50 / p99 are over all requests."""
    import numpy as np

    from paper_2603_28642_gb300 import binding as B
    from paper_2603_28642_gb300 import serving, synth

    mats = synth.serving_matrices(nmat, n_hi=n_hi)
    owner = serving.owners([p.nnz for p in mats], world)
    mine = [k for k in range(nmat) if owner[k] == rank]
    hs = dict(zip(mine, factor_all([mats[k] for k in mine], mu=1.0, p=10, tau=1e-2, correction=B.CORR_AUTO,
                                    cg_steps=2, precision=B.PREC_FP32)))
    out = {"matrices": nmat, "ranks": world, "n_max": int(max(p.n for p in mats)),
           "sum_n": int(sum(p.n for p in mats)), "budget_bytes": 150 * 2**30, "rates": []}
    for rate in rates:
        srv = B.Server(hbm_budget_bytes=150 * 2**30, max_slots=64)
        ids = {k: srv.register(P) for k, P in hs.items()}
        rng = np.random.default_rng(rate)
        which = rng.integers(0, nmat, size=requests)
        arrive = synth.poisson_arrivals(rate, requests, seed=rate)
        todo = serving.requests_for(which, owner, rank)
        rhs = {int(r): synth.serving_rhs(mats[int(which[r])], int(r)) for r in todo}
        lat_ms = []
        pending = {}
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        sent = 0
        while sent < len(todo) or pending:
            now = time.perf_counter() - t0
            while sent < len(todo) and arrive[todo[sent]] <= now:
                r = int(todo[sent])
                pending[srv.submit(ids[int(which[r])], rhs[r])] = int(which[r])
                sent += 1
            for t, w in list(pending.items()):
                got = srv.poll(t, mats[w].n)
                if got is not None:
                    lat_ms.append(1000.0 * got[1]["solve_seconds"])  # submit -> result, as the server counts it
                    del pending[t]
            time.sleep(0.0005)
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        merged = serving.merge_latencies(serving.gather(lat_ms, dist))
        wall = max(serving.gather(wall, dist))
        out["rates"].append({"rate_per_s": rate, "requests": requests, "p50_ms": merged["p50_ms"],
                             "p99_ms": merged["p99_ms"], "mean_ms": merged["mean_ms"],
                             "solves_per_s": merged["requests"] / wall if wall else None,
                             "ticks": st["ticks"], "tick_ms": st["tick_ms"], "tick_device_ms": st["tick_device_ms"],
                             "peak_state_bytes": st["peak_bytes"]})
    return out


def run_workload(args):
    """One JSON line for a non-default workload at its full recipe size.  Under
    torchrun the batched form shards its problems over the ranks and the
    served form routes each request to the rank owning its matrix (no
    collective on the data path); the sparse-dense form runs on rank 0 alone."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    dist = None
    if args.workload in ("batched", "served") and world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    elif rank != 0:
        return
    n_gpus = world if dist is not None else 1
    if args.workload == "sparse-dense":
        r = measure_sparse_dense(args.scale)
        metric, value, unit = "preconditioned LSMR iterations/s (sparse-dense)", r["iter_per_s"], "iter/s"
    elif args.workload == "batched":
        r = measure_batched(args.count or 512, sample=args.count or 512, rank=rank if dist is not None else 0,
                            world=n_gpus, dist=dist)
        metric, value, unit = "batched aggregate LSMR iterations/s", r["aggregate_iter_per_s"], "iter/s"
    else:
        r = measure_served(args.count or 64, requests=args.requests or 2000, rates=(100, 300, 1000, 3000, 5000),
                           rank=rank if dist is not None else 0, world=n_gpus, dist=dist)
        metric, value, unit = "served solves/s at the highest rate", r["rates"][-1]["solves_per_s"], "solves/s"
    if rank == 0:
        print(json.dumps({"metric": metric, "value": value, "unit": unit, "n_gpus": n_gpus, "higher_is_better": True,
                          "scaling": "strong" if args.workload in ("batched", "served") else "weak",
                          "dtype": "f32 apply / f64 recurrences", "data": "synthetic",
                          "config": {"workload": args.workload}, "result": r}))
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "cfg1":
        run_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
