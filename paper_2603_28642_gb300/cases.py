"""Small, self-contained runs of single pieces of the path, for profilers.

Each case builds the 2M x 1M workload recipe (scaled by --scale), factors it
(p = 10, tau = 1e-2, mu = 1, CG(2)) and runs one piece on the GPU, with the
part worth capturing inside an NVTX range named `timed`:

    python -m paper_2603_28642_gb300.cases trsv --system U --schedule coop --scale 0.25
    python -m paper_2603_28642_gb300.cases trsv --system L1 --schedule binned --merge 0 --scale 0.5
    python -m paper_2603_28642_gb300.cases trsv --system L1 --schedule auto --merge 0 --autotune --scale 1
    python -m paper_2603_28642_gb300.cases iteration --scale 0.75
    python -m paper_2603_28642_gb300.cases products --scale 0.5

    python -m paper_2603_28642_gb300.cases setup --scale 1 --threads 8

`trsv` calls rlsq_trsv on one system a few times; `products` runs three LSMR
iterations with the default mappings (the A and A^T products); `iteration` autotunes and
profiles one preconditioned LSMR iteration; `setup` times the host-only set-up
(ILUP, split, level sets; no GPU needed) with a given thread count and prints a
checksum of the factor, which is the same for every thread count.  Everything
runs through the C ABI.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np

from . import binding as B
from . import synth

SYSTEMS = {"L1": B.SYS_L1, "L1t": B.SYS_L1T, "U": B.SYS_U, "Ut": B.SYS_UT}
SCHEDULES = {"auto": B.TRSV_AUTO, "level": B.TRSV_LEVEL, "syncfree": B.TRSV_SYNCFREE, "coop": B.TRSV_COOP,
             "wave": B.TRSV_WAVE, "binned": B.TRSV_BINNED}
FACTOR = dict(p=10, tau=1e-2, mu=1.0, correction=B.CORR_CG, cg_steps=2)


def _nvtx(push: bool):
    try:
        import torch

        if push:
            torch.cuda.nvtx.range_push("timed")
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_2603_28642_gb300.cases")
    sub = ap.add_subparsers(dest="case", required=True)
    t = sub.add_parser("trsv")
    t.add_argument("--system", choices=list(SYSTEMS), default="U")
    t.add_argument("--schedule", choices=list(SCHEDULES), default="coop")
    t.add_argument("--merge", type=int, default=1, help="levels fused per group (0: chosen per system)")
    t.add_argument("--autotune", action="store_true", help="autotune the mapping as the bench does")
    t.add_argument("--repeat", type=int, default=3)
    t.add_argument("--scale", type=float, default=0.25)
    pr = sub.add_parser("products")
    pr.add_argument("--scale", type=float, default=0.5)
    it = sub.add_parser("iteration")
    it.add_argument("--scale", type=float, default=0.75)
    it.add_argument("--fp32", action="store_true")
    su = sub.add_parser("setup")
    su.add_argument("--scale", type=float, default=1.0)
    su.add_argument("--threads", type=int, default=0, help="host threads (0: the library's default)")
    args = ap.parse_args(argv)

    prob = synth.config_problem(1, scale=args.scale)
    if args.case == "setup":
        import hashlib
        import time

        t0 = time.perf_counter()
        H = B.HostSetup(prob.m, prob.n, prob.rowptr, prob.colidx, prob.vals, p=FACTOR["p"], tau=FACTOR["tau"],
                        mu=FACTOR["mu"], host_threads=args.threads)
        dt = time.perf_counter() - t0
        h = hashlib.sha1()
        for a in H.split():
            h.update(np.ascontiguousarray(a).tobytes())
        for part in (B.PART_L1, B.PART_L2, B.PART_U):
            for a in H.factor_csr(part):
                h.update(np.ascontiguousarray(a).tobytes())
        threads = B.load().rlsq_setup_threads(args.threads, prob.m, prob.n)
        print(f"setup {prob.m} x {prob.n}: {dt:.2f} s on {threads} threads, sizes {H.sizes()}, "
              f"factor sha1 {h.hexdigest()[:16]}")
        return 0
    P = B.Problem.from_problem(prob)
    if args.case == "trsv":
        P.factor(**FACTOR, trsv_schedule=SCHEDULES[args.schedule], level_merge=args.merge,
                 autotune=1 if args.autotune else 0)
        b = np.random.default_rng(0).standard_normal(prob.n)
        _nvtx(True)
        for _ in range(args.repeat):
            x = P.trsv(SYSTEMS[args.system], b)
        _nvtx(False)
        print(f"trsv {args.system} ({args.schedule}, merge {args.merge}): |x| = {np.linalg.norm(x):.6e}")
    elif args.case == "products":
        # three LSMR iterations (the A and A^T products with the residual pair),
        # default mappings, no autotuning
        P.factor(**FACTOR)
        _nvtx(True)
        res = P.solve(prob.b, atol=0.0, maxit=3, check_every=1)
        _nvtx(False)
        print(f"products: {res.info['iterations']} iterations")
    else:
        info = P.factor(**FACTOR, precision=B.PREC_FP32 if args.fp32 else B.PREC_FP64, autotune=1)
        _nvtx(True)
        prof = P.profile(prob.b, warmup=1, iters=1)
        _nvtx(False)
        print(f"iteration: {prof['ms_per_iter']:.4f} ms, schedules {info['trsv_schedule']}, "
              f"levels {info['solve_levels']}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
