"""rlsq_trsv_noalloc: the triangular solve for callers that cannot allocate
device memory while they run (latency-critical serving loops, where a
cudaMalloc may stall the device, or processes whose device memory is already
held by another allocator).  Its working memory is a static device array
instead of library-allocated buffers; the caller passes device input and
output arrays.

Checked here: its output equals that of the ordinary entry point rlsq_trsv
within the tolerance the other triangular-solve tests use (1e-12 relative),
on two calls in a row (the static array keeps the previous call's contents,
so the second call checks that everything that must start at zero is
cleared), for all four systems.  This file is collected last so that a run
stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2603_28642_gb300 import binding as B
from paper_2603_28642_gb300 import synth

pytestmark = pytest.mark.gpu

SYSTEMS = [B.SYS_L1, B.SYS_L1T, B.SYS_U, B.SYS_UT]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# (nonzeros per row of A, p): with p = 10 the factor rows average at most 12
# entries and the solves take one lane per row; with 24 per row and p = 30
# (13 entries per row of L1, 24 of U) they take groups of 4 and 8 lanes.
ROWS = [(6, 10), (24, 30)]


@pytest.mark.parametrize("sched", [B.TRSV_SYNCFREE, B.TRSV_LEVEL])
@pytest.mark.parametrize("rows", ROWS)
def test_noalloc_matches_trsv_on_two_calls(sched, rows):
    import torch

    per_row, p = rows
    prob = synth.sparse_problem(30_000, 20_000, per_row, seed=7)
    P = B.Problem.from_problem(prob)
    P.factor(mu=1.0, p=p, tau=1e-2, correction=B.CORR_NONE, trsv_schedule=sched)
    rng = np.random.default_rng(11)
    for which in SYSTEMS:
        for call in range(2):
            b = rng.standard_normal(prob.n)
            ref = P.trsv(which, b)
            bd = torch.from_numpy(b).cuda()
            xd = torch.full((prob.n,), float("nan"), dtype=torch.float64, device="cuda")
            B.trsv_noalloc(P, which, bd, xd)
            torch.cuda.synchronize()
            assert rel(xd.cpu().numpy(), ref) <= 1e-12, (which, call)


def test_noalloc_rejects_float32_factors():
    import torch

    prob = synth.config_problem(0)
    P = B.Problem.from_problem(prob)
    P.factor(mu=1.0, correction=B.CORR_NONE, precision=B.PREC_FP32)
    bd = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    xd = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    with pytest.raises(B.RlsqError) as e:
        B.trsv_noalloc(P, B.SYS_L1, bd, xd)
    assert e.value.code == -1
