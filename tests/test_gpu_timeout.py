"""Failure detection without a GPU fault: a bounded device-side wait that runs
out.

Every wait inside the tensor-core GEMM's main loop is bounded.  The test
lowers that bound from the host (bcur_set_wait_budget_ns) to 1 ns on a valid
input, so the first wait that does not succeed at once gives up: the kernel
records BCUR_ETIMEOUT in the plan's status word, drains the copies and
products it has issued, releases its tensor memory and returns.  The host
reads the status, restores the bound, and the next decomposition on the same
plan must succeed with results bit for bit equal to a run that never timed
out."""
import numpy as np
import pytest

from _gpu_common import device, to_dev, torch  # noqa: F401
import bcur_inputs as bi

pytestmark = pytest.mark.gpu


def test_wait_that_runs_out_is_reported_and_the_context_stays_usable():
    import paper_1703_06065_gb300 as pkg

    dev = device()
    L = pkg.load()
    p = bi.scaled_haar(4096, 4096, 256, k=20, p=10, q=2, g_col=4, g_row=4, seed=31, rank=200,
                       noise=1e-4)
    A = to_dev(p.matrix())
    om = to_dev(np.ascontiguousarray(p.omega().T), torch.float32)
    uc, ur = to_dev(p.u_col()), to_dev(p.u_row())
    plan = pkg.Plan(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row, dtype="f32",
                    sketch_prec="bf16", fit_prec="bf16x3")
    before = pkg.decompose(plan, A, om, uc, ur)
    plan.sync_status()
    before = {k: v.clone() for k, v in before.items()}
    try:
        assert L.bcur_set_wait_budget_ns(1) == 0
        plan.scores(A, om)          # K = 4096 per tile: the accumulators take microseconds
        torch.cuda.synchronize()
    finally:
        assert L.bcur_set_wait_budget_ns(2_000_000_000) == 0
    with pytest.raises(pkg.BcurError) as ei:
        plan.sync_status()
    assert ei.value.status == 6     # BCUR_ETIMEOUT
    plan.sync_status()              # the status word was cleared by the read
    after = pkg.decompose(plan, A, om, uc, ur)
    plan.sync_status()
    for key in ("col_scores", "row_scores", "col_idx", "row_idx", "U", "err"):
        assert torch.equal(before[key], after[key]), key


def test_wait_budget_is_validated():
    import paper_1703_06065_gb300 as pkg

    device()
    L = pkg.load()
    assert L.bcur_set_wait_budget_ns(0) == 1                 # BCUR_EINVAL
    assert L.bcur_set_wait_budget_ns(61_000_000_000) == 1
    assert L.bcur_set_wait_budget_ns(2_000_000_000) == 0
