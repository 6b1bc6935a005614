"""The adaptive split-BF16 fit (fit_prec "bf16x3a") against the FP64 oracle.

The core products (W = A Q_R, M = Q_C^T W and the triangular products that
turn M into U) and the residual start with one BF16 term inside bcur_fit; the
device redoes them with three terms when the one-term residual is too coarse
for the error it reports (one term's rounding could move e by more than
2.5e-4, e < 0.031).  e depends on errors in M at second order only (the
perturbation Q_C dM Q_R^T is orthogonal to A - Q_C M Q_R^T), U at first order.
"""
import numpy as np
import pytest
import torch

from _gpu_common import UNIT, assert_indices_to_first_tie, bi, run_problem, u_bound

pytestmark = pytest.mark.gpu


def _rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def _rank8():
    return bi.Problem("rank8_exact", 1024, 1536, k=8, p=8, q=2,
                      col_off=bi.uniform_blocks(1536, 64), row_off=bi.uniform_blocks(1024, 64),
                      g_col=3, g_row=3, seed=21, storage="f32",
                      recipe=dict(kind="small_lowrank", rank=8, noise=0.0))


@pytest.mark.parametrize("noise", [1e-4, 1e-3])
def test_one_term_is_kept_when_the_error_is_large(noise):
    """Haar spectrum with noise: e is far above 0.031, so the device keeps one
    term.  The one-term residual it decided from is the error bcur_error
    reports, within the 1e-3 gate of the oracle's; the indices are the
    oracle's up to the first tie (the scores do not depend on the fit), and
    U is within the least-squares perturbation bound of one BF16 term."""
    p = bi.scaled_haar(1536, 2048, 64, k=10, p=10, q=2, g_col=6, g_row=5, seed=7, rank=120,
                       noise=noise)
    ref, gpu, plan = run_problem(p, "bf16", "bf16x3a")
    terms, est = plan.fit_terms()
    assert ref["rel"] > 0.1
    assert terms == 1 and est == gpu["err"][1], (terms, est, gpu["err"])
    assert abs(gpu["err"][1] - ref["rel"]) <= 1e-3
    assert_indices_to_first_tie(ref, gpu, p)
    _check_u_and_cur(ref, gpu)


def _check_u_and_cur(ref, gpu):
    """U within the least-squares perturbation bound of one BF16 term, and
    CUR within what that bound implies, ||C||_2 ||U - U_orc||_F ||R||_2 (the
    1e-3 * ||A|| check of the split fit is a 16-bit figure: one term leaves
    CUR about 2^-8 * ||A|| from the oracle's)."""
    c, r = gpu["rank"][0], gpu["rank"][1]
    assert (c, r) == (ref["C"].shape[1], ref["R"].shape[0])
    ub = u_bound(ref["C"], ref["R"], ref["rel"], UNIT["bf16"])
    du = _rel(gpu["U"][:c, :r], ref["U"])
    assert du <= ub, (du, ub)
    cur_gpu = gpu["C"][:, :c] @ gpu["U"][:c, :r] @ gpu["R"][:r]
    cur_orc = ref["C"] @ ref["U"] @ ref["R"]
    bound = (np.linalg.norm(ref["C"], 2) * np.linalg.norm(ref["R"], 2) * ub *
             np.linalg.norm(ref["U"]))
    assert np.linalg.norm(cur_gpu - cur_orc) <= bound


def test_three_terms_when_the_error_is_small_and_bitwise_equal_to_the_split_fit():
    """Exactly rank-8 data: e is at the FP32 storage level (one term would
    report about 3e-3), so the device redoes the core products and the
    residual with three terms.  The refined launches are the split fit's
    own, so U and the error equal those of a fit_prec "bf16x3" plan bit for
    bit."""
    p = _rank8()
    ref, gpu, plan = run_problem(p, "bf16", "bf16x3a")
    terms, est = plan.fit_terms()
    assert terms == 3 and 0.0 <= est < 0.031, (terms, est)
    ref3, gpu3, plan3 = run_problem(p, "bf16", "bf16x3")
    assert plan3.fit_terms() == (3, -1.0)
    np.testing.assert_array_equal(gpu["U"], gpu3["U"])
    np.testing.assert_array_equal(gpu["err"], gpu3["err"])
    assert abs(gpu["err"][1] - ref["rel"]) <= 1e-3 and gpu["err"][1] < 5e-4


def test_adaptive_fit_at_the_benchmark_code_paths():
    """c = 2560 (five outer Cholesky panels), r = 2304, m = 4500 (ragged
    against the 128-row MMA tile): one term is kept and the error, the
    indices, U and CUR meet their gates."""
    p = bi.scaled_haar(4500, 6144, 128, k=20, p=10, q=2, g_col=20, g_row=18, seed=23, rank=400,
                       noise=1e-3)
    ref, gpu, plan = run_problem(p, "bf16", "bf16x3a")
    terms, est = plan.fit_terms()
    assert terms == 1 and est == gpu["err"][1], (terms, est, gpu["err"])
    assert abs(gpu["err"][1] - ref["rel"]) <= 1e-3
    assert_indices_to_first_tie(ref, gpu, p)
    _check_u_and_cur(ref, gpu)


def test_adaptive_fit_is_deterministic():
    """The decision and every product are taken on the device in a fixed
    order: two fits of the same blocks give bit-identical U and errors, in
    both the one-term and the three-term outcome."""
    import paper_1703_06065_gb300 as pkg
    from _gpu_common import device, to_dev

    device()
    for p, want in ((_rank8(), 3),
                    (bi.scaled_haar(1536, 2048, 64, k=10, p=10, q=2, g_col=6, g_row=5, seed=7,
                                    rank=120, noise=1e-4), 1)):
        A = to_dev(p.matrix(), torch.float32)
        plan = pkg.Plan(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row,
                        dtype="f32", sketch_prec="bf16", fit_prec="bf16x3a")
        cs, rs = plan.scores(A, to_dev(p.omega().T, torch.float32))
        ci, ri, _, _ = plan.sample(cs, rs, to_dev(p.u_col()), to_dev(p.u_row()))
        U1 = plan.fit(A, ci, ri).clone()
        e1 = plan.error(A).clone()
        t1 = plan.fit_terms()
        U2 = plan.fit(A, ci, ri)
        e2 = plan.error(A)
        plan.sync_status()
        assert t1[0] == want and plan.fit_terms() == t1
        assert torch.equal(U1, U2) and torch.equal(e1, e2)


def test_fit_reuses_the_sketch_copy_of_a():
    """The adaptive fit takes A's BF16 hi half from the sketch when the
    scores were computed on the same A pointer, and splits A itself
    otherwise: both give bit-identical U and errors."""
    import paper_1703_06065_gb300 as pkg
    from _gpu_common import device, to_dev

    device()
    p = bi.scaled_haar(1536, 2048, 64, k=10, p=10, q=2, g_col=6, g_row=5, seed=7, rank=120,
                       noise=1e-4)
    A = to_dev(p.matrix(), torch.float32)
    A2 = A.clone()
    om = to_dev(p.omega().T, torch.float32)
    out = []
    for Ascores in (A, A2):
        plan = pkg.Plan(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row,
                        dtype="f32", sketch_prec="bf16", fit_prec="bf16x3a")
        cs, rs = plan.scores(Ascores, om)
        ci, ri, _, _ = plan.sample(cs, rs, to_dev(p.u_col()), to_dev(p.u_row()))
        U = plan.fit(A, ci, ri).clone()
        e = plan.error(A).clone()
        plan.sync_status()
        out.append((U, e))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
