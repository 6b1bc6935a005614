"""End-to-end parity of the library against the FP64 oracle on the same
stored matrices (small sizes the oracle finishes in seconds)."""
import itertools

import numpy as np
import pytest

from _gpu_common import (UNIT, assert_indices_to_first_tie, device, run_problem, score_bound,  # noqa: F401
                         to_dev, torch, u_bound)
import bcur_inputs as bi
import oracle as orc

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_plain_fp64_512x1024():
    p = bi.plain_fp64_512x1024()
    ref, gpu, plan = run_problem(p)
    for side in ("col", "row"):
        d = np.max(np.abs(gpu[f"{side}_scores"] - ref[f"{side}_scores"]))
        assert d <= 1e-6 * np.max(ref[f"{side}_scores"]), side
        assert abs(np.sum(gpu[f"{side}_scores"]) - p.k) < 1e-9
    assert gpu["col_ok_draws"] == p.g_col and gpu["row_ok_draws"] == p.g_row
    assert gpu["col_idx"] == ref["col_idx"]
    assert gpu["row_idx"] == ref["row_idx"]
    np.testing.assert_array_equal(gpu["C"], ref["C"])
    np.testing.assert_array_equal(gpu["R"], ref["R"])
    assert _rel(gpu["U"], ref["U"]) < 1e-7
    assert abs(gpu["err"][1] - ref["rel"]) <= 1e-3
    assert abs(gpu["err"][0] - ref["err"]) <= 1e-9 * ref["err"]
    assert gpu["rank"] == (256, 192, 256, 192)


@pytest.mark.parametrize("sp,fp", [("f32", "f32")])
def test_haar_fp32_small(sp, fp):
    p = bi.scaled_haar(1536, 2048, 64, k=10, p=10, q=2, g_col=6, g_row=5, seed=7, rank=120,
                       noise=1e-4)
    ref, gpu, plan = run_problem(p, sp, fp)
    for side in ("col", "row"):
        d = np.max(np.abs(gpu[f"{side}_scores"] - ref[f"{side}_scores"]))
        assert d <= 1e-4 * np.max(ref[f"{side}_scores"]), (side, d)
    for side in ("col", "row"):
        n_ok = gpu[f"{side}_ok_draws"]
        assert gpu[f"{side}_idx"][:n_ok] == ref[f"{side}_idx"][:n_ok]
    assert abs(gpu["err"][1] - ref["rel"]) <= 1e-3
    assert abs(gpu["err"][0] - ref["err"]) <= 1e-4 * ref["err"]


@pytest.mark.parametrize("i", [0, 1, 2])
def test_biometric_batch_members(i):
    # the smallest members of the 512-matrix uneven batch
    probs = sorted(bi.batched_biometric(512), key=lambda q: q.m * q.n)[: 3]
    p = probs[i]
    ref, gpu, plan = run_problem(p, "f32", "f32")
    assert abs(gpu["err"][1] - ref["rel"]) <= 1e-3
    for side in ("col", "row"):
        n_ok = gpu[f"{side}_ok_draws"]
        assert gpu[f"{side}_idx"][:n_ok] == ref[f"{side}_idx"][:n_ok]


def test_ragged_blocks_fp64():
    rg = np.random.default_rng(3)
    m, n = 203, 331
    A = rg.standard_normal((m, 6)) @ rg.standard_normal((6, n)) + 0.01 * rg.standard_normal((m, n))
    col_off = np.array([0, 1, 40, 41, 100, 200, 300, 331], dtype=np.int64)
    row_off = bi.uniform_blocks(m, 25)                     # short last block
    p = bi.Problem("ragged", m, n, k=5, p=4, q=1, col_off=col_off, row_off=row_off, g_col=3,
                   g_row=4, seed=2, storage="f64", recipe={})
    ref, gpu, plan = run_problem(p, A=A)
    np.testing.assert_allclose(gpu["col_scores"], ref["col_scores"], atol=1e-9)
    np.testing.assert_allclose(gpu["row_scores"], ref["row_scores"], atol=1e-9)
    assert gpu["col_idx"][:gpu["col_ok_draws"]] == ref["col_idx"][:gpu["col_ok_draws"]]
    c, r, kc, kr = gpu["rank"]
    assert c == ref["C"].shape[1] and r == ref["R"].shape[0]
    assert abs(gpu["err"][0] - ref["err"]) <= 1e-8 * ref["err"]
    # C has more columns than A has rows, so U is not unique (the oracle's is
    # the minimum-norm one); the product CUR is, and it must agree.
    assert kc <= m and c > m
    cur_gpu = gpu["C"][:, :c] @ gpu["U"][:c, :r] @ gpu["R"][:r]
    cur_orc = ref["C"] @ ref["U"] @ ref["R"]
    assert _rel(cur_gpu, cur_orc) < 1e-8


def test_duplicate_blocks_with_replacement():
    """Drawing the same block twice makes C rank deficient: the library drops
    the dependent directions and still reaches the least-squares error."""
    rg = np.random.default_rng(4)
    A = rg.standard_normal((96, 128))
    off_c, off_r = bi.uniform_blocks(128, 16), bi.uniform_blocks(96, 16)
    import paper_1703_06065_gb300 as pkg

    dev = device()
    plan = pkg.Plan(96, 128, 4, 4, 1, off_c, off_r, 3, 2, dtype="f64", replacement=True)
    At = to_dev(A)
    ci = to_dev(np.array([2, 5, 2], dtype=np.int32))
    ri = to_dev(np.array([1, 1], dtype=np.int32))
    plan.fit(At, ci, ri)
    e = plan.error(At).cpu().numpy()
    C = orc.gather_columns(A, off_c, [2, 5, 2])
    R = orc.gather_rows(A, off_r, [1, 1])
    want = orc.residual(A, C, orc.fit_u(A, C, R), R)[0]
    assert abs(e[0] - want) <= 1e-9 * want
    c, r, kc, kr = plan.rank()
    assert (c, r, kc, kr) == (48, 32, 32, 16)


def test_brute_force_all_block_pairs():
    """12 x 16, s = 4: the library's fit and residual on every block choice
    equal the oracle's least-squares error."""
    import paper_1703_06065_gb300 as pkg

    dev = device()
    rg = np.random.default_rng(15)
    A = rg.standard_normal((12, 16))
    col_off, row_off = bi.uniform_blocks(16, 4), bi.uniform_blocks(12, 4)
    plan = pkg.Plan(12, 16, 3, 1, 1, col_off, row_off, 2, 2, dtype="f64")
    At = to_dev(A)
    for cj in itertools.combinations(range(4), 2):
        for ri in itertools.combinations(range(3), 2):
            plan.fit(At, to_dev(np.array(cj, np.int32)), to_dev(np.array(ri, np.int32)))
            e = plan.error(At).cpu().numpy()
            C = orc.gather_columns(A, col_off, cj)
            R = orc.gather_rows(A, row_off, ri)
            want = orc.residual(A, C, orc.fit_u(A, C, R), R)[0]
            assert abs(e[0] - want) <= 1e-10 * np.linalg.norm(A)


def test_nonfinite_input_is_reported():
    import paper_1703_06065_gb300 as pkg

    dev = device()
    p = bi.plain_fp64_512x1024()
    A = p.matrix()
    A[7, 9] = np.nan
    plan = pkg.Plan(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row, dtype="f64")
    plan.scores(to_dev(A), to_dev(p.omega().T))
    with pytest.raises(pkg.BcurError) as ei:
        plan.sync_status()
    assert ei.value.status == 5


def test_error_is_deterministic():
    p = bi.plain_fp64_512x1024()
    import paper_1703_06065_gb300 as pkg

    dev = device()
    A = to_dev(p.matrix())
    plan = pkg.Plan(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row, dtype="f64")
    ci = to_dev(np.arange(8, dtype=np.int32))
    ri = to_dev(np.arange(6, dtype=np.int32))
    plan.fit(A, ci, ri)
    a = plan.error(A).cpu().numpy()
    plan.fit(A, ci, ri)
    b = plan.error(A).cpu().numpy()
    assert a.tobytes() == b.tobytes()


HAAR_SMALL = dict(m=1536, n=2048, s=64, k=10, p=10, q=2, g_col=6, g_row=5, seed=7, rank=120)


@pytest.mark.parametrize("noise", [1e-4, 1e-3])
@pytest.mark.parametrize("sp,fp,score_cap", [
    ("bf16", "f32", 2e-2), ("f32", "bf16x3", 1e-4), ("bf16x3", "bf16x3", 1e-4),
    ("bf16", "bf16x3", 2e-2)])
def test_haar_tensor_core_paths(sp, fp, score_cap, noise):
    """Tensor-core sketch and/or fit against the FP64 oracle.
    - the relative error stays within 1e-3 of the oracle's (the benchmark's gate);
    - scores stay within the first-order rounding bound of the sketch's
      precision (score_bound) wherever that bound is below the largest
      score (at noise 1e-3 the gap at k = 10 is too small for one BF16
      term to resolve), and within the tighter cap observed on the
      quieter input;
    - block indices equal the oracle's up to the first draw that lands
      within the score perturbation of a CDF boundary;
    - U itself (not only CUR) is within the least-squares perturbation bound
      of the fit's precision (u_bound; the noisier input has kappa(C),
      kappa(R) near 20, the quieter one near 200);
    - CUR reproduces the oracle's."""
    h = HAAR_SMALL
    p = bi.scaled_haar(h["m"], h["n"], h["s"], k=h["k"], p=h["p"], q=h["q"], g_col=h["g_col"],
                       g_row=h["g_row"], seed=h["seed"], rank=h["rank"], noise=noise)
    ref, gpu, plan = run_problem(p, sp, fp)
    A = p.matrix().astype(np.float64)
    assert abs(gpu["err"][1] - ref["rel"]) <= 1e-3
    lmax = max(np.max(ref["col_scores"]), np.max(ref["row_scores"]))
    bound = score_bound(A, p.k, UNIT[sp], lmax)
    cap = score_cap * lmax if noise == 1e-4 else np.inf
    n_ok = assert_indices_to_first_tie(ref, gpu, p)
    if bound < lmax:
        # the sketch resolves the gap at k: the scores are pinned
        for side in ("col", "row"):
            d = np.max(np.abs(gpu[f"{side}_scores"] - ref[f"{side}_scores"]))
            assert d <= min(bound, cap), (side, d, bound)
        assert n_ok["col"] >= 1 and n_ok["row"] >= 1, n_ok
    c, r = gpu["rank"][0], gpu["rank"][1]
    assert (c, r) == (ref["C"].shape[1], ref["R"].shape[0])
    ub = u_bound(ref["C"], ref["R"], ref["rel"], UNIT[fp])
    assert _rel(gpu["U"][:c, :r], ref["U"]) <= ub, (_rel(gpu["U"][:c, :r], ref["U"]), ub)
    cur_gpu = gpu["C"][:, :c] @ gpu["U"][:c, :r] @ gpu["R"][:r]
    cur_orc = ref["C"] @ ref["U"] @ ref["R"]
    assert np.linalg.norm(cur_gpu - cur_orc) <= 1e-3 * np.linalg.norm(A)


def test_fp8_sketch_on_a_large_gap():
    """FP8 e4m3 sketch (4 significant bits) on the rank-10 Gaussian-product
    recipe stored in FP32: with sigma_10 / sigma_11 near 1e3 the first-order
    rounding bound of the scores is a few percent of the largest score, and
    the scores and the indices (up to a tie) must respect it.  (The error is
    not the sketch's business here: C of this input has kappa near 6500, so
    kappa^2 u exceeds 1 for every FP32-storage fit and e is set by the fit.)"""
    p = bi.plain_fp64_512x1024()
    p.storage = "f32"
    ref, gpu, plan = run_problem(p, "fp8", "bf16x3")
    A = p.matrix().astype(np.float64)
    lmax = max(np.max(ref["col_scores"]), np.max(ref["row_scores"]))
    bound = score_bound(A, p.k, UNIT["fp8"], lmax)
    assert bound < 0.1 * lmax
    for side in ("col", "row"):
        d = np.max(np.abs(gpu[f"{side}_scores"] - ref[f"{side}_scores"]))
        assert d <= bound, (side, d, bound)
    n_ok = assert_indices_to_first_tie(ref, gpu, p)
    assert n_ok["col"] >= 1 and n_ok["row"] >= 1, n_ok


def test_fp32_scores_to_1e6_on_a_large_gap():
    """The plain FP32 form (CUDA cores) on the noise-free rank-10 Gaussian
    product stored in FP32: the range finder is exact up to rounding
    (rank <= l) and the gap at k is huge, so the scores must agree with the
    FP64 oracle to a relative 1e-6 end to end, and every index exactly."""
    p = bi.Problem("lowrank10_f32", 512, 1024, k=10, p=10, q=2, col_off=bi.uniform_blocks(1024, 32),
                   row_off=bi.uniform_blocks(512, 32), g_col=8, g_row=6, seed=0, storage="f32",
                   recipe=dict(kind="small_lowrank", rank=10, noise=0.0))
    ref, gpu, plan = run_problem(p, "f32", "f32", force_oracle_idx=False)
    for side in ("col", "row"):
        d = np.max(np.abs(gpu[f"{side}_scores"] - ref[f"{side}_scores"]))
        assert d <= 1e-6 * np.max(ref[f"{side}_scores"]), (side, d)
    assert gpu["col_ok_draws"] == p.g_col and gpu["row_ok_draws"] == p.g_row
    assert gpu["col_idx"] == list(ref["col_idx"]) and gpu["row_idx"] == list(ref["row_idx"])
    assert abs(gpu["err"][1] - ref["rel"]) <= 1e-3


def test_fit_with_several_outer_cholesky_panels():
    """c = 1536 and r = 1280 selected columns / rows: the blocked Cholesky of
    each Gram runs over three outer panels of 512 columns, so the
    left-looking steps read the columns of earlier panels through the outer
    trailing updates.  The decomposition must still reproduce the oracle's
    CUR and relative error."""
    p = bi.scaled_haar(3072, 4096, 128, k=20, p=10, q=2, g_col=12, g_row=10, seed=17, rank=400,
                       noise=1e-4)
    ref, gpu, plan = run_problem(p, "bf16", "bf16x3")
    assert abs(gpu["err"][1] - ref["rel"]) <= 1e-3
    c, r = gpu["rank"][0], gpu["rank"][1]
    assert c == 1536 and r == 1280
    cur_gpu = gpu["C"][:, :c] @ gpu["U"][:c, :r] @ gpu["R"][:r]
    cur_orc = ref["C"] @ ref["U"] @ ref["R"]
    A = p.matrix().astype(np.float64)
    assert np.linalg.norm(cur_gpu - cur_orc) <= 1e-3 * np.linalg.norm(A)


def test_benchmark_code_paths_at_scale():
    """The benchmark's precisions (BF16 sketch, split-BF16 fit) on a case that
    takes the full-size code paths: c = 2560 selected columns (five outer
    Cholesky panels of 512), r = 2304, m = 4500 (not a multiple of the
    128-row MMA tile, so every product with A has a ragged edge) and a short
    last row block.  U must be within the least-squares perturbation bound
    of the split-BF16 unit round-off (kappa(C) near 40, kappa(R) near 24
    here), CUR and the error within their gates, and the indices equal up to
    the first tie."""
    p = bi.scaled_haar(4500, 6144, 128, k=20, p=10, q=2, g_col=20, g_row=18, seed=23, rank=400,
                       noise=1e-3)
    ref, gpu, plan = run_problem(p, "bf16", "bf16x3")
    assert abs(gpu["err"][1] - ref["rel"]) <= 1e-3
    c, r = gpu["rank"][0], gpu["rank"][1]
    assert (c, r) == (2560, 2304) and (c, r) == (ref["C"].shape[1], ref["R"].shape[0])
    n_ok = assert_indices_to_first_tie(ref, gpu, p)
    ub = u_bound(ref["C"], ref["R"], ref["rel"], UNIT["bf16x3"])
    assert _rel(gpu["U"][:c, :r], ref["U"]) <= ub, (_rel(gpu["U"][:c, :r], ref["U"]), ub)
    A = p.matrix().astype(np.float64)
    cur_gpu = gpu["C"][:, :c] @ gpu["U"][:c, :r] @ gpu["R"][:r]
    cur_orc = ref["C"] @ ref["U"] @ ref["R"]
    assert np.linalg.norm(cur_gpu - cur_orc) <= 1e-3 * np.linalg.norm(A)


def test_residual_refines_when_the_error_is_small():
    """Exactly rank-8 data: the true relative error is at the FP32 storage
    level, far below what one BF16 term resolves (about 3e-3 here).  The plan
    must detect that on the device and recompute the residual with BF16
    pairs, keeping the error within the 1e-3 target of the oracle's."""
    p = bi.Problem("rank8_exact", 1024, 1536, k=8, p=8, q=2, col_off=bi.uniform_blocks(1536, 64),
                   row_off=bi.uniform_blocks(1024, 64), g_col=3, g_row=3, seed=21, storage="f32",
                   recipe=dict(kind="small_lowrank", rank=8, noise=0.0))
    ref, gpu, plan = run_problem(p, "bf16", "bf16x3")
    assert ref["rel"] < 1e-5
    assert abs(gpu["err"][1] - ref["rel"]) <= 1e-3
    assert gpu["err"][1] < 5e-4, gpu["err"]  # one BF16 term would give about 3e-3


def test_residual_one_term_when_the_error_is_large():
    """Large relative error: one BF16 term is kept, and its deviation from
    the oracle follows the rounding model u^2 (1 - e^2) / (3 e), u = 2^-8."""
    p = bi.scaled_haar(1536, 2048, 64, k=10, p=10, q=2, g_col=6, g_row=5, seed=7, rank=120,
                       noise=1e-4)
    ref, gpu, plan = run_problem(p, "bf16", "bf16x3")
    e = ref["rel"]
    assert e > 0.1
    model = 0.00390625 ** 2 * (1 - e * e) / (3 * e)
    assert abs(gpu["err"][1] - e) <= max(5 * model, 1e-6)


@pytest.mark.parametrize("dtype,sp,fp", [("f64", "f64", "f64"), ("f32", "bf16", "bf16x3")])
def test_decompose_from_host_buffers(dtype, sp, fp):
    """bcur_decompose_host (host inputs copied in, host results copied out, one
    call) gives bit for bit the results of the device-pointer stage calls on
    the same inputs, and those meet the oracle's error gate."""
    import paper_1703_06065_gb300 as pkg

    dev = device()
    p = bi.plain_fp64_512x1024() if dtype == "f64" else bi.scaled_haar(
        1024, 1536, 64, k=10, p=10, q=2, g_col=5, g_row=4, seed=7, rank=120, noise=1e-4)
    A = p.matrix()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    om = np.ascontiguousarray(p.omega().T)
    A_h = torch.from_numpy(A).to(tdt).pin_memory()
    om_h = torch.from_numpy(om).to(tdt).pin_memory()
    uc_h = torch.from_numpy(p.u_col()).pin_memory()
    ur_h = torch.from_numpy(p.u_row()).pin_memory()
    plan = pkg.Plan(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row, dtype=dtype,
                    sketch_prec=sp, fit_prec=fp)
    out = plan.decompose_host(A_h, om_h, uc_h, ur_h)
    torch.cuda.synchronize()
    plan.sync_status()
    res = pkg.decompose(plan, A_h.to(dev), om_h.to(dev), uc_h.to(dev), ur_h.to(dev))
    torch.cuda.synchronize()
    for key in ("col_scores", "row_scores", "col_idx", "row_idx", "err"):
        assert torch.equal(out[key], res[key].cpu()), key
    assert torch.equal(out["U"], res["U"].cpu())
    ref = orc.block_cur(A.astype(np.float64), p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row,
                        p.omega(), p.u_col(), p.u_row())
    assert abs(float(out["err"][1]) - ref["rel"]) <= 1e-3
