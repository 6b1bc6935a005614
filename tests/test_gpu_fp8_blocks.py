"""FP8 e4m3 sketch with one scale per 128 x 128 block of A (sketch_prec
"fp8b") against the FP64 oracle, beside the per-row form ("fp8").

A block's scale varies along the K index of both products with A, so it
cannot come out of one accumulation: the GEMM accumulates each 128-deep K
block in its own tensor-memory buffer and the epilogue adds it scaled by the
block's factor (FP32 in registers).
"""
import numpy as np
import pytest

from _gpu_common import UNIT, assert_indices_to_first_tie, bi, run_problem, score_bound

pytestmark = pytest.mark.gpu


def test_block_scaled_fp8_on_a_large_gap():
    """The rank-10 recipe stored in FP32 (sigma_10 / sigma_11 near 1e3): the
    scores stay within the first-order rounding bound of e4m3 (u = 2^-4) and
    the indices equal the oracle's up to the first tie, as for per-row
    scales."""
    p = bi.plain_fp64_512x1024()
    p.storage = "f32"
    ref, gpu, plan = run_problem(p, "fp8b", "bf16x3")
    A = p.matrix().astype(np.float64)
    lmax = max(np.max(ref["col_scores"]), np.max(ref["row_scores"]))
    bound = score_bound(A, p.k, UNIT["fp8"], lmax)
    assert bound < 0.1 * lmax
    for side in ("col", "row"):
        d = np.max(np.abs(gpu[f"{side}_scores"] - ref[f"{side}_scores"]))
        assert d <= bound, (side, d, bound)
    n_ok = assert_indices_to_first_tie(ref, gpu, p)
    assert n_ok["col"] >= 1 and n_ok["row"] >= 1, n_ok


def test_block_scales_keep_quiet_column_blocks_that_row_scales_lose():
    """Every other 128-column block of a rank-10 matrix scaled by 1e-6, with
    a ragged last row and column block (m, n not multiples of 128).  A row's
    scale is set by its loud blocks, so per-row e4m3 maps the quiet entries
    to at most 448e-6 of the row's scale, below half the smallest subnormal
    (2^-10), i.e. to zero, and the quiet blocks score zero; per-block scales
    keep each quiet block at e4m3's own relative precision (2^-4 per entry),
    so its scores stay within 30% of the oracle's."""
    m, n, s = 700, 1000, 50
    p = bi.Problem("graded_rank10", m, n, k=10, p=10, q=2, col_off=bi.uniform_blocks(n, s),
                   row_off=bi.uniform_blocks(m, s), g_col=6, g_row=6, seed=3, storage="f32",
                   recipe=dict(kind="small_lowrank", rank=10, noise=0.0))
    A = p.matrix().astype(np.float32)
    quiet = np.zeros(n, dtype=bool)
    for b in range(0, (n + 127) // 128, 2):
        quiet[128 * b:128 * (b + 1)] = True
    A[:, quiet] *= np.float32(1e-6)
    qblocks = [g for g in range(len(p.col_off) - 1)
               if quiet[p.col_off[g]:p.col_off[g + 1]].all()]
    assert len(qblocks) >= 5
    refb, gpub, _ = run_problem(p, "fp8b", "bf16x3", A=A)
    refr, gpur, _ = run_problem(p, "fp8", "bf16x3", A=A)
    ref = refb["col_scores"][qblocks]
    assert np.all(ref > 0)
    rel_b = np.abs(gpub["col_scores"][qblocks] - ref) / ref
    rel_r = np.abs(gpur["col_scores"][qblocks] - ref) / ref
    assert np.max(rel_b) <= 0.3, rel_b
    assert np.min(rel_r) >= 0.9, rel_r          # flushed: the quiet blocks score about 0
    # the loud blocks and the row side meet the e4m3 bound in both forms
    lmax = max(np.max(refb["col_scores"]), np.max(refb["row_scores"]))
    bound = score_bound(A.astype(np.float64), p.k, UNIT["fp8"], lmax)
    for gpu in (gpub, gpur):
        assert np.max(np.abs(gpu["row_scores"] - refb["row_scores"])) <= bound
        loud = [g for g in range(len(p.col_off) - 1) if g not in qblocks]
        assert np.max(np.abs(gpu["col_scores"][loud] - refb["col_scores"][loud])) <= bound


@pytest.mark.parametrize("M,N,K", [(20, 700, 1000), (64, 1024, 768), (120, 4096, 333)])
def test_block_scaled_fp8_gemm_is_exact_to_fp32_accumulation(M, N, K):
    """The block-scaled FP8 product against an FP64 product of the same e4m3
    operands and factors: D = diag(s_m) sum_kb s_B(j/128, kb) A_kb B_kb^T.
    Products of e4m3 values are exact in FP32, so the only rounding is the
    FP32 accumulation of each 128-deep K block and of the scaled sum; block
    factors spread over six orders of magnitude and ragged M, N, K (K not a
    multiple of 128 or of 16) are covered."""
    import paper_1703_06065_gb300 as pkg
    from _gpu_common import device

    torch = pytest.importorskip("torch")
    dev = device()
    g = torch.Generator(device="cpu").manual_seed(M + N + K)
    Kp = (K + 15) // 16 * 16
    A = (torch.randn(M, Kp, generator=g) * 40).clamp(-440, 440)
    B = (torch.randn(N, Kp, generator=g) * 40).clamp(-440, 440)
    A8 = A.to(torch.float8_e4m3fn).to(dev)[:, :K]
    B8 = B.to(torch.float8_e4m3fn).to(dev)[:, :K]
    gn, gk = (N + 127) // 128, (K + 127) // 128
    bs = (10.0 ** (torch.rand(gn, gk, generator=g) * 6 - 3)).to(dev)
    sm = (torch.rand(M, generator=g) + 0.5).to(dev)
    D = pkg.gemm_fp8_blocks(A8, B8, bs, scale_m=sm)
    torch.cuda.synchronize()
    Ad = A8.double().cpu()
    Bd = B8.double().cpu()
    ref = torch.zeros(M, N, dtype=torch.float64)
    for kb in range(gk):
        k0, k1 = 128 * kb, min(K, 128 * kb + 128)
        part = Ad[:, k0:k1] @ Bd[:, k0:k1].T
        ref += part * bs.double().cpu()[:, kb].repeat_interleave(128)[:N].view(1, N)
    ref *= sm.double().cpu().view(M, 1)
    # FP32 rounding of each block sum (at most 128 terms: 128 * 2^-24 = 7.6e-6 of
    # the block's sum of |products|) and of the scaled accumulation, bounded
    # with the largest factor for every block
    scale = (Ad.abs() @ Bd.abs().T) * bs.double().cpu().max() * sm.double().cpu().max()
    err = (D.double().cpu() - ref).abs()
    assert torch.all(err <= 1e-5 * scale + 1e-30), float((err / (scale + 1e-30)).max())
