"""Host-side checks of the C ABI: the library loads, exports every entry
point include/bcur.h declares, and validates descriptors without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1703_06065_gb300 import build

    build.build()
    import paper_1703_06065_gb300 as pkg

    return pkg.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "bcur.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bcur_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    from paper_1703_06065_gb300 import _lib

    names = header_functions()
    assert "bcur_plan" in names and "bcur_error" in names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(_lib.EXPORTS) == names
    assert lib.bcur_version().decode().count(".") == 2


def _desc(m=256, n=512, lda=None, k=8, p=8, q=1, s=32, g_col=4, g_row=3, dtype=1, sp=1, fp=1,
          replacement=0, col_off=None, row_off=None):
    from paper_1703_06065_gb300 import _lib

    co = np.asarray(col_off if col_off is not None else np.arange(0, n + 1, s), dtype=np.int64)
    ro = np.asarray(row_off if row_off is not None else np.arange(0, m + 1, s), dtype=np.int64)
    d = _lib.Desc()
    d.m, d.n, d.lda = m, n, lda or n
    d.a_dtype, d.k, d.p, d.q = dtype, k, p, q
    d.G_col, d.col_off = len(co) - 1, co.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.G_row, d.row_off = len(ro) - 1, ro.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.g_col, d.g_row, d.replacement = g_col, g_row, replacement
    d.sketch_prec, d.fit_prec = sp, fp
    return d, (co, ro)


def _plan(lib, **kw):
    d, keep = _desc(**kw)
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    st = lib.bcur_plan(ctypes.byref(d), None, ctypes.byref(h), ctypes.byref(ws))
    if st == 0:
        lib.bcur_destroy(h)
    return st, ws.value


@pytest.mark.parametrize("kw,want", [
    (dict(), 0),
    (dict(dtype=0, sp=0, fp=0), 0),
    (dict(sp=2, fp=2), 7),                   # TF32 stages are not offered by plans
    (dict(sp=3, fp=4), 0),                   # BF16 sketch, split-BF16 fit
    (dict(sp=4, fp=3), 7),                   # a one-term BF16 fit is refused
    (dict(sp=4, fp=4), 0),
    (dict(sp=5, fp=4), 0),                   # FP8 sketch, split-BF16 fit
    (dict(sp=1, fp=5), 1),                   # FP8 is a sketch precision only
    (dict(dtype=0, sp=5, fp=0), 1),          # FP8 sketch needs FP32 storage
    (dict(sp=6, fp=1), 1),                   # the adaptive split form is a fit precision
    (dict(sp=3, fp=6), 0),                   # BF16 sketch, adaptive split-BF16 fit
    (dict(dtype=0, sp=0, fp=6), 1),          # FP64 data with a BF16 fit
    (dict(sp=7, fp=4), 0),                   # FP8 sketch with 128 x 128 block scales
    (dict(sp=7, fp=6), 0),
    (dict(dtype=0, sp=7, fp=0), 1),          # block-scaled FP8 needs FP32 storage
    (dict(sp=3, fp=7), 1),                   # FP8 is a sketch precision only
    (dict(sp=8, fp=4), 1),
    (dict(lda=100), 1),                      # lda < n
    (dict(k=100, p=40), 1),                  # l > 128
    (dict(k=0), 1),
    (dict(q=17), 1),
    (dict(g_col=17), 1),                     # more blocks than exist, no replacement
    (dict(g_col=17, replacement=1), 0),      # fine with replacement
    (dict(dtype=0, sp=2, fp=0), 1),          # FP64 data with a TF32 stage
    (dict(dtype=1, sp=0, fp=1), 1),          # FP32 data with an FP64 stage
    (dict(col_off=[0, 32, 32, 512]), 1),     # empty block
    (dict(col_off=[0, 100, 500]), 1),        # does not end at n
    (dict(col_off=[0, 100, 512], g_col=2), 0),  # unequal blocks are allowed
    (dict(m=20, n=30, s=5, k=20, p=5, g_col=2, g_row=2), 1),  # l > m
])
def test_plan_validation(lib, kw, want):
    st, ws = _plan(lib, **kw)
    assert st == want
    if want == 0:
        assert ws > 0


def test_calls_before_workspace_and_null_plan(lib):
    d, keep = _desc()
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    assert lib.bcur_plan(ctypes.byref(d), None, ctypes.byref(h), ctypes.byref(ws)) == 0
    dummy = ctypes.c_void_p(0x1000)
    assert lib.bcur_scores(h, dummy, dummy, dummy, dummy) == 8      # ESTATE
    assert lib.bcur_fit(h, dummy, dummy, dummy, None, None, None) == 8
    assert lib.bcur_error(h, dummy, dummy) == 8
    t, e = ctypes.c_int32(), ctypes.c_double()
    assert lib.bcur_fit_terms(h, ctypes.byref(t), ctypes.byref(e)) == 8
    assert lib.bcur_fit_terms(h, None, None) == 1
    assert lib.bcur_fit_terms(None, ctypes.byref(t), None) == 1
    assert lib.bcur_set_workspace(h, ctypes.c_void_p(0x1001), ws.value) == 1  # misaligned
    assert lib.bcur_set_workspace(h, ctypes.c_void_p(0x1000), ws.value - 256) == 2
    lib.bcur_destroy(h)
    assert lib.bcur_scores(None, dummy, dummy, dummy, dummy) == 1
    assert lib.bcur_status_string(5).decode().startswith("non-finite")


def test_workspace_grows_with_blocks(lib):
    _, a = _plan(lib, g_col=2, g_row=2)
    _, b = _plan(lib, g_col=8, g_row=6)
    assert b > a


def _batch_plan(lib, items, q=2):
    arr = _lib_batch_items(lib, items)
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    st = lib.bcur_batch_plan(arr, len(items), q, None, ctypes.byref(h), ctypes.byref(ws))
    if st == 0:
        lib.bcur_batch_destroy(h)
    return st, ws.value


_GOOD = dict(m=512, n=1024, k=10, p=10, block=64, g_col=3, g_row=2)


@pytest.mark.parametrize("change,want", [
    ({}, 0),
    ({"p": 60}, 0),                       # l = 70: 128-row panels
    ({"p": 120}, 1),                      # l = 130 > 128
    ({"g_col": 17}, 1),                   # more blocks than G = 16
    ({"block": 256, "g_col": 3}, 1),      # c = 768 > 512
    ({"lda": 1022}, 1),                   # lda < n
    ({"lda": 1026}, 1),                   # lda not a multiple of 4
    ({"k": 0}, 1),
    ({"n": 1000, "block": 48}, 0),        # short last block
])
def test_batch_plan_validation(lib, change, want):
    it = dict(_GOOD, **change)
    st, ws = _batch_plan(lib, [_GOOD, it])
    assert st == want
    if want == 0:
        assert ws > 2 * 512 * 1024 * 4       # at least the two BF16 pairs of A


def test_batch_plan_rejects_empty_and_bad_q(lib):
    assert _batch_plan(lib, [])[0] == 1
    assert _batch_plan(lib, [_GOOD], q=17)[0] == 1
    # workspace grows with the batch
    w1 = _batch_plan(lib, [_GOOD])[1]
    w2 = _batch_plan(lib, [_GOOD, _GOOD])[1]
    assert w2 > w1


def test_new_entry_points_validate_on_the_host(lib):
    """Every argument error of the plan-free, boosting, host-buffer and
    settings calls is refused before anything touches the GPU."""
    d, keep = _desc()
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    assert lib.bcur_plan(ctypes.byref(d), None, ctypes.byref(h), ctypes.byref(ws)) == 0
    p = ctypes.c_void_p(0x1000)
    # host-buffer decomposition: no workspace yet, then a null plan
    assert lib.bcur_host_staging_bytes(h) >= 256 * 512 * 4
    assert lib.bcur_decompose_host(h, p, p, p, p, p, 1 << 40, None, None, None, None, None,
                                   p) == 8                       # ESTATE
    assert lib.bcur_decompose_host(None, p, p, p, p, p, 1 << 40, None, None, None, None, None,
                                   p) == 1
    assert lib.bcur_host_staging_bytes(None) == 0
    assert lib.bcur_rank_k_error(h, p, p) == 8                   # no scores / error yet
    assert lib.bcur_rank_k_error(None, p, p) == 1
    lib.bcur_destroy(h)
    # plan-free factorisation pieces
    assert lib.bcur_cholesky_inverse(p, 100, 0, p, p, p, ctypes.c_double(0.0), p, 256,
                                     None) == 1                  # w not a multiple of 64
    assert lib.bcur_cholesky_inverse(p, 128, 3, p, p, p, ctypes.c_double(0.0), p, 256,
                                     None) == 1                  # dtype
    assert lib.bcur_cholesky_inverse(p, 128, 0, p, p, p, ctypes.c_double(0.0), p, 128,
                                     None) == 1                  # scratch too small
    assert lib.bcur_cholesky_inverse(None, 128, 0, p, p, p, ctypes.c_double(0.0), p, 256,
                                     None) == 1
    assert lib.bcur_svd_small(p, 129, 0, p, p, p, p, 1 << 20, None, None) == 1
    assert lib.bcur_svd_small(p, 64, 0, p, p, p, p, 64, None, None) == 2  # work too small
    off = p
    assert lib.bcur_gather_blocks(p, 10, 8, 16, 0, 1, off, 2, p, 1, 8, p, 8, p, None) == 1  # lda < n
    assert lib.bcur_batch_set_fit(None, 4) == 1
    assert lib.bcur_batch_fit_terms(None, p) == 1
    assert lib.bcur_gemm_fp8_blocks(4, 16, 32, None, 32, p, 32, None, p, 1, 1, p, 16, None) == 1
    assert lib.bcur_gemm_fp8_blocks(4, 16, 32, p, 32, p, 32, None, None, 1, 1, p, 16, None) == 1
    assert lib.bcur_gemm_fp8_blocks(200, 500, 32, p, 32, p, 32, None, p, 1, 1, p, 500,
                                    None) == 7          # M >= 128: not the transposed path
    assert lib.bcur_gather_blocks(p, 16, 8, 16, 0, 2, off, 2, p, 1, 8, p, 8, p, None) == 1  # axis
    assert lib.bcur_gather_blocks(p, 16, 8, 16, 0, 1, off, 2, p, 1, 8, p, 4, p, None) == 1  # ldo < m
    # boosting's choice
    assert lib.bcur_boost_select(0, p, 3, None, 0, None, 0, None, 0, None, None, None, None,
                                 None, None) == 1                # t < 1
    assert lib.bcur_boost_select(2, p, 2, None, 0, None, 0, None, 0, None, None, None, None,
                                 None, None) == 1                # stride < 3
    assert lib.bcur_boost_select(2, p, 3, None, 0, None, 4, None, 0, None, p, None, None,
                                 None, None) == 1                # output without input
    assert lib.bcur_incoherence(None, 0, 4, 16, 16, p, p, None) == 1
    assert lib.bcur_incoherence(p, 3, 4, 16, 16, p, p, None) == 1        # dtype
    # settings
    assert lib.bcur_set_wait_budget_ns(0) == 1
    assert lib.bcur_set_wait_budget_ns(61_000_000_000) == 1
    assert lib.bcur_autotune_measured() == 0


def test_handles_of_the_other_kind_are_refused(lib):
    """Plan and batch handles are both opaque pointers; each carries a tag, so
    a single-matrix plan passed to a batch call is refused (BCUR_EINVAL) and
    left intact, instead of being written through as the wrong struct."""
    d, keep = _desc()
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    assert lib.bcur_plan(ctypes.byref(d), None, ctypes.byref(h), ctypes.byref(ws)) == 0
    terms = (ctypes.c_int32 * 4)()
    assert lib.bcur_batch_set_fit(h, 6) == 1
    assert lib.bcur_batch_fit_terms(h, ctypes.cast(terms, ctypes.c_void_p)) == 1
    from paper_1703_06065_gb300 import _lib

    io = (_lib.BatchIO * 1)()
    assert lib.bcur_batch_run(h, io, 0) == 1
    assert lib.bcur_batch_sync_status(h) == 1
    assert lib.bcur_batch_profile_count(h) == 0
    lib.bcur_batch_destroy(h)                     # not a batch: nothing is freed
    dummy = ctypes.c_void_p(0x1000)
    assert lib.bcur_scores(h, dummy, dummy, dummy, dummy) == 8   # still a plan (no workspace)
    lib.bcur_destroy(h)


def test_stage_plan_and_batch_calls_refuse_bad_arguments_on_the_host(lib):
    """The stage calls, the plan calls after bcur_plan and the batch calls
    refuse NULL operands, out-of-range sizes, a missing or short workspace
    and calls out of order before any work is enqueued."""
    p = ctypes.c_void_p(0x1000)
    F64, F32, BF16 = 0, 1, 3
    # GEMMs
    assert lib.bcur_gemm(4, 4, 4, None, 4, 0, p, 4, 0, p, 4, F32, F32, None) == 1
    assert lib.bcur_gemm(-1, 4, 4, p, 4, 0, p, 4, 0, p, 4, F32, F32, None) == 1
    assert lib.bcur_gemm(4, 4, 4, p, 4, 0, p, 4, 0, p, 4, F64, F32, None) == 1  # F64 data, F32
    assert lib.bcur_gemm_split(4, 4, 4, p, None, 4, 0, p, p, 4, 1, p, 4, None) == 1
    # the fused residual
    ws_need = lib.bcur_residual_workspace(300, 500, F32)
    assert ws_need >= 16
    assert lib.bcur_residual(None, 500, p, 8, p, 500, 300, 500, 8, F32, F32, p, p, ws_need,
                             None) == 1
    assert lib.bcur_residual(p, 400, p, 8, p, 500, 300, 500, 8, F32, F32, p, p, ws_need,
                             None) == 1                                  # ldx < n
    assert lib.bcur_residual(p, 500, None, 8, p, 500, 300, 500, 8, F32, F32, p, p, ws_need,
                             None) == 1                                  # r > 0 without P
    assert lib.bcur_residual(p, 500, p, 8, p, 500, 300, 500, 8, F32, F32, p, p, ws_need - 8,
                             None) == 2                                  # workspace too small
    assert lib.bcur_residual_noalloc(p, 500, p, 8, p, 500, 300, 500, 8, BF16, F32, p,
                                     None) == 1                          # BF16 needs prec BF16
    assert lib.bcur_residual_noalloc(p, 500, p, 8, p, 500, 300, 500, 8, 9, 9, p, None) == 1
    # block scores, stable rank, sampling
    off = (ctypes.c_int64 * 3)(0, 16, 32)
    assert lib.bcur_block_scores(None, F32, 4, 32, 32, off, 2, p, None) == 1
    assert lib.bcur_block_scores(p, F32, 4, 32, 16, off, 2, p, None) == 1     # ldf < h
    assert lib.bcur_block_scores(p, BF16, 4, 32, 32, off, 2, p, None) == 1    # dtype
    assert lib.bcur_block_stable_rank_workspace(4, 2) > 0
    assert lib.bcur_block_stable_rank(p, F32, 129, 32, 32, off, 2, p, p, 1 << 20, None) == 1
    assert lib.bcur_sample_blocks(None, 2, p, 1, 0, p, None, None) == 1
    assert lib.bcur_sample_blocks(p, 2, p, 3, 0, p, None, None) == 1          # g > G
    assert lib.bcur_sample_blocks(p, 0, p, 0, 0, p, None, None) == 1          # G < 1
    # Alg. 1 as printed
    assert lib.bcur_alg1_workspace(64, 32, None, 2, 8, 1, F32) == 0
    assert lib.bcur_alg1_workspace(64, 32, off, 2, 8, 1, F32) > 0
    # plan calls before a workspace, and with NULL arguments
    d, keep = _desc()
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    assert lib.bcur_plan(ctypes.byref(d), None, ctypes.byref(h), ctypes.byref(ws)) == 0
    c64 = ctypes.c_int64()
    assert lib.bcur_factors(h, p, p, p) == 8
    assert lib.bcur_rank(h, ctypes.byref(c64), ctypes.byref(c64), None, None) == 8
    assert lib.bcur_truncate(h, p, 4, p, p, p) == 8
    assert lib.bcur_sample(h, None, p, p, p, p, p, None, None) == 1
    lib.bcur_destroy(h)
    assert lib.bcur_factors(None, p, p, p) == 1
    assert lib.bcur_sync_status(None) == 1
    # batch calls
    arr = _lib_batch_items(lib, [_GOOD, _GOOD])
    hb = ctypes.c_void_p()
    wsb = ctypes.c_size_t()
    assert lib.bcur_batch_plan(arr, 2, 2, None, ctypes.byref(hb), ctypes.byref(wsb)) == 0
    cm, rm, nl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    assert lib.bcur_batch_dims(hb, 1, ctypes.byref(cm), ctypes.byref(rm), ctypes.byref(nl)) == 0
    assert (cm.value, rm.value) == (_GOOD["g_col"] * _GOOD["block"], _GOOD["g_row"] * _GOOD["block"])
    assert lib.bcur_batch_dims(hb, 2, None, None, None) == 1              # no item 2
    assert lib.bcur_batch_set_workspace(hb, ctypes.c_void_p(0x1001), wsb.value) == 1  # misaligned
    assert lib.bcur_batch_set_workspace(hb, ctypes.c_void_p(0x1000), wsb.value - 256) == 2
    lab, ms = ctypes.c_char_p(), ctypes.c_double()
    assert lib.bcur_batch_profile_count(hb) == 0
    assert lib.bcur_batch_profile_entry(hb, 0, ctypes.byref(lab), ctypes.byref(ms)) == 1
    lib.bcur_batch_destroy(hb)
    assert lib.bcur_batch_dims(None, 0, None, None, None) == 1
    assert lib.bcur_batch_set_stream(None, None) == 1
    assert lib.bcur_batch_profile(None, 1) == 1
    assert lib.bcur_batch_profile_count(None) == 0


def _lib_batch_items(lib, items):
    from paper_1703_06065_gb300 import _lib

    arr = (_lib.BatchItem * max(1, len(items)))()
    for i, it in enumerate(items):
        a = arr[i]
        a.m, a.n, a.lda = it["m"], it["n"], it.get("lda", it["n"])
        a.k, a.p, a.block = it["k"], it["p"], it["block"]
        a.g_col, a.g_row = it["g_col"], it["g_row"]
    return arr
