"""Block CUR (arXiv 1703.06065) hot path on GB300: Python binding.

Thin wrappers with the C ABI's names.  Tensors must live on the current CUDA
device; the library runs on torch's current stream.  Nothing here computes:
the arithmetic of every stage is in libbcur.so.

Typical use::

    plan = Plan(m, n, k=50, p=10, q=2, col_off=..., row_off=..., g_col=16, g_row=16,
                dtype="f32", sketch_prec="tf32", fit_prec="tf32")
    cs, rs = plan.scores(A, omega)            # Def. 2 block leverage scores
    ci, ri, cp, rp = plan.sample(cs, rs, u_col, u_row)
    U = plan.fit(A, ci, ri)                   # U = C^+ A R^+
    err, rel, norm_a = plan.error(A).tolist()  # ||A - CUR||_F without forming CUR
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_int64, c_size_t, c_void_p
from typing import Optional, Sequence

import numpy as np

from . import _lib
from ._lib import BCUR_BF16, BCUR_F32, BCUR_F64, BCUR_TF32, PREC, BcurError  # noqa: F401

__all__ = ["Plan", "Batch", "alg1", "boosted", "boosted_batch", "block_scores", "block_stable_rank", "incoherence", "sample_blocks", "residual", "gemm", "gemm_split", "gemm_fp8_blocks",
           "decompose", "load", "BcurError", "PREC"]

load = _lib.load


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> c_void_p:
    return c_void_p(0 if t is None else t.data_ptr())


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float64:
        return BCUR_F64
    if t.dtype == torch.float32:
        return BCUR_F32
    if t.dtype == torch.bfloat16:
        return BCUR_BF16
    if t.dtype == getattr(torch, "float8_e4m3fn", None):
        return _lib.BCUR_FP8
    raise TypeError(f"unsupported dtype {t.dtype}")


def _need_cuda(*ts):
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("tensor must be on a CUDA device")
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")


class Plan:
    """A validated Block CUR problem with its device workspace."""

    def __init__(self, m: int, n: int, k: int, p: int, q: int, col_off: Sequence[int],
                 row_off: Sequence[int], g_col: int, g_row: int, dtype: str = "f32",
                 lda: Optional[int] = None, replacement: bool = False,
                 sketch_prec: Optional[str] = None, fit_prec: Optional[str] = None,
                 device=None, workspace=None):
        torch = _torch()
        L = _lib.load()
        self._L = L
        self.dtype = dtype
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        sp = sketch_prec or dtype
        fp = fit_prec or dtype
        self._col_off = np.ascontiguousarray(np.asarray(col_off, dtype=np.int64))
        self._row_off = np.ascontiguousarray(np.asarray(row_off, dtype=np.int64))
        d = _lib.Desc()
        d.m, d.n, d.lda = m, n, lda or n
        d.a_dtype = PREC[dtype]
        d.k, d.p, d.q = k, p, q
        d.G_col = len(self._col_off) - 1
        d.col_off = self._col_off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.G_row = len(self._row_off) - 1
        d.row_off = self._row_off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.g_col, d.g_row = g_col, g_row
        d.replacement = int(bool(replacement))
        d.sketch_prec, d.fit_prec = PREC[sp], PREC[fp]
        self.desc = d
        self.m, self.n, self.k, self.p, self.q = m, n, k, p, q
        self.G_col, self.G_row, self.g_col, self.g_row = d.G_col, d.G_row, g_col, g_row
        h = c_void_p()
        ws = c_size_t()
        _lib.check(L.bcur_plan(byref(d), _stream(), byref(h), byref(ws)), "bcur_plan")
        self._h = h
        self.workspace_bytes = ws.value
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        if workspace is not None:   # caller-owned device memory (e.g. a serving arena)
            if workspace.numel() < ws.value:
                raise ValueError(f"workspace of {workspace.numel()} bytes < {ws.value} needed")
            self._ws = workspace
        else:
            self._ws = torch.empty(max(ws.value, 256), dtype=torch.uint8, device=dev)
        _lib.check(L.bcur_set_workspace(h, _ptr(self._ws), c_size_t(self._ws.numel())),
                   "bcur_set_workspace")
        self.c_max = self._max_sum(self._col_off, g_col, replacement)
        self.r_max = self._max_sum(self._row_off, g_row, replacement)

    @staticmethod
    def _max_sum(off, g, replacement):
        sz = np.sort(np.diff(off))[::-1]
        return int(g * sz[0]) if replacement else int(sz[:g].sum())

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                self._L.bcur_destroy(h)
            except Exception:  # pragma: no cover
                pass
            self._h = None

    # -- stages ------------------------------------------------------------
    def scores(self, A, omega, out=None):
        torch = _torch()
        _need_cuda(A, omega)
        cs = torch.empty(self.G_col, dtype=torch.float64, device=A.device) if out is None else out[0]
        rs = torch.empty(self.G_row, dtype=torch.float64, device=A.device) if out is None else out[1]
        _lib.check(self._L.bcur_scores(self._h, _ptr(A), _ptr(omega), _ptr(cs), _ptr(rs)),
                   "bcur_scores")
        return cs, rs

    def factors(self):
        torch = _torch()
        Vt = torch.empty(self.k, self.n, dtype=self.tdtype, device=self.device)
        Ut = torch.empty(self.k, self.m, dtype=self.tdtype, device=self.device)
        sig = torch.empty(self.k, dtype=torch.float64, device=self.device)
        _lib.check(self._L.bcur_factors(self._h, _ptr(Vt), _ptr(Ut), _ptr(sig)), "bcur_factors")
        return Vt, Ut, sig

    def sample(self, cs, rs, u_col, u_row, out=None):
        torch = _torch()
        _need_cuda(cs, rs, u_col, u_row)
        dev = cs.device
        if out is not None:
            ci, ri, cp, rp = out
        else:
            ci = torch.empty(self.g_col, dtype=torch.int32, device=dev)
            ri = torch.empty(self.g_row, dtype=torch.int32, device=dev)
            cp = torch.empty(self.g_col, dtype=torch.float64, device=dev)
            rp = torch.empty(self.g_row, dtype=torch.float64, device=dev)
        _lib.check(self._L.bcur_sample(self._h, _ptr(cs), _ptr(rs), _ptr(u_col), _ptr(u_row),
                                       _ptr(ci), _ptr(ri), _ptr(cp), _ptr(rp)), "bcur_sample")
        return ci, ri, cp, rp

    def fit(self, A, ci, ri, want_c: bool = False, want_r: bool = False, U=None):
        torch = _torch()
        _need_cuda(A, ci, ri)
        if U is None:
            U = torch.empty(self.c_max, self.r_max, dtype=self.tdtype, device=A.device)
        C = torch.empty(self.c_max, self.m, dtype=self.tdtype, device=A.device) if want_c else None
        R = torch.empty(self.r_max, self.n, dtype=self.tdtype, device=A.device) if want_r else None
        _lib.check(self._L.bcur_fit(self._h, _ptr(A), _ptr(ci), _ptr(ri), _ptr(U), _ptr(C),
                                    _ptr(R)), "bcur_fit")
        if want_c or want_r:
            return U, C, R
        return U

    def fit_terms(self):
        """(terms, estimate): the BF16 terms the last fit took for its core
        products (1 or 3 for fit_prec "bf16x3a", decided on the device; 3 for
        "bf16x3"; 0 on CUDA cores) and the relative-error estimate the
        adaptive choice was made from (-1 when none was taken)."""
        t = ctypes.c_int32(0)
        e = ctypes.c_double(-1.0)
        _lib.check(self._L.bcur_fit_terms(self._h, ctypes.byref(t), ctypes.byref(e)),
                   "bcur_fit_terms")
        return int(t.value), float(e.value)

    def error(self, A, out=None):
        torch = _torch()
        _need_cuda(A)
        out = torch.empty(3, dtype=torch.float64, device=A.device) if out is None else out
        _lib.check(self._L.bcur_error(self._h, _ptr(A), _ptr(out)), "bcur_error")
        return out

    def decompose_host(self, A, omega, u_col, u_row, out=None):
        """The whole decomposition from host tensors through one C-ABI call
        (bcur_decompose_host): the inputs are copied to the device on the
        plan's stream, the method runs there and the results are copied back.
        ``A``, ``omega`` (l x n panel), ``u_col``, ``u_row``: contiguous CPU
        tensors (page-locked for full-speed copies).  ``out``: an optional
        dict of preallocated CPU tensors (keys col_scores, row_scores,
        col_idx, row_idx, U, err) to fill; the filled dict is returned.  The
        results are valid once torch's current stream has been synchronised."""
        torch = _torch()
        for t in (A, omega, u_col, u_row):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError("host inputs must be contiguous CPU tensors")
        if out is None:
            pin = A.is_pinned()
            mk = lambda *sh, dtype: torch.empty(*sh, dtype=dtype, pin_memory=pin)  # noqa: E731
            out = {"col_scores": mk(self.G_col, dtype=torch.float64),
                   "row_scores": mk(self.G_row, dtype=torch.float64),
                   "col_idx": mk(self.g_col, dtype=torch.int32),
                   "row_idx": mk(self.g_row, dtype=torch.int32),
                   "U": mk(self.c_max, self.r_max, dtype=self.tdtype),
                   "err": mk(3, dtype=torch.float64)}
        need = self._L.bcur_host_staging_bytes(self._h)
        if getattr(self, "_staging", None) is None or self._staging.numel() < need:
            self._staging = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
        _lib.check(self._L.bcur_decompose_host(
            self._h, _ptr(A), _ptr(omega), _ptr(u_col), _ptr(u_row), _ptr(self._staging),
            c_size_t(self._staging.numel()), _ptr(out.get("col_scores")),
            _ptr(out.get("row_scores")), _ptr(out.get("col_idx")), _ptr(out.get("row_idx")),
            _ptr(out.get("U")), _ptr(out["err"])), "bcur_decompose_host")
        return out

    def rank_k_error(self, A):
        """{||A - A_k||_F, ||A - CUR||_F / ||A - A_k||_F} (device FP64): the
        rank-k comparison of Sec. 4.1, A_k from the last scores' top-k factors
        and ||A - CUR||_F from the last error call."""
        torch = _torch()
        _need_cuda(A)
        out = torch.empty(2, dtype=torch.float64, device=A.device)
        _lib.check(self._L.bcur_rank_k_error(self._h, _ptr(A), _ptr(out)), "bcur_rank_k_error")
        return out

    def truncate(self, A, kt: int, omega, want_u: bool = True):
        """Rank-kt U_k of the last fit (Sec. 4.1) and ||A - C U_k R||_F
        (returns U_k or None, and {err, rel, ||A||})."""
        torch = _torch()
        _need_cuda(A, omega)
        Uk = torch.empty(self.c_max, self.r_max, dtype=self.tdtype, device=A.device) if want_u else None
        out = torch.empty(3, dtype=torch.float64, device=A.device)
        _lib.check(self._L.bcur_truncate(self._h, _ptr(A), kt, _ptr(omega), _ptr(Uk), _ptr(out)),
                   "bcur_truncate")
        return Uk, out

    def rank(self):
        v = [c_int64() for _ in range(4)]
        _lib.check(self._L.bcur_rank(self._h, *[byref(x) for x in v]), "bcur_rank")
        return tuple(x.value for x in v)

    def sync_status(self):
        _lib.check(self._L.bcur_sync_status(self._h), "device status")


# -- plan-free stage kernels -------------------------------------------------


class Batch:
    """Many decompositions of different sizes in one pass of the method.

    ``items``: sequence of dicts with keys m, n, k, p, block, g_col, g_row (and
    optionally lda).  Every stage runs as one launch over the whole batch
    (BF16 sketch, split-BF16 fit, FP32 storage; ``fit_prec="bf16x3a"`` for
    the adaptive fit, whose core products start with one BF16 term per item).
    The plan and its workspace are built once; :meth:`run` takes per-item
    device tensors.
    """

    def __init__(self, items, q: int = 2, device=None, workspace=None, fit_prec: str = "bf16x3"):
        torch = _torch()
        L = _lib.load()
        self._L = L
        self.items = [dict(it) for it in items]
        B = len(self.items)
        arr = (_lib.BatchItem * B)()
        for i, it in enumerate(self.items):
            a = arr[i]
            a.m, a.n = it["m"], it["n"]
            a.lda = it.get("lda", it["n"])
            a.k, a.p, a.block = it["k"], it["p"], it["block"]
            a.g_col, a.g_row = it["g_col"], it["g_row"]
        self._arr = arr
        self.B, self.q = B, q
        h = c_void_p()
        ws = c_size_t()
        _lib.check(L.bcur_batch_plan(arr, B, q, _stream(), byref(h), byref(ws)), "bcur_batch_plan")
        self._h = h
        self.workspace_bytes = ws.value
        self.fit_prec = fit_prec
        _lib.check(L.bcur_batch_set_fit(h, PREC[fit_prec]), "bcur_batch_set_fit")
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        if workspace is not None:
            if workspace.numel() < ws.value:
                raise ValueError(f"workspace of {workspace.numel()} bytes < {ws.value} needed")
            self._ws = workspace
        else:
            self._ws = torch.empty(max(ws.value, 256), dtype=torch.uint8, device=dev)
        _lib.check(L.bcur_batch_set_workspace(h, _ptr(self._ws), c_size_t(self._ws.numel())),
                   "bcur_batch_set_workspace")
        self.G_col = [-(-it["n"] // it["block"]) for it in self.items]
        self.G_row = [-(-it["m"] // it["block"]) for it in self.items]
        self.c_max = [it["g_col"] * it["block"] for it in self.items]
        self.r_max = [it["g_row"] * it["block"] for it in self.items]
        self._out = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                self._L.bcur_batch_destroy(h)
            except Exception:  # pragma: no cover
                pass
            self._h = None

    def _outputs(self, want_u: bool):
        """One flat buffer per output kind; per-item views into it."""
        torch = _torch()
        if self._out is not None and self._out["want_u"] == want_u:
            return self._out
        dev = self.device

        flats = {}

        def views(sizes, dtype, kind):
            flat = torch.zeros(max(1, sum(sizes)), dtype=dtype, device=dev)
            flats[kind] = (flat, list(sizes))
            out, at = [], 0
            for s in sizes:
                out.append(flat[at:at + s])
                at += s
            return out

        its = self.items
        o = dict(want_u=want_u,
                 col_scores=views(self.G_col, torch.float64, "col_scores"),
                 row_scores=views(self.G_row, torch.float64, "row_scores"),
                 col_idx=views([it["g_col"] for it in its], torch.int32, "col_idx"),
                 row_idx=views([it["g_row"] for it in its], torch.int32, "row_idx"),
                 err=views([3] * self.B, torch.float64, "err"))
        if want_u:
            us = views([c * r for c, r in zip(self.c_max, self.r_max)], torch.float32, "U")
            o["U"] = [u.view(c, r) for u, c, r in zip(us, self.c_max, self.r_max)]
        else:
            o["U"] = [None] * self.B
        # the flat buffer behind each kind of output and the per-item sizes
        o["flat"] = flats
        self._out = o
        return o

    def run(self, As, omegas, u_cols, u_rows, want_u: bool = True, use_graph: bool = False):
        """Scores, sampling, fit and error for every item (asynchronous on the
        plan's stream).  ``omegas[i]`` is the test matrix as an l x n panel.
        Returns dict of per-item device tensors (reused by the next run)."""
        B = self.B
        if not (len(As) == len(omegas) == len(u_cols) == len(u_rows) == B):
            raise ValueError("one A, omega, u_col, u_row per item")
        _need_cuda(*As, *omegas, *u_cols, *u_rows)
        o = self._outputs(want_u)
        io = (_lib.BatchIO * B)()
        for i in range(B):
            e = io[i]
            e.A, e.omega = As[i].data_ptr(), omegas[i].data_ptr()
            e.u_col, e.u_row = u_cols[i].data_ptr(), u_rows[i].data_ptr()
            e.col_scores, e.row_scores = o["col_scores"][i].data_ptr(), o["row_scores"][i].data_ptr()
            e.col_idx, e.row_idx = o["col_idx"][i].data_ptr(), o["row_idx"][i].data_ptr()
            e.U = o["U"][i].data_ptr() if want_u else None
            e.err = o["err"][i].data_ptr()
        self._keep = (As, omegas, u_cols, u_rows)
        _lib.check(self._L.bcur_batch_run(self._h, io, int(bool(use_graph))), "bcur_batch_run")
        return o

    @property
    def launches_per_run(self) -> int:
        c, r, nl = c_int64(), c_int64(), c_int64()
        _lib.check(self._L.bcur_batch_dims(self._h, 0, byref(c), byref(r), byref(nl)),
                   "bcur_batch_dims")
        return nl.value

    def fit_terms(self):
        """The BF16 terms each item's core products took in the last run (1 or
        3; 3 for every item of a "bf16x3" batch)."""
        out = (ctypes.c_int32 * self.B)()
        _lib.check(self._L.bcur_batch_fit_terms(self._h, ctypes.cast(out, c_void_p)),
                   "bcur_batch_fit_terms")
        return [int(v) for v in out]

    def sync_status(self):
        _lib.check(self._L.bcur_batch_sync_status(self._h), "bcur_batch_sync_status")

    def set_stream(self, stream):
        """Run on `stream` (a torch.cuda.Stream) from now on."""
        _lib.check(self._L.bcur_batch_set_stream(self._h, c_void_p(stream.cuda_stream)),
                   "bcur_batch_set_stream")

    def profile(self, enable: bool = True):
        """Record an event after every launch of the following eager runs."""
        _lib.check(self._L.bcur_batch_profile(self._h, int(bool(enable))), "bcur_batch_profile")

    def profile_steps(self):
        """[(label, ms)] of the last profiled run (after it has completed)."""
        out = []
        for i in range(self._L.bcur_batch_profile_count(self._h)):
            lab = ctypes.c_char_p()
            ms = ctypes.c_double()
            _lib.check(self._L.bcur_batch_profile_entry(self._h, i, byref(lab), byref(ms)),
                       "bcur_batch_profile_entry")
            out.append((lab.value.decode(), ms.value))
        return out

def block_scores(Ft, off, out=None):
    """Def. 2 scores of the factor whose panel (k x h) is ``Ft``; ``off`` device int64."""
    torch = _torch()
    _need_cuda(Ft, off)
    G = off.numel() - 1
    out = torch.empty(G, dtype=torch.float64, device=Ft.device) if out is None else out
    k, h = Ft.shape
    _lib.check(_lib.load().bcur_block_scores(_ptr(Ft), _dtype_code(Ft), k, h, h, _ptr(off), G,
                                             _ptr(out), _stream()), "bcur_block_scores")
    return out


def block_stable_rank(Ft, off):
    """Per-block ||F_g||_F^2 / ||F_g||_2^2 of the factor whose panel is ``Ft``;
    alpha of Sec. 3.2 is the minimum over blocks."""
    torch = _torch()
    _need_cuda(Ft, off)
    L = _lib.load()
    G = off.numel() - 1
    k, h = Ft.shape
    ws = torch.empty(max(L.bcur_block_stable_rank_workspace(k, G), 256), dtype=torch.uint8,
                     device=Ft.device)
    out = torch.empty(G, dtype=torch.float64, device=Ft.device)
    _lib.check(L.bcur_block_stable_rank(_ptr(Ft), _dtype_code(Ft), k, h, h, _ptr(off), G, _ptr(out),
                                        _ptr(ws), c_size_t(ws.numel()), _stream()),
               "bcur_block_stable_rank")
    return out


def incoherence(Ut):
    """mu = (m/k) max_i ||U_k^T e_i||^2 (Sec. 3.2) from the panel U_k^T (k x m):
    a device FP64 tensor of one element (bcur_incoherence)."""
    torch = _torch()
    _need_cuda(Ut)
    k, m = Ut.shape
    out = torch.empty(1, dtype=torch.float64, device=Ut.device)
    scratch = torch.empty(1, dtype=torch.int64, device=Ut.device)
    _lib.check(_lib.load().bcur_incoherence(_ptr(Ut), _dtype_code(Ut), k, m, m, _ptr(out),
                                            _ptr(scratch), _stream()), "bcur_incoherence")
    return out[0]


def sample_blocks(scores, u, g: int, replacement: bool = False):
    torch = _torch()
    _need_cuda(scores, u)
    idx = torch.empty(g, dtype=torch.int32, device=scores.device)
    prob = torch.empty(g, dtype=torch.float64, device=scores.device)
    _lib.check(_lib.load().bcur_sample_blocks(_ptr(scores), scores.numel(), _ptr(u), g,
                                              int(bool(replacement)), _ptr(idx), _ptr(prob),
                                              _stream()), "bcur_sample_blocks")
    return idx, prob


def residual(X, P, Q, prec: str = None):
    """{||X - P Q||_F^2, ||X||_F^2} (device FP64) from the fused residual kernel."""
    torch = _torch()
    _need_cuda(X, P, Q)
    L = _lib.load()
    m, n = X.shape[0], Q.shape[1]
    r = P.shape[0] and P.shape[1]
    code = BCUR_BF16 if P.dtype == torch.bfloat16 else _dtype_code(X)
    prec = PREC[prec] if prec else code
    wsb = L.bcur_residual_workspace(m, n, code)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=X.device)
    out = torch.empty(2, dtype=torch.float64, device=X.device)
    _lib.check(L.bcur_residual(_ptr(X), X.shape[1], _ptr(P), P.shape[1], _ptr(Q), Q.shape[1], m,
                               n, P.shape[1] if code != BCUR_BF16 else r, code, prec, _ptr(out),
                               _ptr(ws), c_size_t(ws.numel()), _stream()), "bcur_residual")
    return out


def gemm(A, B, transA: bool = False, transB: bool = False, prec: str = None, out=None):
    """D = op(A) op(B) on the library's kernels (row-major tensors)."""
    torch = _torch()
    _need_cuda(A, B)
    M = A.shape[1] if transA else A.shape[0]
    K = A.shape[0] if transA else A.shape[1]
    N = B.shape[0] if transB else B.shape[1]
    code = _dtype_code(A)
    prec = PREC[prec] if prec else code
    ddt = A.dtype if code in (BCUR_F64, BCUR_F32) else torch.float32
    D = torch.empty(M, N, dtype=ddt, device=A.device) if out is None else out
    _lib.check(_lib.load().bcur_gemm(M, N, K, _ptr(A), A.shape[1], int(transA), _ptr(B),
                                     B.shape[1], int(transB), _ptr(D), D.shape[1], code, prec,
                                     _stream()), "bcur_gemm")
    return D


def gemm_fp8_blocks(A8, B8, bscale, scale_m=None, out=None):
    """D = diag(scale_m) sum over 128-deep K blocks kb of bscale[j/128, kb] A8[:, kb] B8[:, kb]^T
    (e4m3 A8: M x K, B8: N x K, both K-major; bscale: ceil(N/128) x ceil(K/128) FP32)."""
    torch = _torch()
    for t in (A8, B8, bscale):   # row views with padded leading dimensions are fine
        if not t.is_cuda or t.stride(-1) != 1:
            raise ValueError("operands must be CUDA tensors with unit inner stride")
    M, K = A8.shape
    N = B8.shape[0]
    D = torch.empty(M, N, dtype=torch.float32, device=A8.device) if out is None else out
    _lib.check(_lib.load().bcur_gemm_fp8_blocks(M, N, K, _ptr(A8), A8.stride(0), _ptr(B8),
                                                B8.stride(0), _ptr(scale_m), _ptr(bscale),
                                                bscale.stride(0), bscale.stride(1), _ptr(D),
                                                D.stride(0), _stream()), "bcur_gemm_fp8_blocks")
    return D


def gemm_split(A_hi, A_lo, B_hi, B_lo, transA: bool = False, transB: bool = False, out=None):
    """D = A B from BF16 hi/lo pairs (3-term split product, FP32 result)."""
    torch = _torch()
    _need_cuda(A_hi, A_lo, B_hi, B_lo)
    M = A_hi.shape[1] if transA else A_hi.shape[0]
    K = A_hi.shape[0] if transA else A_hi.shape[1]
    N = B_hi.shape[0] if transB else B_hi.shape[1]
    D = torch.empty(M, N, dtype=torch.float32, device=A_hi.device) if out is None else out
    _lib.check(_lib.load().bcur_gemm_split(M, N, K, _ptr(A_hi), _ptr(A_lo), A_hi.shape[1],
                                           int(transA), _ptr(B_hi), _ptr(B_lo), B_hi.shape[1],
                                           int(transB), _ptr(D), D.shape[1], _stream()),
               "bcur_gemm_split")
    return D


def alg1(A, col_off, r: int, g: int, u_rows, u_cols, want_u: bool = True):
    """The paper's Algorithm 1 as printed (uniform rows, scores of R's row space,
    blocks with replacement and the scaling of Sec. 3.1, U = W^+)."""
    torch = _torch()
    _need_cuda(A, u_rows, u_cols)
    L = _lib.load()
    m, n = A.shape
    off = np.ascontiguousarray(np.asarray(col_off, dtype=np.int64))
    G = len(off) - 1
    code = _dtype_code(A)
    offp = off.ctypes.data_as(ctypes.c_void_p)
    wsb = L.bcur_alg1_workspace(m, n, offp, G, r, g, code)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=A.device)
    dev = A.device
    ri = torch.empty(r, dtype=torch.int32, device=dev)
    ci = torch.empty(g, dtype=torch.int32, device=dev)
    cs = torch.empty(G, dtype=torch.float64, device=dev)
    cp = torch.empty(g, dtype=torch.float64, device=dev)
    c_max = int(g * np.max(np.diff(off)))
    U = torch.empty(c_max, r, dtype=A.dtype, device=dev) if want_u else None
    err = torch.empty(3, dtype=torch.float64, device=dev)
    _lib.check(L.bcur_alg1(_ptr(A), n, m, n, code, offp, G, r, g, _ptr(u_rows), _ptr(u_cols),
                           _ptr(ri), _ptr(ci), _ptr(cs), _ptr(cp), _ptr(U), _ptr(err), _ptr(ws),
                           c_size_t(ws.numel()), _stream()), "bcur_alg1")
    return dict(row_idx=ri, col_idx=ci, col_scores=cs, col_prob=cp, U=U, err=err)


def _boost_pick(t, err_all, U_all, ci_all, ri_all):
    """Device-side choice of the run with the smallest ||A - CUR||_F
    (bcur_boost_select) among t runs stored contiguously."""
    torch = _torch()
    dev = err_all.device
    best = torch.empty(1, dtype=torch.int32, device=dev)
    err = torch.empty(3, dtype=torch.float64, device=dev)
    ci = torch.empty(ci_all.shape[1], dtype=torch.int32, device=dev)
    ri = torch.empty(ri_all.shape[1], dtype=torch.int32, device=dev)
    U = torch.empty(U_all.shape[1:], dtype=U_all.dtype, device=dev) if U_all is not None else None
    ub = 0 if U_all is None else U_all[0].numel() * U_all.element_size()
    _lib.check(_lib.load().bcur_boost_select(
        t, _ptr(err_all), err_all.shape[1], _ptr(U_all), ub, _ptr(ci_all), ci_all.shape[1],
        _ptr(ri_all), ri_all.shape[1], _ptr(U), _ptr(ci), _ptr(ri), _ptr(err), _ptr(best),
        _stream()), "bcur_boost_select")
    return dict(col_idx=ci, row_idx=ri, U=U, err=err), best


def boosted(plan: Plan, A, omegas, u_cols, u_rows):
    """Boosting (Sec. 3.3): the decomposition is repeated once per (omega,
    u_col, u_row) triple and the run with the smallest ||A - CUR||_F is kept.
    The runs write into contiguous device buffers and the library picks the
    best one on the device, so nothing waits for the host.  Returns the
    chosen run's outputs (device tensors col_idx, row_idx, U, err) and its
    index (device int32 tensor of one element)."""
    torch = _torch()
    t = len(omegas)
    dev = A.device
    err_all = torch.empty(t, 3, dtype=torch.float64, device=dev)
    U_all = torch.empty(t, plan.c_max, plan.r_max, dtype=plan.tdtype, device=dev)
    ci_all = torch.empty(t, plan.g_col, dtype=torch.int32, device=dev)
    ri_all = torch.empty(t, plan.g_row, dtype=torch.int32, device=dev)
    for i, (om, uc, ur) in enumerate(zip(omegas, u_cols, u_rows)):
        cs, rs = plan.scores(A, om)
        _lib.check(plan._L.bcur_sample(plan._h, _ptr(cs), _ptr(rs), _ptr(uc), _ptr(ur),
                                       _ptr(ci_all[i]), _ptr(ri_all[i]), c_void_p(0), c_void_p(0)),
                   "bcur_sample")
        plan.fit(A, ci_all[i], ri_all[i], U=U_all[i])
        plan.error(A, out=err_all[i])
    return _boost_pick(t, err_all, U_all, ci_all, ri_all)


def boosted_batch(item: dict, A, omegas, u_cols, u_rows, q: int = 2, use_graph: bool = False):
    """Boosting (Sec. 3.3) in one batched pass: the t independent runs on the
    same resident A (FP32) are the t members of one Batch (every stage one
    launch over all runs, BF16 sketch and split-BF16 fit), and the run with
    the smallest ||A - CUR||_F is picked on the device.  ``item`` holds the
    Batch keys m, n, k, p, block, g_col, g_row.  Returns the chosen run's
    outputs (device tensors col_idx, row_idx, U, err), its index (device
    int32 tensor) and the Batch (reusable for further draws)."""
    t = len(omegas)
    b = Batch([item] * t, q=q)
    out = b.run([A] * t, omegas, u_cols, u_rows, want_u=True, use_graph=use_graph)
    # identical items: the batch's flat output buffers are t runs side by side
    fl = out["flat"]
    c, r = b.c_max[0], b.r_max[0]
    best, idx = _boost_pick(t, fl["err"][0][:3 * t].view(t, 3), fl["U"][0][:t * c * r].view(t, c, r),
                            fl["col_idx"][0][:t * item["g_col"]].view(t, item["g_col"]),
                            fl["row_idx"][0][:t * item["g_row"]].view(t, item["g_row"]))
    return best, idx, b
def decompose(plan: Plan, A, omega, u_col, u_row, col_idx=None, row_idx=None):
    """All stages on one matrix; returns a dict of device tensors."""
    cs, rs = plan.scores(A, omega)
    ci, ri, cp, rp = plan.sample(cs, rs, u_col, u_row)
    if col_idx is not None:
        ci = col_idx
    if row_idx is not None:
        ri = row_idx
    U = plan.fit(A, ci, ri)
    e = plan.error(A)
    return dict(col_scores=cs, row_scores=rs, col_idx=ci, row_idx=ri, col_prob=cp, row_prob=rp,
                U=U, err=e)
