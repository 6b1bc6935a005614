"""Row-sharded Block CUR: one matrix whose row blocks are spread over the ranks
of a ``torch.distributed`` group.

The paper motivates block sampling with matrices stored as blocks across the
machines of a cluster (Sec. 1; the Spark experiments of Sec. 4.2 keep row
blocks as partitions).  Here every rank holds whole row blocks of A (a
contiguous row range that starts and ends on row-block boundaries) and the
method runs on the ranks with these exchange steps and no others:

* sketch and subspace iteration: Y_r = A_r Omega is local; the Cholesky-QR2
  of Y needs the l x l Gram sum_r Y_r^T Y_r (one all-reduce per pass); the
  product Z = A^T Q = sum_r A_r^T Q_r is one all-reduce of n x l, after which
  Z and its Cholesky-QR2 are replicated;
* projection: B^T = A^T Q, one all-reduce of n x l; the small SVD, V_k and
  the column-block scores are replicated, U_k is local (rows of A_r);
* row-block scores: each rank scores its own blocks; one all-reduce of the
  G_row scores (every block has exactly one owner, the others add zero);
* sampling: replicated (same scores, same uniforms, same indices everywhere);
* C = A[:, J]: local rows C_r; its Cholesky-QR2 needs the c x c Gram
  sum_r C_r^T C_r (one all-reduce per pass);
* R = A[I, :]: each chosen row block is broadcast from the rank that owns it;
  R's Cholesky-QR2 is replicated;
* M = Q_C^T A Q_R = sum_r Q_{C,r}^T A_r Q_R: one all-reduce of c x r; U is
  replicated;
* ||A - CUR||_F^2 and ||A||_F^2: one all-reduce of two scalars.

The arithmetic is supplied by ``ops``: :class:`LibraryOps` runs every step in
this library's CUDA kernels through the C ABI (bcur_gemm, bcur_cholesky_inverse,
bcur_svd_small, bcur_block_scores, bcur_sample_blocks, bcur_gather_blocks,
bcur_residual).  The exchange schedule above is the same for any ``ops``.
Only one GPU is available to this build, so the multi-rank form is exercised
with CPU ranks (gloo) in the tests.
"""
from __future__ import annotations

from ctypes import c_double, c_size_t, c_void_p
from typing import Optional, Sequence

import numpy as np

from . import _lib


def _torch():
    import torch
    return torch


class LibraryOps:
    """The local arithmetic of the row-sharded form on this library's kernels
    (device tensors, FP64 or FP32, CUDA cores).  Matrices are row-major torch
    tensors; ``mm(A, B, tA, tB)`` is op(A) op(B)."""

    def __init__(self, dtype: str = "f64", device=None):
        torch = _torch()
        self.L = _lib.load()
        self.code = _lib.PREC[dtype]
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        self.device = device if device is not None else torch.device("cuda",
                                                                     torch.cuda.current_device())
        self._scratch = torch.empty(4096, dtype=torch.uint8, device=self.device)

    def _s(self):
        return c_void_p(_torch().cuda.current_stream().cuda_stream)

    @staticmethod
    def _p(t):
        return c_void_p(0 if t is None else t.data_ptr())

    def empty(self, *shape, dtype=None):
        return _torch().empty(*shape, dtype=dtype or self.tdtype, device=self.device)

    def zeros(self, *shape, dtype=None):
        return _torch().zeros(*shape, dtype=dtype or self.tdtype, device=self.device)

    def mm(self, A, B, tA: bool = False, tB: bool = False):
        M = A.shape[1] if tA else A.shape[0]
        K = A.shape[0] if tA else A.shape[1]
        N = B.shape[0] if tB else B.shape[1]
        D = self.empty(M, N)
        _lib.check(self.L.bcur_gemm(M, N, K, self._p(A), A.shape[1], int(tA), self._p(B),
                                    B.shape[1], int(tB), self._p(D), N, self.code, self.code,
                                    self._s()), "bcur_gemm")
        return D

    def chol_inv(self, G):
        """Lower L with G = L L^T (drop rule) and L^{-1}; w padded to 64."""
        w = G.shape[0]
        wp = -(-w // 64) * 64
        Gp = self.zeros(wp, wp)
        Gp[:w, :w] = G
        L, Li = self.empty(wp, wp), self.empty(wp, wp)
        kept = self.zeros(1, dtype=_torch().int32)
        _lib.check(self.L.bcur_cholesky_inverse(self._p(Gp), wp, self.code, self._p(L),
                                                self._p(Li), self._p(kept), c_double(0.0),
                                                self._p(self._scratch),
                                                c_size_t(self._scratch.numel()), self._s()),
                   "bcur_cholesky_inverse")
        return L[:w, :w].contiguous(), Li[:w, :w].contiguous()

    def svd_small(self, X):
        """X = Ut diag(sigma) W^T (columns of Ut and W are the singular vectors)."""
        torch = _torch()
        w = X.shape[0]
        X64 = X.to(torch.float64).contiguous()
        Ut, W = self.empty(w, w), self.empty(w, w)
        sig = self.empty(w, dtype=torch.float64)
        work = self.empty((w + 1) * (w + 1))
        _lib.check(self.L.bcur_svd_small(self._p(X64), w, self.code, self._p(Ut), self._p(W),
                                         self._p(sig), self._p(work),
                                         c_size_t(work.numel() * work.element_size()), None,
                                         self._s()), "bcur_svd_small")
        return Ut, sig, W

    def block_scores(self, F, off):
        """Def. 2 for the factor F (h x k): F is passed as its panel F^T."""
        torch = _torch()
        Ft = F.t().contiguous()
        offd = torch.as_tensor(np.asarray(off, dtype=np.int64), device=self.device)
        out = self.empty(len(off) - 1, dtype=torch.float64)
        _lib.check(self.L.bcur_block_scores(self._p(Ft), self.code, Ft.shape[0], Ft.shape[1],
                                            Ft.shape[1], self._p(offd), len(off) - 1,
                                            self._p(out), self._s()), "bcur_block_scores")
        return out

    def sample(self, scores, u, g: int, replacement: bool = False):
        torch = _torch()
        idx = self.empty(g, dtype=torch.int32)
        prob = self.empty(g, dtype=torch.float64)
        _lib.check(self.L.bcur_sample_blocks(self._p(scores), scores.numel(), self._p(u), g,
                                             int(replacement), self._p(idx), self._p(prob),
                                             self._s()), "bcur_sample_blocks")
        return idx

    def _gather(self, A, off, idx, axis, cap, out, ldo):
        torch = _torch()
        offd = torch.as_tensor(np.asarray(off, dtype=np.int64), device=self.device)
        mp = self.empty(cap + 1, dtype=torch.int64)
        m, n = A.shape
        _lib.check(self.L.bcur_gather_blocks(self._p(A), n, m, n, self.code, axis, self._p(offd),
                                             len(off) - 1, self._p(idx), idx.numel(), cap,
                                             self._p(out), ldo, self._p(mp), self._s()),
                   "bcur_gather_blocks")
        return out

    def gather_cols_t(self, A, off, idx, c: int):
        """C^T (c x m) for the column blocks idx of A (m x n)."""
        out = self.empty(c, A.shape[0])
        return self._gather(A, off, idx, 1, c, out, A.shape[0])

    def gather_rows_into(self, A, off, idx, out):
        """The row blocks idx of A into ``out`` (rows x n, contiguous)."""
        return self._gather(A, off, idx, 0, out.shape[0], out, out.shape[1])

    def residual(self, X, P, Q):
        """{sum (X - P Q)^2, sum X^2} (FP64, 2 elements)."""
        torch = _torch()
        m, n = X.shape
        r = P.shape[1]
        wsb = self.L.bcur_residual_workspace(m, n, self.code)
        ws = self.empty(max(wsb, 256), dtype=torch.uint8)
        out = self.empty(2, dtype=torch.float64)
        _lib.check(self.L.bcur_residual(self._p(X), n, self._p(P), r, self._p(Q), n, m, n, r,
                                        self.code, self.code, self._p(out), self._p(ws),
                                        c_size_t(ws.numel()), self._s()), "bcur_residual")
        return out


class RowSharded:
    """Block CUR of one m x n matrix held as row blocks across the ranks of
    ``group`` (None: the default group, or a single process when
    torch.distributed is not initialised).

    ``rows = (r0, r1)``: this rank's rows of A, on row-block boundaries, the
    ranks' ranges in rank order covering [0, m).  ``ops``: the local
    arithmetic (default :class:`LibraryOps` in FP64).  Method parameters as
    :class:`paper_1703_06065_gb300.Plan` (without replacement)."""

    def __init__(self, m: int, n: int, k: int, p: int, q: int, col_off: Sequence[int],
                 row_off: Sequence[int], g_col: int, g_row: int, rows, ops=None, group=None):
        self.m, self.n, self.k, self.p, self.q = m, n, k, p, q
        self.l = k + p
        self.col_off = np.asarray(col_off, dtype=np.int64)
        self.row_off = np.asarray(row_off, dtype=np.int64)
        self.g_col, self.g_row = g_col, g_row
        self.r0, self.r1 = int(rows[0]), int(rows[1])
        if self.r0 not in self.row_off or self.r1 not in self.row_off:
            raise ValueError("a rank's rows must start and end on row-block boundaries")
        self.ops = ops if ops is not None else LibraryOps("f64")
        self.group = group
        # this rank's row blocks and their offsets relative to r0
        b0 = int(np.searchsorted(self.row_off, self.r0))
        b1 = int(np.searchsorted(self.row_off, self.r1))
        self.blocks = (b0, b1)
        self.local_off = self.row_off[b0:b1 + 1] - self.r0
        self.log = []   # (collective, elements) of the last run, in order

    # -- collectives ---------------------------------------------------------
    def _dist(self):
        torch = _torch()
        d = torch.distributed
        return d if d.is_available() and d.is_initialized() else None

    def _world(self):
        d = self._dist()
        return d.get_world_size(self.group) if d else 1

    def _allreduce(self, t, what: str):
        self.log.append(("all_reduce:" + what, t.numel()))
        d = self._dist()
        if d and self._world() > 1:
            d.all_reduce(t, op=d.ReduceOp.SUM, group=self.group)
        return t

    def _owner(self, block: int):
        """Rank that holds row block `block` (ranks' ranges are exchanged once)."""
        return int(np.searchsorted(self._starts, self.row_off[block], side="right") - 1)

    # -- Cholesky-QR2, summing the Gram across ranks when `shared` -----------
    def _cqr2_panel(self, Xt, shared: bool, what: str):
        """Xt: panel X^T (w x h_local).  Returns Q^T (w x h_local) and the
        factors (L1, L1^{-1}), (L2, L2^{-1}) with X = Q (L1 L2)^T."""
        ops = self.ops
        Ls = []
        for _ in range(2):
            G = ops.mm(Xt, Xt, False, True)
            if shared:
                G = self._allreduce(G, what)
            L, Li = ops.chol_inv(G)
            Xt = ops.mm(Li, Xt)
            Ls.append((L, Li))
        return Xt, Ls[0], Ls[1]

    def run(self, A_local, omega, u_col, u_row):
        """A_local: this rank's rows (r1 - r0) x n; omega: the n x l test
        matrix as an l x n panel (the same on every rank); u_col, u_row: the
        uniforms (the same on every rank).  Returns col_scores, row_scores,
        col_idx, row_idx, U (c x r) and err = {||A - CUR||_F, its ratio to
        ||A||_F, ||A||_F}, all replicated."""
        torch = _torch()
        ops = self.ops
        self.log = []
        d = self._dist()
        world = self._world()
        starts = [self.r0]
        if d and world > 1:
            st = torch.tensor([self.r0], dtype=torch.int64)
            allst = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
            d.all_gather(allst, st, group=self.group)
            starts = [int(x.item()) for x in allst]
            self.log.append(("all_gather:row_ranges", world))
        self._starts = np.asarray(starts, dtype=np.int64)
        k = self.k
        # range finder with q steps of subspace iteration (Sec. 3.1 allows sketching)
        Yt = ops.mm(omega, A_local, False, True)                  # (A_r Omega)^T, l x m_r
        Qt, _, _ = self._cqr2_panel(Yt, True, "gram_l")
        for _ in range(self.q):
            Zt = self._allreduce(ops.mm(Qt, A_local), "AtQ")       # (A^T Q)^T, l x n
            Zt, _, _ = self._cqr2_panel(Zt, False, "")
            Yt = ops.mm(Zt, A_local, False, True)
            Qt, _, _ = self._cqr2_panel(Yt, True, "gram_l")
        Bt = self._allreduce(ops.mm(Qt, A_local), "AtQ")           # B = Q^T A, l x n
        QBt, (L1, _), (L2, _) = self._cqr2_panel(Bt, False, "")    # B = (L1 L2) Q_B^T
        Ut, sig, W = ops.svd_small(ops.mm(L1, L2))
        Vk = ops.mm(QBt, W[:, :k].contiguous(), True, False)       # n x k, replicated
        Uk_loc = ops.mm(Qt, Ut[:, :k].contiguous(), True, False)   # m_r x k, local rows
        cs = ops.block_scores(Vk, self.col_off)                    # Def. 2
        rs = ops.zeros(len(self.row_off) - 1, dtype=torch.float64)
        rs[self.blocks[0]:self.blocks[1]] = ops.block_scores(Uk_loc, self.local_off)
        rs = self._allreduce(rs, "row_scores")
        # sampling (Alg. 1 step 2), identical on every rank
        ci = ops.sample(cs, u_col, self.g_col)
        ri = ops.sample(rs, u_row, self.g_row)
        ci_h = [int(x) for x in ci.cpu().tolist()]
        ri_h = [int(x) for x in ri.cpu().tolist()]
        csz = np.diff(self.col_off)
        rsz = np.diff(self.row_off)
        c = int(sum(csz[j] for j in ci_h))
        r = int(sum(rsz[j] for j in ri_h))
        # C: local rows; R: each chosen row block from its owner
        Ct = ops.gather_cols_t(A_local, self.col_off, ci, c)       # C_r^T, c x m_r
        R = ops.zeros(r, self.n)
        at = 0
        for j in ri_h:
            h = int(rsz[j])
            owner = self._owner(j)
            dst = R[at:at + h]
            if owner == (d.get_rank(self.group) if d and world > 1 else 0):
                lj = torch.tensor([j - self.blocks[0]], dtype=torch.int32, device=R.device)
                ops.gather_rows_into(A_local, self.local_off, lj, dst)
            if d and world > 1:
                self.log.append((f"broadcast:R_block_from_{owner}", dst.numel()))
                d.broadcast(dst, src=d.get_global_rank(self.group, owner)
                            if self.group is not None else owner, group=self.group)
            at += h
        # QR of C (Gram summed across ranks) and of R^T (replicated)
        QCt, (_, L1Ci), (_, L2Ci) = self._cqr2_panel(Ct, True, "gram_c")  # Q_C^T, c x m_r
        QRt, (_, L1Ri), (_, L2Ri) = self._cqr2_panel(R, False, "")         # Q_R^T, r x n
        M = self._allreduce(ops.mm(ops.mm(QCt, A_local), QRt, False, True), "M")  # c x r
        # C = Q_C (L1C L2C)^T and R^T = Q_R (L1R L2R)^T, so
        # U = C^+ A R^+ = L1C^{-T} L2C^{-T} M L2R^{-1} L1R^{-1}
        U = ops.mm(L1Ci, ops.mm(L2Ci, M, True, False), True, False)
        U = ops.mm(ops.mm(U, L2Ri), L1Ri)
        # ||A - CUR||_F: local residuals of the rows of A_r, summed
        P = ops.mm(Ct, U, True, False)                             # C_r U, m_r x r
        e2 = self._allreduce(ops.residual(A_local, P, R), "residual")
        e = torch.sqrt(e2[0])
        a = torch.sqrt(e2[1])
        err = torch.stack([e, e / a, a])
        return dict(col_scores=cs, row_scores=rs, col_idx=ci, row_idx=ri, U=U, err=err)
