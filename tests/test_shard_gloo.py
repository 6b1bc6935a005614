"""The row-sharded form's exchange schedule on CPU ranks (gloo, world size 2).

Each rank holds half of A's row blocks; the local arithmetic is supplied by a
plain FP64 stand-in written here (the product form runs it in the library's
kernels on each rank's GPU), so what is under test is the schedule: which
sums are all-reduced, which row blocks are broadcast from their owners, and
that the result equals the one-rank FP64 oracle's.  A is never sent: the
largest message is the n x l product A^T Q."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bcur_inputs as bi  # noqa: E402
import oracle as orc  # noqa: E402


class NumpyOps:
    """FP64 CPU stand-in for the library's local arithmetic (torch tensors)."""

    def empty(self, *shape, dtype=torch.float64):
        return torch.empty(*shape, dtype=dtype)

    def zeros(self, *shape, dtype=torch.float64):
        return torch.zeros(*shape, dtype=dtype)

    def mm(self, A, B, tA=False, tB=False):
        return (A.T if tA else A) @ (B.T if tB else B)

    def chol_inv(self, G):
        L = torch.linalg.cholesky(G)
        return L, torch.linalg.inv(L)

    def svd_small(self, X):
        U, s, Vh = torch.linalg.svd(X)
        return U, s, Vh.T

    def block_scores(self, F, off):
        return torch.from_numpy(orc.block_scores(F.numpy(), off))

    def sample(self, scores, u, g, replacement=False):
        idx, _ = orc.sample_blocks(scores.numpy(), u.numpy(), g, replacement)
        return torch.tensor(idx, dtype=torch.int32)

    def gather_cols_t(self, A, off, idx, c):
        cols = orc.block_cols(off, idx.tolist())
        return A[:, torch.from_numpy(cols)].T.contiguous()

    def gather_rows_into(self, A, off, idx, out):
        rows = orc.block_cols(off, idx.tolist())
        out.copy_(A[torch.from_numpy(rows)])
        return out

    def residual(self, X, P, Q):
        D = X - P @ Q
        return torch.stack([(D * D).sum(), (X * X).sum()])


def _problem():
    p = bi.plain_fp64_512x1024()
    return p, p.matrix()


def _worker(rank, world, port, out_dir, split):
    import torch.distributed as dist

    from paper_1703_06065_gb300.shard import RowSharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, A = _problem()
        r0, r1 = split[rank], split[rank + 1]
        rs = RowSharded(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row,
                        rows=(r0, r1), ops=NumpyOps())
        res = rs.run(torch.from_numpy(A[r0:r1].copy()),
                     torch.from_numpy(np.ascontiguousarray(p.omega().T)),
                     torch.from_numpy(p.u_col()), torch.from_numpy(p.u_row()))
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"),
                 **{k: v.numpy() for k, v in res.items()},
                 log_names=np.array([a for a, _ in rs.log]),
                 log_sizes=np.array([b for _, b in rs.log]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("split", [(0, 256, 512), (0, 96, 512)])
def test_two_cpu_ranks_reproduce_the_oracle(tmp_path, split):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path), list(split)), nprocs=2,
                       join=True, start_method="spawn")
    p, A = _problem()
    ref = orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row, p.omega(),
                        p.u_col(), p.u_row())
    outs = [np.load(tmp_path / f"rank{r}.npz") for r in range(2)]
    for o in outs:
        np.testing.assert_allclose(o["col_scores"], ref["col_scores"], rtol=0, atol=1e-10)
        np.testing.assert_allclose(o["row_scores"], ref["row_scores"], rtol=0, atol=1e-10)
        assert o["col_idx"].tolist() == list(ref["col_idx"])
        assert o["row_idx"].tolist() == list(ref["row_idx"])
        assert np.linalg.norm(o["U"] - ref["U"]) <= 1e-7 * np.linalg.norm(ref["U"])
        assert abs(o["err"][0] - ref["err"]) <= 1e-9 * ref["err"]
        assert abs(o["err"][1] - ref["rel"]) <= 1e-9
    # both ranks hold the same replicated results
    for key in ("col_idx", "row_idx", "U", "err"):
        np.testing.assert_array_equal(outs[0][key], outs[1][key])
    # the schedule: only these exchanges, never a piece of A
    names = [str(x) for x in outs[0]["log_names"]]
    sizes = outs[0]["log_sizes"]
    l, c, r = p.l, p.g_col * 32, p.g_row * 32
    assert names.count("all_reduce:gram_l") == 2 * (1 + p.q)
    assert names.count("all_reduce:AtQ") == p.q + 1
    assert names.count("all_reduce:gram_c") == 2
    assert names.count("all_reduce:M") == 1 and names.count("all_reduce:residual") == 1
    assert sum(n.startswith("broadcast:R_block") for n in names) == p.g_row
    assert max(sizes) <= max(p.n * l, c * c, c * r, 32 * p.n)
    assert max(sizes) < (split[2] - split[1]) * p.n
