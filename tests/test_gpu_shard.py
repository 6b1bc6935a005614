"""The row-sharded form's local arithmetic on the library's kernels (one rank:
the exchange steps are the identity; the two-rank schedule is tested on CPU
ranks in test_shard_gloo.py)."""
import numpy as np
import pytest

from _gpu_common import device, to_dev, torch  # noqa: F401
import bcur_inputs as bi
import oracle as orc

pytestmark = pytest.mark.gpu


def test_one_rank_on_the_library_matches_the_oracle():
    from paper_1703_06065_gb300.shard import LibraryOps, RowSharded

    device()
    p = bi.plain_fp64_512x1024()
    A = p.matrix()
    rs = RowSharded(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row,
                    rows=(0, p.m), ops=LibraryOps("f64"))
    res = rs.run(to_dev(A), to_dev(np.ascontiguousarray(p.omega().T)), to_dev(p.u_col()),
                 to_dev(p.u_row()))
    ref = orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row, p.omega(),
                        p.u_col(), p.u_row())
    np.testing.assert_allclose(res["col_scores"].cpu().numpy(), ref["col_scores"], rtol=0,
                               atol=1e-10)
    np.testing.assert_allclose(res["row_scores"].cpu().numpy(), ref["row_scores"], rtol=0,
                               atol=1e-10)
    assert res["col_idx"].cpu().tolist() == list(ref["col_idx"])
    assert res["row_idx"].cpu().tolist() == list(ref["row_idx"])
    U = res["U"].cpu().numpy()
    assert np.linalg.norm(U - ref["U"]) <= 1e-7 * np.linalg.norm(ref["U"])
    e = res["err"].cpu().numpy()
    assert abs(e[0] - ref["err"]) <= 1e-9 * ref["err"]


def test_cholesky_inverse_entry_point():
    """bcur_cholesky_inverse on an SPD matrix (w = 200 padded to 256 with
    zeros, which are dropped): L L^T = G and L L^{-1} = I to FP64 round-off."""
    from paper_1703_06065_gb300.shard import LibraryOps

    device()
    rg = np.random.default_rng(3)
    X = rg.standard_normal((300, 200))
    G = X.T @ X
    ops = LibraryOps("f64")
    L, Li = ops.chol_inv(to_dev(G))
    L, Li = L.cpu().numpy(), Li.cpu().numpy()
    assert np.allclose(np.triu(L, 1), 0) and np.allclose(np.triu(Li, 1), 0)
    assert np.linalg.norm(L @ L.T - G) <= 1e-13 * np.linalg.norm(G)
    assert np.linalg.norm(L @ Li - np.eye(200)) <= 1e-11
