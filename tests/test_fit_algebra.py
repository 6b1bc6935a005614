"""The algebra the tensor-core fit relies on, checked in FP64 on the host.

The second Cholesky-QR pass stops at its triangular factor: with
G1 = C^T C = L1 L1^T, Q1 = C L1^{-T}, G2 = Q1^T Q1 = L2 L2^T and Q = Q1 L2^{-T}
(and the same for R^T), the fit forms M1 = Q1_C^T A Q1_R and

    M2 = L2C^{-T} L2C^{-1} M1 L2R^{-T} L2R^{-1},   U = L1C^{-T} M2 L1R^{-1},

and reconstructs CUR as Q1_C M2 Q1_R^T.  These must equal U = C^+ A R^+ (the
least-squares core) and the orthogonal projection P_C A P_R."""
import numpy as np
import pytest


def _chol_qr(X):
    G = X.T @ X
    L = np.linalg.cholesky(G)
    return X @ np.linalg.inv(L).T, L


@pytest.mark.parametrize("seed,m,n,c,r", [(0, 60, 50, 12, 9), (1, 90, 70, 20, 25)])
def test_folded_second_pass_gives_the_least_squares_core(seed, m, n, c, r):
    g = np.random.default_rng(seed)
    A = g.standard_normal((m, n))
    # correlated columns / rows so that the second pass has work to do
    C = A[:, :c] @ (np.eye(c) + 0.5 * g.standard_normal((c, c)))
    R = (np.eye(r) + 0.5 * g.standard_normal((r, r))) @ A[:r, :]
    Q1c, L1c = _chol_qr(C)
    Q1r, L1r = _chol_qr(R.T)
    _, L2c = _chol_qr(Q1c)
    _, L2r = _chol_qr(Q1r)
    inv = np.linalg.inv
    M1 = Q1c.T @ A @ Q1r
    M2 = inv(L2c).T @ inv(L2c) @ M1 @ inv(L2r).T @ inv(L2r)
    U = inv(L1c).T @ M2 @ inv(L1r)
    U_ls = np.linalg.pinv(C) @ A @ np.linalg.pinv(R)
    assert np.linalg.norm(U - U_ls) <= 1e-9 * np.linalg.norm(U_ls)
    CUR = Q1c @ M2 @ Q1r.T
    Pc = C @ np.linalg.pinv(C)
    Pr = np.linalg.pinv(R) @ R
    assert np.linalg.norm(CUR - Pc @ A @ Pr) <= 1e-9 * np.linalg.norm(A)
    assert np.linalg.norm(CUR - C @ U @ R) <= 1e-9 * np.linalg.norm(A)
    # the residual the fused kernel reduces equals the one of the explicit CUR
    Q = Q1c @ inv(L2c).T
    Qr = Q1r @ inv(L2r).T
    M = Q.T @ A @ Qr
    assert np.isclose(np.linalg.norm(A - CUR), np.linalg.norm(A - Q @ M @ Qr.T), rtol=1e-10)
