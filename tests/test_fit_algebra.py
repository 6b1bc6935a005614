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


@pytest.mark.parametrize("seed,m,n,c,r", [(2, 80, 60, 14, 11), (3, 120, 90, 24, 20)])
def test_second_pass_factor_moves_e_at_second_order_and_u_at_first(seed, m, n, c, r):
    """The reading behind taking the second pass's Gram G2 = Q1^T Q1 (near I)
    with one BF16 term: for G2 perturbed by a symmetric eps S (both sides),
    Q1 (G2 + eps S)^{-1} Q1^T differs from the projector onto range(C) only
    inside range(C) x range(C), which is orthogonal to A - P_C A P_R, so the
    relative residual e grows by O(eps^2) while U moves by O(eps).  Doubling
    eps multiplies the change of e by about 4 and that of U by about 2."""
    g = np.random.default_rng(seed)
    A = g.standard_normal((m, n))
    C = A[:, :c] @ (np.eye(c) + 0.5 * g.standard_normal((c, c)))
    R = (np.eye(r) + 0.5 * g.standard_normal((r, r))) @ A[:r, :]
    Q1c, L1c = _chol_qr(C)
    Q1r, L1r = _chol_qr(R.T)
    inv = np.linalg.inv

    def sym(k):
        S = g.standard_normal((k, k))
        S = S + S.T
        return S / np.linalg.norm(S, 2)

    Sc, Sr = sym(c), sym(r)
    M1 = Q1c.T @ A @ Q1r

    def fit(eps):
        L2c = np.linalg.cholesky(Q1c.T @ Q1c + eps * Sc)
        L2r = np.linalg.cholesky(Q1r.T @ Q1r + eps * Sr)
        M2 = inv(L2c).T @ inv(L2c) @ M1 @ inv(L2r).T @ inv(L2r)
        e = np.linalg.norm(A - Q1c @ M2 @ Q1r.T) / np.linalg.norm(A)
        return e, inv(L1c).T @ M2 @ inv(L1r)

    e0, U0 = fit(0.0)
    de, du = [], []
    for eps in (1e-3, 2e-3):
        e, U = fit(eps)
        de.append(e - e0)
        du.append(np.linalg.norm(U - U0) / np.linalg.norm(U0))
    assert de[0] > 0 and 3.5 <= de[1] / de[0] <= 4.5, de      # e only grows, as eps^2
    assert 1.8 <= du[1] / du[0] <= 2.2, du                      # U moves as eps
    assert de[0] < 1e-3 * du[0], (de, du)                        # second order against first
