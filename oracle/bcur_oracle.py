"""FP64 CPU oracle for the Block CUR hot path (arXiv 1703.06065).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against.  Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does.

Everything is written in FP64 NumPy (LAPACK for QR / SVD), in the paper's
order and notation, with no blocking or fusion:

1.  Top-k singular subspace of A by a randomized range finder with subspace
    iteration (the paper allows replacing its score estimate by sketching,
    Sec. 3.1; the iteration is Halko, Martinsson & Tropp 2011, Alg. 4.4,
    followed by their Alg. 5.1 for the SVD of the projected matrix).
2.  Block leverage scores, Def. 2 (Sec. 3):  l_g = ||V_{A,k}^T E_g||_F^2, and
    the row-block analogue from U_{A,k} (Sec. 3 applies the column rules to
    A^T; Corollary 1 in the appendix samples rows by ||e_i^T U_{A,k}||^2).
3.  Block sampling by inverse CDF (Alg. 1 step 2), without replacement by
    default as in the experiments (Sec. 4.1 footnote); with replacement and
    the scaling matrix S of Sec. 3.1 as an option.
4.  C = A[:, chosen column blocks], R = A[chosen row blocks, :] (Alg. 1).
5.  U = C^+ A R^+ (the least-squares optimal middle factor; see the readings
    below) and the residual ||A - CUR||_F with its relative form (Sec. 4.2).

Readings where the paper is silent (each restated where it is used):
* the sketch is a Rademacher (+-1) test matrix Omega of l = k + p columns,
  supplied by the caller (it is a random input, not part of the method);
* orthonormalisation is Householder QR; singular-vector signs are not
  normalised (scores do not depend on them);
* sampling picks, for draw t with uniform u_t, the first remaining block j
  whose running FP64 prefix sum S_j (sequential, increasing j) satisfies
  S_j > u_t * T, T the sequential FP64 sum of the remaining scores; if
  rounding leaves no such block it takes the last remaining block with a
  positive score, and if all remaining scores are zero the first remaining
  block;  p_j = l_j / sum(l) is reported for every draw;
* C and R are reported unscaled: with U = C^+ A R^+ the product CUR does not
  depend on a nonsingular scaling of the chosen blocks, so the scaling of
  Sec. 3.1 only matters for the paper's U = W^+ variant;
* pinv uses the singular-value threshold max(rows, cols) * eps64 * sigma_1.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

EPS64 = np.finfo(np.float64).eps


# ----------------------------------------------------------------------------
# 1. Randomized range finder and top-k singular factors
# ----------------------------------------------------------------------------

def orth(Y: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(Y) by Householder QR (reduced)."""
    q, _ = np.linalg.qr(np.asarray(Y, dtype=np.float64), mode="reduced")
    return q


def range_finder(A: np.ndarray, Omega: np.ndarray, q: int) -> np.ndarray:
    """Q with orthonormal columns approximating the dominant range of A.

    Randomized subspace iteration (Halko-Martinsson-Tropp 2011, Alg. 4.4):
    Q = orth(A Omega); then q times Z = orth(A^T Q), Q = orth(A Z).
    """
    A = np.asarray(A, dtype=np.float64)
    Q = orth(A @ Omega)
    for _ in range(q):
        Z = orth(A.T @ Q)
        Q = orth(A @ Z)
    return Q


def top_k_factors(A: np.ndarray, Q: np.ndarray, k: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """U_k, sigma_k, V_k of A restricted to range(Q) (HMT 2011 Alg. 5.1).

    B = Q^T A is formed through its transpose B^T = A^T Q = Q_B T (QR), so
    B = T^T Q_B^T; with the SVD T^T = U~ Sigma W^T the right singular vectors
    of B are Q_B W and the left singular vectors of A are Q U~ (Sec. 2.1
    notation: A = U Sigma V^T).
    """
    A = np.asarray(A, dtype=np.float64)
    Bt = A.T @ Q
    Qb, T = np.linalg.qr(Bt, mode="reduced")
    Ut, sig, Wt = np.linalg.svd(T.T)
    V = Qb @ Wt.T
    U = Q @ Ut
    return U[:, :k], sig[:k], V[:, :k]


def exact_top_k(A: np.ndarray, k: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Top-k singular triplets of A from a full LAPACK SVD (Sec. 2.1)."""
    U, s, Vt = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
    return U[:, :k], s[:k], Vt[:k].T


# ----------------------------------------------------------------------------
# 2. Block leverage scores (Def. 2) and diagnostics (Sec. 3.2)
# ----------------------------------------------------------------------------

def block_scores(F: np.ndarray, off: Sequence[int]) -> np.ndarray:
    """l_g = ||F^T E_g||_F^2 for the contiguous blocks [off[g], off[g+1]).

    With F = V_{A,k} (n x k) this is Def. 2 for column blocks; with
    F = U_{A,k} (m x k) it is the row-block score (Sec. 3, applied to A^T).
    """
    F = np.asarray(F, dtype=np.float64)
    G = len(off) - 1
    out = np.zeros(G)
    for g in range(G):
        blk = F[off[g]:off[g + 1], :]
        out[g] = float(np.sum(blk * blk))
    return out


def column_leverage_scores(V_k: np.ndarray) -> np.ndarray:
    """Def. 1: l_j = ||V_{A,k}^T e_j||^2 for every column j."""
    V_k = np.asarray(V_k, dtype=np.float64)
    return np.sum(V_k * V_k, axis=1)


def block_stable_rank_terms(V_k: np.ndarray, off: Sequence[int]) -> np.ndarray:
    """||V_k^T E_g||_F^2 / ||V_k^T E_g||_2^2 for every block g (NaN for a zero block)."""
    out = np.full(len(off) - 1, np.nan)
    for g in range(len(off) - 1):
        blk = np.asarray(V_k[off[g]:off[g + 1], :], dtype=np.float64)
        fro2 = float(np.sum(blk * blk))
        if fro2 == 0.0:
            continue
        spec = float(np.linalg.norm(blk, 2))
        out[g] = fro2 / (spec * spec)
    return out


def block_stable_rank(V_k: np.ndarray, off: Sequence[int]) -> float:
    """alpha = min_g ||V_k^T E_g||_F^2 / ||V_k^T E_g||_2^2 (Sec. 3.2 definition).

    Blocks whose restriction is exactly zero carry no information and are
    skipped (the ratio is undefined there).
    """
    t = block_stable_rank_terms(V_k, off)
    t = t[~np.isnan(t)]
    return float(t.min()) if t.size else float("nan")


def incoherence(U_k: np.ndarray) -> float:
    """mu = (m/k) max_i ||U_k^T e_i||^2 (Sec. 3.2 definition)."""
    U_k = np.asarray(U_k, dtype=np.float64)
    m, k = U_k.shape
    return (m / k) * float(np.max(np.sum(U_k * U_k, axis=1)))


# ----------------------------------------------------------------------------
# 3. Sampling (Alg. 1 step 2, the matrix S of Sec. 3.1)
# ----------------------------------------------------------------------------

def sample_blocks(scores: Sequence[float], u: Sequence[float], g: int,
                  replacement: bool = False) -> Tuple[List[int], List[float]]:
    """Draw ``g`` blocks with probability proportional to ``scores``.

    Pure-Python FP64 arithmetic (each + and * rounds once, no fused
    multiply-add), sequential in increasing block index, as stated in the
    module header.  Returns the block indices in draw order and, for each
    draw, p_j = l_j / sum(l) of the chosen block.
    """
    l = [float(x) for x in scores]
    G = len(l)
    if not replacement and g > G:
        raise ValueError("cannot draw more blocks than exist without replacement")
    total0 = 0.0
    for j in range(G):
        total0 = total0 + l[j]
    remaining = [True] * G
    idx: List[int] = []
    prob: List[float] = []
    for t in range(g):
        T = 0.0
        for j in range(G):
            if remaining[j]:
                T = T + l[j]
        x = float(u[t]) * T
        pick = -1
        S = 0.0
        for j in range(G):
            if remaining[j]:
                S = S + l[j]
                if S > x:
                    pick = j
                    break
        if pick < 0:
            positive = [j for j in range(G) if remaining[j] and l[j] > 0.0]
            if positive:
                pick = positive[-1]
            else:
                pick = next(j for j in range(G) if remaining[j])
        idx.append(pick)
        prob.append(l[pick] / total0 if total0 > 0.0 else 0.0)
        if not replacement:
            remaining[pick] = False
    return idx, prob


def sampling_matrix(idx: Sequence[int], prob: Sequence[float], off: Sequence[int]) -> np.ndarray:
    """S (n x sum_t s_{j_t}) of Sec. 3.1: block (j_t, t) is I / sqrt(g p_{j_t}).

    Column block t of S selects block j_t.  With equal blocks this is the
    printed n x g s matrix; Sec. 3 notes the method extends to blocks of
    varying size, which here means block column t is as wide as block j_t.
    """
    g = len(idx)
    sizes = np.diff(np.asarray(off))
    n = int(off[-1])
    widths = [int(sizes[j]) for j in idx]
    S = np.zeros((n, int(sum(widths))))
    c0 = 0
    for t, (j, p) in enumerate(zip(idx, prob)):
        w = widths[t]
        S[off[j]:off[j + 1], c0:c0 + w] = np.eye(w) / math.sqrt(g * p)
        c0 += w
    return S


def block_cols(off: Sequence[int], idx: Sequence[int]) -> np.ndarray:
    """Concatenated index list of the chosen blocks, in draw order."""
    return np.concatenate([np.arange(off[j], off[j + 1]) for j in idx]) if len(idx) else np.zeros(0, np.int64)


# ----------------------------------------------------------------------------
# 4-5. C, R, U and the residual
# ----------------------------------------------------------------------------

def gather_columns(A: np.ndarray, off: Sequence[int], idx: Sequence[int]) -> np.ndarray:
    """C = A[:, blocks idx] (unscaled; see the module header)."""
    return np.asarray(A, dtype=np.float64)[:, block_cols(off, idx)]


def gather_rows(A: np.ndarray, off: Sequence[int], idx: Sequence[int]) -> np.ndarray:
    """R = A[blocks idx, :] (unscaled)."""
    return np.asarray(A, dtype=np.float64)[block_cols(off, idx), :]


def pinv(X: np.ndarray) -> np.ndarray:
    """Moore-Penrose pseudoinverse (Sec. 2.1: X^+ = V Sigma^-1 U^T) by SVD.

    Singular values at or below max(rows, cols) * eps64 * sigma_1 are treated
    as zero.
    """
    X = np.asarray(X, dtype=np.float64)
    if X.size == 0:
        return X.T.copy()
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    tol = max(X.shape) * EPS64 * (s[0] if s.size else 0.0)
    inv = np.where(s > tol, 1.0 / np.where(s > tol, s, 1.0), 0.0)
    return (Vt.T * inv) @ U.T


def fit_u(A: np.ndarray, C: np.ndarray, R: np.ndarray) -> np.ndarray:
    """U = C^+ A R^+, the minimiser of ||A - C U R||_F over U."""
    return pinv(C) @ np.asarray(A, dtype=np.float64) @ pinv(R)


def fit_w_pinv(R: np.ndarray, S: np.ndarray) -> np.ndarray:
    """The paper's U = W^+ with W = R S, the scaled intersection (Alg. 1 step 3)."""
    return pinv(np.asarray(R, dtype=np.float64) @ S)


def truncate_rank(U: np.ndarray, k: int) -> np.ndarray:
    """U_k, the best rank-k approximation of U (Sec. 4.1)."""
    Uu, s, Vt = np.linalg.svd(np.asarray(U, dtype=np.float64), full_matrices=False)
    return (Uu[:, :k] * s[:k]) @ Vt[:k]


def residual(A: np.ndarray, C: np.ndarray, U: np.ndarray, R: np.ndarray) -> Tuple[float, float]:
    """||A - C U R||_F and its relative form ||A - CUR||_F / ||A||_F (Sec. 4.2)."""
    A = np.asarray(A, dtype=np.float64)
    D = A - C @ U @ R
    err = float(np.linalg.norm(D))
    na = float(np.linalg.norm(A))
    return err, (err / na if na > 0.0 else 0.0)


def tail_norm(A: np.ndarray, k: int) -> float:
    """||A - A_k||_F, the best rank-k error (Sec. 2.1, Eckart-Young)."""
    s = np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False)
    return float(np.sqrt(np.sum(s[k:] ** 2)))


def numerical_rank(X: np.ndarray) -> int:
    """Number of singular values above max(rows, cols) * eps64 * sigma_1."""
    X = np.asarray(X, dtype=np.float64)
    if X.size == 0:
        return 0
    s = np.linalg.svd(X, compute_uv=False)
    return int(np.sum(s > max(X.shape) * EPS64 * s[0])) if s[0] > 0 else 0


def algorithm1(A: np.ndarray, col_off: Sequence[int], r: int, g: int, u_rows: Sequence[float],
               u_cols: Sequence[float]) -> Dict:
    """Alg. 1 (Sec. 3.1) as printed: r rows uniformly (p_i = 1/m, with
    replacement) with R = S_R^T A scaled by 1/sqrt(r p_i); column-block scores
    l_i(R) = ||V_R^T E_i||_F^2 from the right singular vectors of R; g blocks
    drawn with replacement from p_i = l_i / sum(l); C = A S and W = R S with
    the scaling of Sec. 3.1; U = W^+.

    Reading: when rank(R) = rho < r the top-r right singular vectors include
    arbitrary null-space directions, so V_R keeps the rho vectors of the
    numerical row space (sum(l) = rho) -- the scores are then unique.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    rows, _ = sample_blocks(np.ones(m), u_rows, r, replacement=True)
    R = math.sqrt(m / r) * A[rows, :]
    _, sR, VtR = np.linalg.svd(R, full_matrices=False)
    rho = numerical_rank(R)
    V_R = VtR[:rho].T
    scores = block_scores(V_R, col_off)
    cols, prob = sample_blocks(scores, u_cols, g, replacement=True)
    S = sampling_matrix(cols, prob, col_off)
    C = A @ S
    W = R @ S
    U = pinv(W)
    err, rel = residual(A, C, U, R)
    return dict(row_idx=rows, R=R, rank_R=rho, col_scores=scores, col_idx=cols, col_prob=prob,
                S=S, C=C, W=W, U=U, err=err, rel=rel)


# ----------------------------------------------------------------------------
# Whole pipeline
# ----------------------------------------------------------------------------

def block_cur(A: np.ndarray, col_off: Sequence[int], row_off: Sequence[int], k: int, q: int,
              g_col: int, g_row: int, Omega: np.ndarray, u_col: Sequence[float],
              u_row: Sequence[float], replacement: bool = False,
              col_idx: Sequence[int] = None, row_idx: Sequence[int] = None) -> Dict:
    """Run the hot path end to end in FP64 and return every intermediate.

    ``col_idx`` / ``row_idx`` force the block choice (used where a draw lands
    on a CDF boundary within tolerance and the downstream steps must follow
    the oracle's own choice).
    """
    A64 = np.asarray(A, dtype=np.float64)
    Q = range_finder(A64, Omega, q)
    U_k, sig, V_k = top_k_factors(A64, Q, k)
    cs = block_scores(V_k, col_off)
    rs = block_scores(U_k, row_off)
    ci, cp = sample_blocks(cs, u_col, g_col, replacement)
    ri, rp = sample_blocks(rs, u_row, g_row, replacement)
    if col_idx is not None:
        ci = [int(x) for x in col_idx]
    if row_idx is not None:
        ri = [int(x) for x in row_idx]
    C = gather_columns(A64, col_off, ci)
    R = gather_rows(A64, row_off, ri)
    U = fit_u(A64, C, R)
    err, rel = residual(A64, C, U, R)
    return dict(Q=Q, U_k=U_k, sigma=sig, V_k=V_k, col_scores=cs, row_scores=rs,
                col_idx=ci, row_idx=ri, col_prob=cp, row_prob=rp, C=C, R=R, U=U,
                err=err, rel=rel)
