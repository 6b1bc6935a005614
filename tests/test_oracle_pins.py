"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these re-types an oracle formula: each compares the oracle with a
closed form, an independent computation (a different LAPACK route, a
Kronecker least-squares system, brute force), a value printed in the paper,
or an exact probability.
"""
import itertools
import math
import os

import numpy as np
import pytest

import bcur_inputs as bi
import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


# ----------------------------------------------------------------------------
# Block leverage scores (Def. 1, Def. 2)
# ----------------------------------------------------------------------------

def test_scores_sum_to_k():
    """V_k has orthonormal columns, so the block scores sum to k (Def. 2)."""
    p = bi.plain_fp64_512x1024()
    A = p.matrix()
    Q = orc.range_finder(A, p.omega(), p.q)
    U_k, s, V_k = orc.top_k_factors(A, Q, p.k)
    for F, off in ((V_k, p.col_off), (U_k, p.row_off)):
        sc = orc.block_scores(F, off)
        assert abs(sc.sum() - p.k) <= 1e-12 * p.k
        assert np.all(sc >= 0)


def test_single_block_scores_equal_k():
    rg = _rng(1)
    A = rg.standard_normal((40, 60))
    Om = bi.rademacher(60, 12, 5)
    U_k, s, V_k = orc.top_k_factors(A, orc.range_finder(A, Om, 2), 7)
    sc = orc.block_scores(V_k, [0, 60])
    assert sc.shape == (1,) and abs(sc[0] - 7) < 1e-12


def test_block_size_one_is_column_leverage_from_full_svd():
    """s = 1 reduces Def. 2 to Def. 1; rank(A) <= l makes the sketch exact,
    so the randomized scores equal those of a full LAPACK SVD of A."""
    rg = _rng(2)
    m, n, rank, k, l = 50, 70, 8, 5, 12
    A = rg.standard_normal((m, rank)) @ (np.diag([9, 7, 5, 4, 3, 2, 1.5, 1.0]) @ rg.standard_normal((rank, n)))
    Om = bi.rademacher(n, l, 3)
    U_k, s, V_k = orc.top_k_factors(A, orc.range_finder(A, Om, 1), k)
    got = orc.block_scores(V_k, np.arange(n + 1))
    Uf, sf, Vtf = np.linalg.svd(A)
    want = np.sum(Vtf[:k].T ** 2, axis=1)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11)
    np.testing.assert_allclose(s, sf[:k], rtol=1e-11)
    # rows: U_k row norms
    got_r = orc.block_scores(U_k, np.arange(m + 1))
    np.testing.assert_allclose(got_r, np.sum(Uf[:, :k] ** 2, axis=1), rtol=0, atol=1e-11)


def _structured_factor(rows, k, rg):
    """Orthonormal rows x k factor whose column t is cos(th) e_a + sin(th) e_b
    on disjoint supports, with its exact squared row norms."""
    perm = rg.permutation(rows)[: 2 * k]
    th = rg.uniform(0.1, 1.4, size=k)
    F = np.zeros((rows, k))
    lev = np.zeros(rows)
    for t in range(k):
        a, b = perm[2 * t], perm[2 * t + 1]
        F[a, t], F[b, t] = math.cos(th[t]), math.sin(th[t])
        lev[a], lev[b] = math.cos(th[t]) ** 2, math.sin(th[t]) ** 2
    return F, lev


def test_closed_form_block_scores():
    """A = U diag(sigma) V^T with hand-built sparse orthonormal U, V: every
    block score is a sum of known cos^2 / sin^2 terms."""
    rg = _rng(4)
    m, n, k, s = 48, 64, 6, 8
    U, levU = _structured_factor(m, k, rg)
    V, levV = _structured_factor(n, k, rg)
    sig = np.array([10.0, 8.0, 6.0, 4.0, 3.0, 2.0])
    A = (U * sig) @ V.T
    col_off, row_off = bi.uniform_blocks(n, s), bi.uniform_blocks(m, s)
    Om = bi.rademacher(n, k + 4, 11)
    r = orc.block_cur(A, col_off, row_off, k, 1, 3, 3, Om, [0.3, 0.6, 0.9], [0.2, 0.5, 0.8])
    want_c = np.array([levV[col_off[g]:col_off[g + 1]].sum() for g in range(n // s)])
    want_r = np.array([levU[row_off[g]:row_off[g + 1]].sum() for g in range(m // s)])
    np.testing.assert_allclose(r["col_scores"], want_c, atol=1e-12)
    np.testing.assert_allclose(r["row_scores"], want_r, atol=1e-12)


def test_scores_invariant_to_permutation_within_block():
    rg = _rng(5)
    m, n, s, k, l = 30, 48, 6, 4, 9
    A = rg.standard_normal((m, 5)) @ rg.standard_normal((5, n)) + 1e-3 * rg.standard_normal((m, n))
    Om = bi.rademacher(n, l, 6)
    off = bi.uniform_blocks(n, s)
    perm = np.concatenate([off[g] + rg.permutation(s) for g in range(n // s)])
    _, _, V1 = orc.top_k_factors(A, orc.range_finder(A, Om, 2), k)
    _, _, V2 = orc.top_k_factors(A[:, perm], orc.range_finder(A[:, perm], Om[perm], 2), k)
    np.testing.assert_allclose(orc.block_scores(V1, off), orc.block_scores(V2, off), atol=1e-12)


def test_range_finder_exact_for_low_rank():
    """rank(A) <= l: randomized top-k triplets equal the exact SVD's."""
    rg = _rng(6)
    A = rg.standard_normal((80, 6)) @ rg.standard_normal((6, 90))
    Q = orc.range_finder(A, bi.rademacher(90, 10, 2), 0)
    U_k, s, V_k = orc.top_k_factors(A, Q, 4)
    Ue, se, Ve = orc.exact_top_k(A, 4)
    np.testing.assert_allclose(s, se, rtol=1e-12)
    np.testing.assert_allclose(V_k @ V_k.T, Ve @ Ve.T, atol=1e-12)
    np.testing.assert_allclose(U_k @ U_k.T, Ue @ Ue.T, atol=1e-12)


def test_block_stable_rank_and_incoherence_bounds():
    """1 <= alpha <= s (Sec. 3.2) and 1 <= mu <= m/k."""
    rg = _rng(7)
    A = rg.standard_normal((60, 80))
    U_k, s, V_k = orc.exact_top_k(A, 6)
    for sz in (1, 4, 8, 16):
        a = orc.block_stable_rank(V_k, bi.uniform_blocks(80, sz))
        assert 1.0 - 1e-12 <= a <= sz + 1e-12
    mu = orc.incoherence(U_k)
    assert 1.0 - 1e-12 <= mu <= 60 / 6 + 1e-12
    # a rank-1 block has stable rank exactly 1
    V = np.zeros((8, 2)); V[0:2, 0] = [0.6, 0.8]; V[2:8, 1] = 1 / math.sqrt(6)
    assert abs(orc.block_stable_rank(V, [0, 2, 8]) - 1.0) < 1e-12


# ----------------------------------------------------------------------------
# Sampling (Alg. 1 step 2, Sec. 3.1)
# ----------------------------------------------------------------------------

def test_inverse_cdf_hand_cases():
    sc = [1.0, 2.0, 3.0, 4.0]  # T = 10, prefix sums 1, 3, 6, 10
    assert orc.sample_blocks(sc, [0.05], 1, True)[0] == [0]   # x = 0.5 < 1
    assert orc.sample_blocks(sc, [0.1], 1, True)[0] == [1]    # x = 1.0: strict >
    assert orc.sample_blocks(sc, [0.95], 1, True)[0] == [3]   # x = 9.5
    assert orc.sample_blocks(sc, [0.0], 1, True)[0] == [0]
    # without replacement: 3 (x=9.5 of 10), then 2 (x=5.7 of 6), then 0 (x=0 of 3)
    idx, pr = orc.sample_blocks(sc, [0.95, 0.95, 0.0], 3, False)
    assert idx == [3, 2, 0]
    assert pr == [0.4, 0.3, 0.1]
    # zero-score blocks are never drawn while positive mass remains; once it
    # is exhausted the lowest remaining index is taken.
    idx, _ = orc.sample_blocks([0.0, 5.0, 0.0, 5.0], [0.0, 0.0, 0.0, 0.0], 4, False)
    assert idx == [1, 3, 0, 2]
    with pytest.raises(ValueError):
        orc.sample_blocks(sc, [0.1] * 5, 5, False)


def test_sampling_frequencies_match_successive_probabilities():
    """Ordered pairs drawn without replacement have probability
    p_a * p_b / (1 - p_a); chi-square at a fixed seed."""
    from scipy.stats import chisquare

    sc = np.array([1.0, 2.0, 3.0, 4.0])
    p = sc / sc.sum()
    N = 20000
    u = bi.uniforms(2 * N, 123, 9).reshape(N, 2)
    counts = {}
    for t in range(N):
        key = tuple(orc.sample_blocks(sc, u[t], 2, False)[0])
        counts[key] = counts.get(key, 0) + 1
    pairs = [(a, b) for a in range(4) for b in range(4) if a != b]
    exp = np.array([p[a] * p[b] / (1 - p[a]) for a, b in pairs]) * N
    obs = np.array([counts.get(pr, 0) for pr in pairs])
    assert obs.sum() == N
    assert chisquare(obs, exp).pvalue > 1e-3


def test_sampling_matrix_matches_printed_example():
    """S for the order [1, 3, 2] with G = 4 (Sec. 3.1, printed example)."""
    rows = []
    with open(os.path.join(GOLDEN, "s_matrix_example.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(x) for x in line.split()))
    G, g, s = 4, 3, 2
    pvals = {1: 0.1, 2: 0.2, 3: 0.3, 4: 0.4}
    order = [1, 3, 2]
    S = orc.sampling_matrix([j - 1 for j in order], [pvals[j] for j in order],
                            bi.uniform_blocks(G * s, s))
    assert S.shape == (G * s, g * s)
    want = np.zeros_like(S)
    for rb, cb, pj in rows:
        want[(rb - 1) * s:rb * s, (cb - 1) * s:cb * s] = np.eye(s) / math.sqrt(g * pvals[pj])
    np.testing.assert_array_equal(S, want)
    assert not S[3 * s:].any()


def test_with_replacement_scaling_is_unbiased():
    """E||Q S||_F^2 = ||Q||_F^2 (appendix, proof of Lemma 3) and
    E[(A S)(S^T B)] = A B (block multiplication lemma), Monte Carlo."""
    rg = _rng(8)
    G, s, g = 6, 3, 4
    n = G * s
    off = bi.uniform_blocks(n, s)
    Q = rg.standard_normal((5, n))
    Bm = rg.standard_normal((n, 4))
    w = np.array([np.sum(Q[:, off[i]:off[i + 1]] ** 2) for i in range(G)])
    trials = 6000
    u = bi.uniforms(g * trials, 77, 9).reshape(trials, g)
    acc_norm, acc_prod = 0.0, np.zeros((5, 4))
    for t in range(trials):
        idx, pr = orc.sample_blocks(w, u[t], g, True)
        S = orc.sampling_matrix(idx, pr, off)
        acc_norm += np.sum((Q @ S) ** 2)
        acc_prod += (Q @ S) @ (S.T @ Bm)
    assert abs(acc_norm / trials - np.sum(Q ** 2)) < 0.01 * np.sum(Q ** 2)
    err = np.linalg.norm(acc_prod / trials - Q @ Bm)
    assert err < 0.05 * np.linalg.norm(Q) * np.linalg.norm(Bm)


# ----------------------------------------------------------------------------
# U and the residual
# ----------------------------------------------------------------------------

def _tiny(seed, m=12, n=16, rank=None):
    rg = _rng(seed)
    if rank is None:
        return rg.standard_normal((m, n))
    return rg.standard_normal((m, rank)) @ rg.standard_normal((rank, n))


def _kron_lstsq_err(A, C, R):
    """min_U ||A - C U R||_F by the Kronecker least-squares system
    (R^T kron C) vec(U) = vec(A) -- independent of the pinv route."""
    K = np.kron(R.T, C)
    x, *_ = np.linalg.lstsq(K, A.reshape(-1, order="F"), rcond=None)
    U = x.reshape(C.shape[1], R.shape[0], order="F")
    return float(np.linalg.norm(A - C @ U @ R)), U


def test_error_zero_when_blocks_span_low_rank_matrix():
    A = _tiny(10, 24, 32, rank=3)
    col_off, row_off = bi.uniform_blocks(32, 4), bi.uniform_blocks(24, 4)
    C = orc.gather_columns(A, col_off, [1, 5])
    R = orc.gather_rows(A, row_off, [0, 4])
    U = orc.fit_u(A, C, R)
    err, rel = orc.residual(A, C, U, R)
    assert rel < 1e-12


def test_error_zero_with_all_blocks():
    A = _tiny(11)
    col_off, row_off = bi.uniform_blocks(16, 4), bi.uniform_blocks(12, 4)
    C = orc.gather_columns(A, col_off, [2, 0, 3, 1])
    R = orc.gather_rows(A, row_off, [1, 2, 0])
    assert orc.residual(A, C, orc.fit_u(A, C, R), R)[1] < 1e-12


def test_all_rows_gives_column_subset_selection_error():
    """R = A (every row block): ||A - CUR|| = ||A - C C^+ A|| (Remark, Sec. 3.3)."""
    A = _tiny(12, 20, 24)
    col_off, row_off = bi.uniform_blocks(24, 4), bi.uniform_blocks(20, 5)
    C = orc.gather_columns(A, col_off, [4, 1])
    R = orc.gather_rows(A, row_off, [0, 1, 2, 3])
    X, *_ = np.linalg.lstsq(C, A, rcond=None)
    want = np.linalg.norm(A - C @ X)
    got = orc.residual(A, C, orc.fit_u(A, C, R), R)[0]
    assert abs(got - want) < 1e-11 * np.linalg.norm(A)


def test_pythagoras_normal_equations_and_lower_bounds():
    rg = _rng(13)
    A = rg.standard_normal((30, 6)) @ rg.standard_normal((6, 40)) + 0.3 * rg.standard_normal((30, 40))
    col_off, row_off = bi.uniform_blocks(40, 5), bi.uniform_blocks(30, 5)
    C = orc.gather_columns(A, col_off, [0, 3, 6])
    R = orc.gather_rows(A, row_off, [1, 4])
    U = orc.fit_u(A, C, R)
    err, _ = orc.residual(A, C, U, R)
    Qc, _ = np.linalg.qr(C)
    Qr, _ = np.linalg.qr(R.T)
    M = Qc.T @ A @ Qr
    assert abs(err ** 2 - (np.sum(A ** 2) - np.sum(M ** 2))) < 1e-10 * np.sum(A ** 2)
    np.testing.assert_allclose(C.T @ C @ U @ R @ R.T, C.T @ A @ R.T, atol=1e-9 * np.linalg.norm(A) ** 3)
    sv = np.linalg.svd(A, compute_uv=False)
    rank_cur = min(C.shape[1], R.shape[0])
    assert err >= math.sqrt(np.sum(sv[rank_cur:] ** 2)) - 1e-12
    e_c = np.linalg.norm(A - Qc @ (Qc.T @ A))
    e_r = np.linalg.norm(A - (A @ Qr) @ Qr.T)
    assert err >= max(e_c, e_r) - 1e-12
    kerr, _ = _kron_lstsq_err(A, C, R)
    assert abs(err - kerr) < 1e-10 * np.linalg.norm(A)


def test_regression_identity_from_appendix():
    """A S (B S)^+ B = A S (V_k^T S)^+ V_k^T for rank-k B (proof of Lemma 3)."""
    rg = _rng(14)
    n, s, k = 24, 4, 3
    A = rg.standard_normal((7, n))
    B = rg.standard_normal((5, k)) @ rg.standard_normal((k, n))
    _, _, Vt = np.linalg.svd(B)
    V_k = Vt[:k].T
    off = bi.uniform_blocks(n, s)
    S = orc.sampling_matrix([0, 2, 5], [0.2, 0.3, 0.1], off)
    lhs = A @ S @ orc.pinv(B @ S) @ B
    rhs = A @ S @ orc.pinv(V_k.T @ S) @ V_k.T
    np.testing.assert_allclose(lhs, rhs, atol=1e-10)


def test_brute_force_tiny_all_block_subsets():
    """12 x 16, s = 4: every (column pair, row pair) of blocks; the oracle's
    pinv-based error equals the Kronecker least-squares minimum, and the
    sampled pipeline's error lies within the brute-force range."""
    A = _tiny(15) + 0.0
    col_off, row_off = bi.uniform_blocks(16, 4), bi.uniform_blocks(12, 4)
    errs = []
    for cj in itertools.combinations(range(4), 2):
        for ri in itertools.combinations(range(3), 2):
            C = orc.gather_columns(A, col_off, cj)
            R = orc.gather_rows(A, row_off, ri)
            e = orc.residual(A, C, orc.fit_u(A, C, R), R)[0]
            ek, _ = _kron_lstsq_err(A, C, R)
            assert abs(e - ek) < 1e-10 * np.linalg.norm(A)
            errs.append(e)
    r = orc.block_cur(A, col_off, row_off, 3, 1, 2, 2, bi.rademacher(16, 5, 1),
                      bi.uniforms(2, 1, 3), bi.uniforms(2, 1, 4))
    assert min(errs) - 1e-12 <= r["err"] <= max(errs) + 1e-12


def test_cur_error_can_beat_rank_k_tail_but_not_rank_min_cr():
    """With U = C^+ A R^+ the error is bounded below by ||A - A_{min(c,r)}||,
    not by ||A - A_k|| (all blocks sampled: error 0 < ||A - A_k||)."""
    p = bi.plain_fp64_512x1024()
    A = p.matrix()
    r = orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row,
                      p.omega(), p.u_col(), p.u_row())
    sv = np.linalg.svd(A, compute_uv=False)
    c, rr = r["C"].shape[1], r["R"].shape[0]
    assert r["err"] >= math.sqrt(np.sum(sv[min(c, rr):] ** 2))
    assert abs(sum(r["col_scores"]) - p.k) < 1e-9 and abs(sum(r["row_scores"]) - p.k) < 1e-9
    assert len(set(r["col_idx"])) == p.g_col and len(set(r["row_idx"])) == p.g_row


def test_rank_k_truncation_of_u():
    rg = _rng(16)
    U = rg.standard_normal((9, 7))
    Uk = orc.truncate_rank(U, 3)
    assert np.linalg.matrix_rank(Uk) == 3
    sv = np.linalg.svd(U, compute_uv=False)
    assert abs(np.linalg.norm(U - Uk) - math.sqrt(np.sum(sv[3:] ** 2))) < 1e-12


# ----------------------------------------------------------------------------
# Planted mistakes: each must be caught by one of the pins above.
# ----------------------------------------------------------------------------

def test_planted_mistakes_are_caught(monkeypatch):
    import oracle.bcur_oracle as ob

    # (a) scores from U_k instead of V_k (transposed operand)
    orig = ob.top_k_factors

    def swapped(A, Q, k):
        U, s, V = orig(A, Q, k)
        return V, s, U  # left and right factors exchanged
    monkeypatch.setattr(ob, "top_k_factors", swapped)
    with pytest.raises(Exception):
        test_closed_form_block_scores()
    monkeypatch.setattr(ob, "top_k_factors", orig)

    # (b) non-strict CDF comparison
    orig_s = ob.sample_blocks

    def ge_sampler(scores, u, g, replacement=False):
        l = list(scores); T = sum(l); x = u[0] * T; S = 0.0
        for j, v in enumerate(l):
            S += v
            if S >= x:
                return [j], [v / T]
    monkeypatch.setattr(ob, "sample_blocks", ge_sampler)
    with pytest.raises(AssertionError):
        assert ob.sample_blocks([1.0, 2.0, 3.0, 4.0], [0.1], 1, True)[0] == [1]
    monkeypatch.setattr(ob, "sample_blocks", orig_s)

    # (c) U without the right pseudo-inverse
    bad = lambda A, C, R: ob.pinv(C) @ A @ R.T  # noqa: E731
    monkeypatch.setattr(ob, "fit_u", bad)
    monkeypatch.setattr(orc, "fit_u", bad)
    with pytest.raises(AssertionError):
        test_pythagoras_normal_equations_and_lower_bounds()


def test_paper_u_is_moore_penrose_inverse_of_scaled_intersection():
    """U = W^+ with W = R S (Alg. 1 step 3) satisfies the four Penrose conditions."""
    rg = _rng(17)
    R = rg.standard_normal((5, 24))
    off = bi.uniform_blocks(24, 4)
    S = orc.sampling_matrix([1, 4, 2], [0.2, 0.1, 0.3], off)
    W = R @ S
    U = orc.fit_w_pinv(R, S)
    np.testing.assert_allclose(W @ U @ W, W, atol=1e-10)
    np.testing.assert_allclose(U @ W @ U, U, atol=1e-10)
    np.testing.assert_allclose((W @ U).T, W @ U, atol=1e-10)
    np.testing.assert_allclose((U @ W).T, U @ W, atol=1e-10)


def test_algorithm1_scores_sum_to_rank_and_exact_for_low_rank():
    """Alg. 1 as printed: the scores sum to rank(R); for a rank-3 matrix whose
    sampled rows and blocks span it, rank(W) = rank(A) and A = C W^+ R exactly
    (the classical CUR exactness property of the pseudo-inverse of the
    intersection)."""
    rg = _rng(18)
    A = rg.standard_normal((40, 3)) @ rg.standard_normal((3, 48))
    off = bi.uniform_blocks(48, 4)
    r = orc.algorithm1(A, off, r=8, g=5, u_rows=bi.uniforms(8, 1, 3), u_cols=bi.uniforms(5, 1, 4))
    assert r["rank_R"] == 3
    assert abs(sum(r["col_scores"]) - 3) < 1e-10
    assert np.linalg.matrix_rank(r["W"]) == 3
    assert r["rel"] < 1e-10
    # full-rank noise: scores sum to r, error strictly positive
    A2 = A + 0.1 * rg.standard_normal(A.shape)
    r2 = orc.algorithm1(A2, off, r=8, g=5, u_rows=bi.uniforms(8, 2, 3), u_cols=bi.uniforms(5, 2, 4))
    assert r2["rank_R"] == 8 and abs(sum(r2["col_scores"]) - 8) < 1e-10
    assert r2["rel"] > 1e-3


def test_algorithm1_uniform_rows_follow_the_inverse_cdf():
    """With equal scores the inverse CDF picks floor(u m)."""
    u = [0.0, 0.49, 0.999, 0.25]
    idx, p = orc.sample_blocks(np.ones(10), u, 4, True)
    assert idx == [0, 4, 9, 2] and all(abs(x - 0.1) < 1e-15 for x in p)


def test_sampling_matrix_with_unequal_blocks_selects_and_scales():
    """Blocks of sizes 1, 3, 2: A S takes the drawn blocks in draw order, each
    scaled by 1/sqrt(g p)."""
    off = [0, 1, 4, 6]
    S = orc.sampling_matrix([2, 0, 2], [0.5, 0.25, 0.5], off)
    assert S.shape == (6, 5)
    A = np.arange(12.0).reshape(2, 6)
    got = A @ S
    want = np.hstack([A[:, 4:6] / math.sqrt(1.5), A[:, 0:1] / math.sqrt(0.75),
                      A[:, 4:6] / math.sqrt(1.5)])
    np.testing.assert_allclose(got, want, atol=1e-14)
