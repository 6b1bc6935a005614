"""Helpers shared by the GPU parity tests (oracle on the host, library on cuda:0)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bcur_inputs as bi  # noqa: E402
import oracle as orc  # noqa: E402


def device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06065_gb300 import build

    build.build()
    return torch.device("cuda", torch.cuda.current_device())


def to_dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device())


def tie_draws(scores, u, g, replacement, tol):
    """First draw index whose x = u*T lies within tol of an oracle CDF boundary
    (g if none): up to there the GPU must reproduce the oracle bit for bit."""
    l = [float(v) for v in scores]
    G = len(l)
    rem = [True] * G
    for t in range(g):
        T = 0.0
        for j in range(G):
            if rem[j]:
                T += l[j]
        x = float(u[t]) * T
        S = 0.0
        pick = -1
        for j in range(G):
            if rem[j]:
                S += l[j]
                if abs(S - x) <= tol:
                    return t
                if pick < 0 and S > x:
                    pick = j
        if pick < 0:
            return t
        if not replacement:
            rem[pick] = False
    return g


def run_problem(p, sketch_prec=None, fit_prec=None, A=None, force_oracle_idx=True):
    """Oracle and library on the same stored matrix; returns (oracle dict, gpu dict)."""
    import paper_1703_06065_gb300 as pkg

    dev = device()
    A = p.matrix() if A is None else A
    om = p.omega()
    uc, ur = p.u_col(), p.u_row()
    ref = orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row, om, uc, ur,
                        replacement=p.replacement)
    tdt = torch.float64 if p.storage == "f64" else torch.float32
    plan = pkg.Plan(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row,
                    dtype=p.storage, replacement=p.replacement, sketch_prec=sketch_prec,
                    fit_prec=fit_prec)
    At = to_dev(A, tdt)
    omt = to_dev(om.T, tdt)
    ucd, urd = to_dev(uc), to_dev(ur)
    cs, rs = plan.scores(At, omt)
    ci, ri, cp, rp = plan.sample(cs, rs, ucd, urd)
    gpu = dict(col_scores=cs.cpu().numpy(), row_scores=rs.cpu().numpy(),
               col_idx=ci.cpu().tolist(), row_idx=ri.cpu().tolist(), col_prob=cp.cpu().numpy())
    # Downstream steps follow the oracle's blocks where a draw ties (and,
    # with force_oracle_idx, always) so that U and the error compare like
    # for like.
    tol_c = p.col_off.size * 1e-6 * float(np.sum(ref["col_scores"]))
    tol_r = p.row_off.size * 1e-6 * float(np.sum(ref["row_scores"]))
    gpu["col_ok_draws"] = tie_draws(ref["col_scores"], uc, p.g_col, p.replacement, tol_c)
    gpu["row_ok_draws"] = tie_draws(ref["row_scores"], ur, p.g_row, p.replacement, tol_r)
    if force_oracle_idx:
        ci = to_dev(np.asarray(ref["col_idx"], dtype=np.int32))
        ri = to_dev(np.asarray(ref["row_idx"], dtype=np.int32))
    U, C, R = plan.fit(At, ci, ri, want_c=True, want_r=True)
    e = plan.error(At)
    plan.sync_status()
    gpu.update(U=U.double().cpu().numpy(), C=C.double().cpu().numpy().T,
               R=R.double().cpu().numpy(), err=e.cpu().numpy(), rank=plan.rank())
    return ref, gpu, plan


# Unit round-offs of the arithmetic the precisions stand for: one BF16 term
# (8 significant bits), e4m3 (4 bits), a BF16 hi/lo pair (about 16 bits,
# including the dropped lo*lo term and FP32 accumulation) and FP32 with its
# accumulation over long sums.
UNIT = {"bf16": 2.0 ** -8, "fp8": 2.0 ** -4, "bf16x3": 2.0 ** -16, "f32": 2.0 ** -22}


def score_bound(A, k, u, lmax, safety=2.0):
    """First-order bound on |l_gpu - l_oracle| for block scores computed from
    a sketch at unit round-off u.

    Independent roundings of A and of each orthonormal panel (relative size
    u / sqrt(3) on average) perturb the coupling between the k-th and
    (k+1)-th singular pairs of A by about
        de = u / sqrt(3) * (||A||_F / sqrt(m n) + sigma_1 / sqrt(min(m, n)));
    the top-k subspace then turns by s = safety * de / (sigma_k - sigma_{k+1})
    (Wedin), and a block score l_g = ||E_g^T V_k||_F^2 moves by at most
    2 sqrt(l_g k) s + (k + l_g) s^2 (write V' = V W + V_perp Z with
    ||Z||_F <= sqrt(k) s).  Returned as a bound for the largest score lmax."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    sv = np.linalg.svd(A, compute_uv=False)
    de = u / np.sqrt(3.0) * (np.linalg.norm(A) / np.sqrt(m * n) + sv[0] / np.sqrt(min(m, n)))
    s = safety * de / (sv[k - 1] - sv[k])
    return 2.0 * np.sqrt(lmax * k) * s + (k + lmax) * s * s


def u_bound(C, R, rel_err, u):
    """First-order bound on ||U_gpu - U||_F / ||U||_F for U = C^+ A R^+ computed
    with unit round-off u by a backward-stable least-squares solve on each
    side: u (2 kappa / cos(theta) + kappa^2 tan(theta)) per side (the
    least-squares perturbation theorem, e.g. Golub and Van Loan, Thm. 5.3.1),
    kappa the condition number of C (resp. R), sin(theta) the relative
    residual ||A - CUR||_F / ||A||_F."""
    def kappa(X):
        sv = np.linalg.svd(np.asarray(X, dtype=np.float64), compute_uv=False)
        return sv[0] / sv[-1]
    c = np.sqrt(max(1.0 - rel_err ** 2, 1e-30))
    t = rel_err / c
    return u * sum(2.0 * kp / c + kp * kp * t for kp in (kappa(C), kappa(R)))


def assert_indices_to_first_tie(ref, gpu, p):
    """Block indices equal the oracle's bit for bit up to the first draw whose
    x = u T lies within the score perturbation of an oracle CDF boundary.
    The GPU's prefix sums and total differ from the oracle's by at most the
    L1 norm of the score difference, so a draw farther than twice that from
    every boundary must pick the same block.  Returns the checked draws."""
    out = {}
    for side, u, g in (("col", p.u_col(), p.g_col), ("row", p.u_row(), p.g_row)):
        d1 = float(np.sum(np.abs(np.asarray(gpu[f"{side}_scores"]) - ref[f"{side}_scores"])))
        tol = 2.0 * d1 + 1e-12 * float(np.sum(ref[f"{side}_scores"]))
        n_ok = tie_draws(ref[f"{side}_scores"], u, g, p.replacement, tol)
        assert gpu[f"{side}_idx"][:n_ok] == list(ref[f"{side}_idx"][:n_ok]), side
        out[side] = n_ok
    return out
