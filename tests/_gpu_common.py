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
