"""Rank-k truncation U_k (Sec. 4.1) and boosting (Sec. 3.3) on the GPU."""
import numpy as np
import pytest

from _gpu_common import device, run_problem, to_dev, torch  # noqa: F401
import bcur_inputs as bi
import oracle as orc

pytestmark = pytest.mark.gpu


def test_truncated_u_error_matches_oracle():
    p = bi.plain_fp64_512x1024()
    ref, gpu, plan = run_problem(p)
    A = p.matrix()
    om_u = bi.rademacher(plan.r_max, p.l, 17)
    Uk, out = plan.truncate(to_dev(A), p.k, to_dev(np.ascontiguousarray(om_u.T)))
    e = out.cpu().numpy()
    Uk_orc = orc.truncate_rank(ref["U"], p.k)
    want, want_rel = orc.residual(A, ref["C"], Uk_orc, ref["R"])
    assert abs(e[0] - want) <= 1e-6 * want
    assert abs(e[1] - want_rel) <= 1e-3
    Ug = Uk.cpu().numpy()
    assert np.linalg.matrix_rank(Ug, tol=1e-8 * np.abs(Uk_orc).max()) == p.k
    # C and R are ill-conditioned here (noise directions), so the pseudo-inverses
    # make U's leading directions noise and its spectrum has no gap at k: U_k is
    # not unique enough to compare entrywise.  It must still be near-optimal in
    # the Eckart-Young sense: ||U - U_k||_F within 5% of the exact rank-k tail.
    sv = np.linalg.svd(ref["U"], compute_uv=False)
    tail = np.sqrt(np.sum(sv[p.k:] ** 2))
    assert np.linalg.norm(ref["U"] - Ug) <= 1.05 * tail
    # a rank-k CUR cannot beat the best rank-k approximation
    assert e[0] >= orc.tail_norm(A, p.k) * (1 - 1e-12)


def test_boosting_keeps_the_smallest_error():
    import paper_1703_06065_gb300 as pkg

    dev = device()
    p = bi.plain_fp64_512x1024()
    A = p.matrix()
    plan = pkg.Plan(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row, dtype="f64")
    seeds = [11, 12, 13]
    oms = [to_dev(np.ascontiguousarray(bi.rademacher(p.n, p.l, sd).T)) for sd in seeds]
    ucs = [to_dev(bi.uniforms(p.g_col, sd, 3)) for sd in seeds]
    urs = [to_dev(bi.uniforms(p.g_row, sd, 4)) for sd in seeds]
    best, i = pkg.boosted(plan, to_dev(A), oms, ucs, urs)
    errs = []
    for sd in seeds:
        r = orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row,
                          bi.rademacher(p.n, p.l, sd), bi.uniforms(p.g_col, sd, 3),
                          bi.uniforms(p.g_row, sd, 4))
        errs.append(r["err"])
    assert i == int(np.argmin(errs))
    assert abs(float(best["err"][0]) - min(errs)) <= 1e-9 * min(errs)
