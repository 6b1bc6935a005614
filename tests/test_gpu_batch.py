"""Batched decompositions (one launch per stage over many uneven matrices):
parity of every item with the FP64 oracle, independence of an item's results
from the rest of the batch, and CUDA-graph replay."""
import numpy as np
import pytest

from _gpu_common import device, to_dev, torch  # noqa: F401
import bcur_inputs as bi
import oracle as orc

pytestmark = pytest.mark.gpu


def _problems():
    """Test-sized members of the biometric recipe (AR(1) series mixed by a
    rank-k loading + 0.05 noise), plus shapes with short last blocks and the
    largest c = r = 512."""
    probs = bi.batched_biometric(6, seed=5, m_range=(256, 768), n_range=(512, 1536),
                                 k_range=(5, 20), blocks=(16, 32, 64, 128))
    extra = [
        bi.Problem("short_last", 300, 700, k=6, p=10, q=2, col_off=bi.uniform_blocks(700, 48),
                   row_off=bi.uniform_blocks(300, 48), g_col=4, g_row=3, seed=11, storage="f32",
                   recipe=dict(kind="ar1_mixture", rank=6, phi=0.95, noise=0.05)),
        bi.Problem("wide_fit", 1024, 1536, k=20, p=10, q=2, col_off=bi.uniform_blocks(1536, 256),
                   row_off=bi.uniform_blocks(1024, 256), g_col=2, g_row=2, seed=12, storage="f32",
                   recipe=dict(kind="ar1_mixture", rank=20, phi=0.95, noise=0.05)),
    ]
    return probs + extra


def _item(p):
    return dict(m=p.m, n=p.n, k=p.k, p=p.p, block=int(p.col_off[1] - p.col_off[0]),
                g_col=p.g_col, g_row=p.g_row)


def _inputs(probs):
    As = [to_dev(p.matrix(), torch.float32) for p in probs]
    oms = [to_dev(p.omega().T, torch.float32) for p in probs]
    ucs = [to_dev(p.u_col()) for p in probs]
    urs = [to_dev(p.u_row()) for p in probs]
    return As, oms, ucs, urs


def _host(o, i):
    return {k: (o[k][i].cpu().numpy().copy() if o[k][i] is not None else None)
            for k in ("col_scores", "row_scores", "col_idx", "row_idx", "U", "err")}


def _run(probs, use_graph=False):
    import paper_1703_06065_gb300 as pkg

    device()
    b = pkg.Batch([_item(p) for p in probs], q=2)
    ins = _inputs(probs)
    o = b.run(*ins, use_graph=use_graph)
    b.sync_status()
    return b, ins, [_host(o, i) for i in range(len(probs))]


def _tie_free_draws(ref_scores, gpu_scores, u, g):
    """Draws before the first one whose x = u T lies within the CDF
    perturbation sum |l_gpu - l_orc| (+ rounding) of an oracle boundary."""
    tol = float(np.sum(np.abs(np.asarray(gpu_scores) - np.asarray(ref_scores)))) + 1e-12
    l = [float(v) for v in ref_scores]
    rem = [True] * len(l)
    for t in range(g):
        T = sum(v for v, r in zip(l, rem) if r)
        x = float(u[t]) * T
        S, pick = 0.0, -1
        for j, v in enumerate(l):
            if not rem[j]:
                continue
            S += v
            if abs(S - x) <= tol:
                return t
            if pick < 0 and S > x:
                pick = j
        if pick < 0:
            return t
        rem[pick] = False
    return g


def test_batch_matches_oracle_per_item():
    probs = _problems()
    b, ins, res = _run(probs)
    for p, r in zip(probs, res):
        A = p.matrix().astype(np.float64)
        ref = orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row, p.omega(),
                            p.u_col(), p.u_row())
        # scores: BF16 sketch, re-orthonormalised in FP32/FP64 after every product
        for side in ("col", "row"):
            d = np.max(np.abs(r[f"{side}_scores"] - ref[f"{side}_scores"]))
            assert d <= 2e-2 * np.max(ref[f"{side}_scores"]), (p.name, side, d)
            assert abs(np.sum(r[f"{side}_scores"]) - p.k) <= 2e-2 * p.k, (p.name, side)
        # indices: bit-exact up to the first draw the score perturbation could flip
        for side, u, g in (("col", p.u_col(), p.g_col), ("row", p.u_row(), p.g_row)):
            n_ok = _tie_free_draws(ref[f"{side}_scores"], r[f"{side}_scores"], u, g)
            assert list(r[f"{side}_idx"][:n_ok]) == list(ref[f"{side}_idx"][:n_ok]), (p.name, side)
        # the accuracy gate against the oracle's own decomposition
        assert abs(r["err"][1] - ref["rel"]) <= 1e-3, (p.name, r["err"][1], ref["rel"])
        # the fit on the GPU's own blocks against the oracle's fit on them
        C = orc.gather_columns(A, p.col_off, list(r["col_idx"]))
        R = orc.gather_rows(A, p.row_off, list(r["row_idx"]))
        U = orc.fit_u(A, C, R)
        err, rel = orc.residual(A, C, U, R)
        # one BF16 term in the residual reconstruction adds about
        # u^2 (1 - e^2) / (3 e) to e (u = 2^-8); pairs when that is too coarse
        nA = np.linalg.norm(A)
        model = 0.00390625 ** 2 * (1 - rel * rel) / (3 * rel) if rel > 0 else 1.0
        assert abs(r["err"][0] - err) <= 5 * model * nA + 1e-4 * err + 1e-6 * nA, p.name
        assert abs(r["err"][2] - np.linalg.norm(A)) <= 1e-6 * np.linalg.norm(A)
        c, rr = C.shape[1], R.shape[0]
        Ug = r["U"][:c, :rr].astype(np.float64)
        cur_g = C @ Ug @ R
        cur_o = C @ U @ R
        assert np.linalg.norm(cur_g - cur_o) <= 1e-3 * np.linalg.norm(A), p.name
        assert np.all(r["U"][c:, :] == 0) and np.all(r["U"][:, rr:] == 0)


def test_item_results_do_not_depend_on_the_batch():
    probs = _problems()
    _, _, res_all = _run(probs)
    for i in (0, len(probs) - 1, 3):
        _, _, res_one = _run([probs[i]])
        for k, v in res_one[0].items():
            np.testing.assert_array_equal(v, res_all[i][k], err_msg=f"{probs[i].name} {k}")
    # a different mix (reversed order, one item left out) gives the same bits
    sub = list(reversed(probs[1:]))
    _, _, res_sub = _run(sub)
    for j, p in enumerate(sub):
        i = probs.index(p)
        for k, v in res_sub[j].items():
            np.testing.assert_array_equal(v, res_all[i][k], err_msg=f"{p.name} {k}")


def test_graph_replay_matches_eager_run():
    import paper_1703_06065_gb300 as pkg

    probs = _problems()[:4]
    device()
    b = pkg.Batch([_item(p) for p in probs], q=2)
    As, oms, ucs, urs = _inputs(probs)
    eager = b.run(As, oms, ucs, urs)
    b.sync_status()
    ref = [_host(eager, i) for i in range(len(probs))]
    for _ in range(2):
        o = b.run(As, oms, ucs, urs, use_graph=True)
        b.sync_status()
        for i in range(len(probs)):
            for k, v in _host(o, i).items():
                np.testing.assert_array_equal(v, ref[i][k], err_msg=k)
    # new inputs through the same graph: uniforms swapped between the sides
    o = b.run(As, oms, urs, ucs, use_graph=True) if all(
        u.numel() == v.numel() for u, v in zip(ucs, urs)) else None
    if o is not None:
        b.sync_status()
        b2 = pkg.Batch([_item(p) for p in probs], q=2)
        e2 = b2.run(As, oms, urs, ucs)
        b2.sync_status()
        for i in range(len(probs)):
            for k, v in _host(o, i).items():
                np.testing.assert_array_equal(v, _host(e2, i)[k], err_msg=k)
    assert b.launches_per_run > 10


def test_small_error_items_are_refined():
    """Noise-free (exactly rank-k) members mixed with noisy ones: the items
    whose one-term residual is too coarse are recomputed with BF16 pairs, the
    others keep the one-term value."""
    probs = []
    for i, noise in enumerate((0.0, 0.05, 0.0)):
        probs.append(bi.Problem(f"mix{i}", 512, 768, k=6, p=10, q=2,
                                col_off=bi.uniform_blocks(768, 32),
                                row_off=bi.uniform_blocks(512, 32), g_col=3, g_row=3,
                                seed=40 + i, storage="f32",
                                recipe=dict(kind="ar1_mixture", rank=6, phi=0.95, noise=noise)))
    _, _, res = _run(probs)
    for p, r in zip(probs, res):
        A = p.matrix().astype(np.float64)
        C = orc.gather_columns(A, p.col_off, list(r["col_idx"]))
        R = orc.gather_rows(A, p.row_off, list(r["row_idx"]))
        err, rel = orc.residual(A, C, orc.fit_u(A, C, R), R)
        assert abs(r["err"][1] - rel) <= 1e-3, (p.name, r["err"][1], rel)
        if p.recipe["noise"] == 0.0:
            assert r["err"][1] < 5e-4, (p.name, r["err"])  # one term: about 3e-3


def test_wide_panels_for_large_k():
    """Items with l = k + p > 64 run with 128-row panels; parity with the
    oracle and independence from the batch as for the 64-row form."""
    probs = [
        bi.Problem("k60", 1024, 2048, k=60, p=10, q=2, col_off=bi.uniform_blocks(2048, 128),
                   row_off=bi.uniform_blocks(1024, 128), g_col=2, g_row=2, seed=61, storage="f32",
                   recipe=dict(kind="ar1_mixture", rank=60, phi=0.95, noise=0.05)),
        bi.Problem("k8", 768, 1280, k=8, p=10, q=2, col_off=bi.uniform_blocks(1280, 64),
                   row_off=bi.uniform_blocks(768, 64), g_col=2, g_row=2, seed=62, storage="f32",
                   recipe=dict(kind="ar1_mixture", rank=8, phi=0.95, noise=0.05)),
    ]
    _, _, res = _run(probs)
    for p, r in zip(probs, res):
        A = p.matrix().astype(np.float64)
        ref = orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row, p.omega(),
                            p.u_col(), p.u_row())
        for side in ("col", "row"):
            d = np.max(np.abs(r[f"{side}_scores"] - ref[f"{side}_scores"]))
            assert d <= 2e-2 * np.max(ref[f"{side}_scores"]), (p.name, side, d)
        assert abs(r["err"][1] - ref["rel"]) <= 1e-3, (p.name, r["err"][1], ref["rel"])
    _, _, alone = _run([probs[0]])
    for k, v in alone[0].items():
        np.testing.assert_array_equal(v, res[0][k], err_msg=k)


def test_nonfinite_item_is_reported():
    import paper_1703_06065_gb300 as pkg

    probs = _problems()[:2]
    device()
    b = pkg.Batch([_item(p) for p in probs], q=1)
    As, oms, ucs, urs = _inputs(probs)
    As[1][3, 5] = float("nan")
    b.run(As, oms, ucs, urs)
    with pytest.raises(pkg.BcurError) as e:
        b.sync_status()
    assert e.value.status == 5


def test_autotuned_tile_widths_are_measured_once_and_cached(tmp_path, monkeypatch):
    """The autotuner times each GEMM shape class once and keeps its choice in
    the process table and in the JSON cache file; a second plan of the same
    shapes measures nothing and gives bit for bit the same results."""
    import json

    import paper_1703_06065_gb300 as pkg

    device()
    L = pkg.load()
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("BCUR_AUTOTUNE_CACHE", str(cache))
    # shapes no other test uses, so that their classes are new to the table
    probs = [bi.Problem(f"tune_{i}", m, n, k=k, p=10, q=2, col_off=bi.uniform_blocks(n, s),
                        row_off=bi.uniform_blocks(m, s), g_col=g, g_row=g, seed=40 + i,
                        storage="f32", recipe=dict(kind="ar1_mixture", rank=k, phi=0.95,
                                                   noise=0.05))
             for i, (m, n, k, s, g) in enumerate([(2944, 5120, 17, 160, 3), (1408, 9216, 9, 96, 4)])]
    n0 = L.bcur_autotune_measured()
    b1, ins, r1 = _run(probs)
    n1 = L.bcur_autotune_measured()
    assert n1 > n0
    table = json.loads(cache.read_text())
    assert table and all(v in (64, 128, 256) for v in table.values())
    assert any(k.startswith("w|") for k in table) and any(k.startswith("sketch_y|") for k in table)
    b2 = pkg.Batch([_item(p) for p in probs], q=2)
    assert L.bcur_autotune_measured() == n1           # every class came from the table
    o2 = b2.run(*ins)
    b2.sync_status()
    r2 = [_host(o2, i) for i in range(len(probs))]
    for a, b in zip(r1, r2):
        for key in a:
            if a[key] is not None:
                np.testing.assert_array_equal(a[key], b[key])


def test_worst_conditioned_members_of_the_batch_meet_the_gate():
    """The members of the 512-matrix batch whose C or R is worst conditioned
    (kappa from 410 to 860; 105 and 325 are 512-row members at the two-block
    minimum, c = m/2): batched together, each must meet the 1e-3 error gate
    against the FP64 oracle, with the oracle's blocks up to the first tie."""
    import paper_1703_06065_gb300 as pkg

    device()
    allp = bi.batched_biometric(512, seed=3)
    picks = [allp[i] for i in (314, 418, 65, 387, 105, 325)]
    b = pkg.Batch([_item(p) for p in picks], q=2)
    As = [p.matrix_device(torch.device("cuda")) for p in picks]
    oms = [to_dev(p.omega().T, torch.float32) for p in picks]
    o = b.run(As, oms, [to_dev(p.u_col()) for p in picks], [to_dev(p.u_row()) for p in picks])
    b.sync_status()
    for i, p in enumerate(picks):
        A = As[i].double().cpu().numpy()
        ref = orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row, p.omega(),
                            p.u_col(), p.u_row())
        e = float(o["err"][i][1].item())
        assert abs(e - ref["rel"]) <= 1e-3, (p.name, e, ref["rel"])
        for side, u, g in (("col", p.u_col(), p.g_col), ("row", p.u_row(), p.g_row)):
            n_ok = _tie_free_draws(ref[f"{side}_scores"], o[f"{side}_scores"][i].cpu().numpy(), u, g)
            assert o[f"{side}_idx"][i].cpu().tolist()[:n_ok] == list(ref[f"{side}_idx"][:n_ok])


def test_adaptive_fit_batch():
    """fit_prec "bf16x3a": each item's core products and residual start with
    one BF16 term and are redone with three only where the item's one-term
    residual is too coarse (e < 0.031).  The biometric members (e near 0.05
    to 0.1) keep one term and meet the 1e-3 error gate, with CUR within what
    the least-squares bound of one term implies; an exactly rank-6 member in
    the same batch takes three terms and then equals, bit for bit, the same
    item decomposed by a split-BF16 batch; and every item's results are the
    same alone as in the batch."""
    import paper_1703_06065_gb300 as pkg
    from _gpu_common import UNIT, u_bound

    device()
    probs = _problems()[:4] + [
        bi.Problem("rank6_exact", 512, 768, k=6, p=10, q=2, col_off=bi.uniform_blocks(768, 64),
                   row_off=bi.uniform_blocks(512, 64), g_col=3, g_row=3, seed=14, storage="f32",
                   recipe=dict(kind="small_lowrank", rank=6, noise=0.0))]
    ins = _inputs(probs)
    ba = pkg.Batch([_item(p) for p in probs], q=2, fit_prec="bf16x3a")
    oa = ba.run(*ins)
    ba.sync_status()
    ra = [_host(oa, i) for i in range(len(probs))]
    terms = ba.fit_terms()
    assert terms[-1] == 3, terms
    for t, r in zip(terms, ra):   # e > 0.035: the one-term residual cannot ask for pairs
        if r["err"][1] > 0.035:
            assert t == 1, (terms, [x["err"][1] for x in ra])
    for p, r in zip(probs, ra):
        A = p.matrix().astype(np.float64)
        ref = orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row, p.omega(),
                            p.u_col(), p.u_row())
        assert abs(r["err"][1] - ref["rel"]) <= 1e-3, (p.name, r["err"][1], ref["rel"])
        C = orc.gather_columns(A, p.col_off, list(r["col_idx"]))
        R = orc.gather_rows(A, p.row_off, list(r["row_idx"]))
        U = orc.fit_u(A, C, R)
        e_o = orc.residual(A, C, U, R)[1]
        c, rr = C.shape[1], R.shape[0]
        Ug = r["U"][:c, :rr].astype(np.float64)
        ub = u_bound(C, R, e_o, UNIT["bf16"])
        bound = np.linalg.norm(C, 2) * np.linalg.norm(R, 2) * ub * np.linalg.norm(U)
        assert np.linalg.norm(C @ Ug @ R - C @ U @ R) <= bound, p.name
    b3 = pkg.Batch([_item(probs[-1])], q=2)
    o3 = b3.run(*[x[-1:] for x in ins])
    b3.sync_status()
    r3 = _host(o3, 0)
    for key in ("U", "err", "col_idx", "row_idx"):
        np.testing.assert_array_equal(ra[-1][key], r3[key], err_msg=key)
    for i in (0, 2):
        b1 = pkg.Batch([_item(probs[i])], q=2, fit_prec="bf16x3a")
        o1 = b1.run(*[x[i:i + 1] for x in ins])
        b1.sync_status()
        r1 = _host(o1, 0)
        for key in ("U", "err", "col_scores", "col_idx"):
            np.testing.assert_array_equal(ra[i][key], r1[key], err_msg=key)
