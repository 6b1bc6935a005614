"""Serving loop: requests arriving over time, continuous batching on several
streams, admission by HBM footprint.  Every result must be the same whether
the request ran alone or in the mix, and must pass the accuracy gate against
the FP64 oracle on the same inputs."""
import numpy as np
import pytest

from _gpu_common import device, torch  # noqa: F401
import bcur_inputs as bi
import oracle as orc

pytestmark = pytest.mark.gpu

SMALL = dict(m_range=(256, 1024), n_range=(512, 2048), k_range=(5, 20), blocks=(16, 32, 64, 128))


def _requests(rate=400.0, duration=0.4, heavy_frac=0.1):
    return bi.serving_requests(rate, duration, seed=9, heavy_frac=heavy_frac, heavy_n=2048,
                               **SMALL)


def _server(**kw):
    from paper_1703_06065_gb300 import serve

    device()
    kw.setdefault("hbm_budget", 8e9)
    kw.setdefault("draw", bi.generators.request_inputs_device)
    return serve.Server(**kw)


def test_serving_alone_and_in_the_mix_agree():
    from paper_1703_06065_gb300 import serve

    reqs = _requests()
    assert any(r.heavy for r in reqs) and sum(not r.heavy for r in reqs) > 20
    srv = _server(lanes=3, max_batch=32, keep_u=True)
    done = srv.run(reqs, realtime=True, timeout=120.0)
    assert any(k == "heavy" for k, *_ in srv.jobs)
    assert len(done) == len(reqs)
    stats = serve.latency_stats(done)
    assert stats["p50_ms"] > 0 and stats["p99_ms"] >= stats["p50_ms"]
    by_id = {q.r.rid: q for q in done}
    # several light groups ran
    picks = [r for r in reqs if not r.heavy][:3] + [r for r in reqs if r.heavy][:1]
    for r in picks:
        alone = _server(lanes=1, max_batch=32, keep_u=True).run([r], realtime=False)[0]
        mixed = by_id[r.rid]
        for k in ("err", "col_idx", "row_idx", "U"):
            np.testing.assert_array_equal(alone.result[k], mixed.result[k],
                                          err_msg=f"{r.problem.name} {k}")


def test_serving_matches_the_oracle():
    reqs = _requests(rate=300.0, duration=0.2)
    sample = {r.rid for r in reqs[:: max(1, len(reqs) // 4)]}
    srv = _server(lanes=2, max_batch=16, keep_inputs=lambda r: r.rid in sample)
    done = srv.run(reqs, realtime=True, timeout=120.0)
    checked = 0
    for q in done:
        if q.r.rid not in sample:
            continue
        p = q.r.problem
        A, om, uc, ur = q.result["inputs"]
        ref = orc.block_cur(A.astype(np.float64), p.col_off, p.row_off, p.k, p.q, p.g_col,
                            p.g_row, om.T.astype(np.float64), uc, ur)
        assert abs(q.result["err"][1] - ref["rel"]) <= 1e-3, (p.name, q.result["err"], ref["rel"])
        checked += 1
    assert checked >= 3


def test_admission_respects_the_budget():
    from paper_1703_06065_gb300 import serve

    reqs = _requests(rate=500.0, duration=0.2, heavy_frac=0.0)
    srv = _server(lanes=2, max_batch=8)
    fps = [srv._footprint(serve._Req(r)) for r in reqs]
    # a budget of two requests: never more than that in flight, all still served
    srv.budget = 2.0 * max(fps)
    peak = [0.0]
    orig = srv._admit

    def admit(q):
        ok = orig(q)
        peak[0] = max(peak[0], srv.in_use + (q.bytes if ok else 0.0))
        return ok

    srv._admit = admit
    done = srv.run(reqs, realtime=False, timeout=120.0)
    assert len(done) == len(reqs)
    assert peak[0] <= srv.budget + 1e-6
    assert srv.in_use == pytest.approx(0.0, abs=1e-3)


def test_heavy_requests_batched_path_agrees_with_the_plan_path():
    """Heavy requests are grouped into batches by default; with heavy_plan=True
    each heavy lane runs them one at a time on a single-matrix plan.  Both
    meet the oracle's error gate on the same inputs."""
    reqs = [r for r in _requests(rate=400.0, duration=0.6, heavy_frac=0.5) if r.heavy][:2]
    assert reqs
    keep = lambda r: True  # noqa: E731
    a = _server(lanes=1, max_batch=8, keep_inputs=keep, heavy_plan=True).run(reqs,
                                                                             realtime=False)
    b = _server(lanes=1, max_batch=8, keep_inputs=keep).run(reqs, realtime=False)
    for qa, qb in zip(sorted(a, key=lambda q: q.r.rid), sorted(b, key=lambda q: q.r.rid)):
        p = qa.r.problem
        A, om, uc, ur = qa.result["inputs"]
        ref = orc.block_cur(A.astype(np.float64), p.col_off, p.row_off, p.k, p.q, p.g_col,
                            p.g_row, om.T.astype(np.float64), uc, ur)
        for q in (qa, qb):
            assert abs(q.result["err"][1] - ref["rel"]) <= 1e-3
