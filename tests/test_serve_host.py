"""Host logic of the serving loop (no GPU): the first-fit arena that holds
every admitted matrix and batch workspace, and the latency summary."""
import types

import numpy as np
import pytest

pytest.importorskip("torch")

from paper_1703_06065_gb300 import serve  # noqa: E402


def _check_free_list(ar):
    """Sorted, 256-aligned, inside the buffer, and fully merged."""
    prev_end = -1
    for off, sz in ar.free:
        assert off % 256 == 0 and sz % 256 == 0 and sz > 0
        assert off > prev_end, ar.free          # strictly after (and not touching) the last one
        prev_end = off + sz
    assert prev_end <= ar.size


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_arena_first_fit_against_a_byte_map(seed):
    """A seeded sequence of allocations and releases against a byte-level
    model: every allocation is 256-aligned, inside the buffer, disjoint from
    every live one and is the lowest free offset that fits (first fit);
    refusals happen only when no free run of that size exists; after the
    last release the free list is the whole buffer again."""
    g = np.random.default_rng(seed)
    ar = serve._Arena(64 * 1024, "cpu")
    used = np.zeros(ar.size // 256, dtype=bool)   # one flag per 256-byte unit
    live = {}
    for step in range(600):
        if live and (g.random() < 0.45 or len(live) > 40):
            off = list(live)[int(g.integers(len(live)))]
            n = live.pop(off)
            ar.release(off, n)
            used[off // 256:(off + (n + 255) // 256 * 256) // 256] = False
        else:
            n = int(g.integers(1, 6000))
            units = (n + 255) // 256
            # the model's first fit: lowest start of a free run of `units`
            want = None
            run = 0
            for i, u in enumerate(used):
                run = 0 if u else run + 1
                if run == units:
                    want = (i - units + 1) * 256
                    break
            off = ar.alloc(n)
            assert off == want, (step, off, want)
            if off is not None:
                assert not used[off // 256:off // 256 + units].any()
                used[off // 256:off // 256 + units] = True
                live[off] = n
        _check_free_list(ar)
        # the free list describes exactly the unused units
        model_free = np.ones_like(used)
        for o, s in ar.free:
            model_free[o // 256:(o + s) // 256] = False
        assert np.array_equal(model_free, used)
    for off, n in list(live.items()):
        ar.release(off, n)
    assert ar.free == [(0, ar.size)]


def test_arena_merges_both_neighbours():
    ar = serve._Arena(4096, "cpu")
    a, b, c = ar.alloc(1000), ar.alloc(256), ar.alloc(300)
    assert (a, b, c) == (0, 1024, 1280)
    ar.release(a, 1000)
    ar.release(c, 300)
    assert ar.free == [(0, 1024), (1280, 4096 - 1280)]
    ar.release(b, 256)                         # joins left and right
    assert ar.free == [(0, 4096)]
    assert ar.alloc(4097) is None and ar.alloc(4096) == 0


def test_latency_stats():
    """Latency = completion - arrival; decompositions/s over first arrival to
    last completion."""
    def req(arrival, done):
        q = types.SimpleNamespace(r=types.SimpleNamespace(arrival=arrival), t_done=done)
        return q

    done = [req(0.0, 0.010), req(0.5, 0.530), req(1.0, 1.004), req(1.5, 2.0)]
    st = serve.latency_stats(done)
    lat = np.array([0.010, 0.030, 0.004, 0.5])
    assert st["requests"] == 4
    assert st["p50_ms"] == pytest.approx(np.percentile(lat, 50) * 1e3)
    assert st["p99_ms"] == pytest.approx(np.percentile(lat, 99) * 1e3)
    assert st["max_ms"] == pytest.approx(500.0)
    assert st["mean_ms"] == pytest.approx(lat.mean() * 1e3)
    assert st["decomps_per_s"] == pytest.approx(4 / 2.0)
