"""Per-kernel parity: each library kernel and the oracle get the same inputs."""
import numpy as np
import pytest

from _gpu_common import device, to_dev, torch  # noqa: F401
import bcur_inputs as bi
import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k,h,sizes", [
    (10, 1024, [32] * 32),
    (50, 4000, [512] * 7 + [416]),          # ragged tail block
    (1, 77, [1] * 77),                      # block size 1: column leverage scores
    (7, 300, [300]),                        # single block
    (64, 5000, [1, 2, 3, 500, 4494]),       # uneven sizes
])
def test_block_scores_kernel(dtype, k, h, sizes):
    import paper_1703_06065_gb300 as pkg

    device()
    rg = np.random.default_rng(k * 1000 + h)
    F = rg.standard_normal((h, k)) / np.sqrt(h)
    if dtype == "f32":
        F = F.astype(np.float32)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    want = orc.block_scores(F.astype(np.float64), off)
    got = pkg.block_scores(to_dev(F.T), to_dev(off)).cpu().numpy()
    # Both sides square the same stored values in FP64; only the order of
    # the FP64 additions differs.
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)


@pytest.mark.parametrize("replacement", [False, True])
def test_sample_kernel_bit_exact(replacement):
    import paper_1703_06065_gb300 as pkg

    device()
    rg = np.random.default_rng(5 + replacement)
    for trial in range(40):
        G = int(rg.integers(1, 300))
        sc = rg.random(G) ** 3
        if trial % 5 == 0:
            sc[rg.random(G) < 0.4] = 0.0           # zero-score blocks
        if trial == 7:
            sc[:] = 0.0                            # all zero: lowest index first
        g = int(rg.integers(1, G + 1)) if not replacement else int(rg.integers(1, 2 * G + 2))
        u = bi.uniforms(g, trial, 9 + replacement)
        want_i, want_p = orc.sample_blocks(sc, u, g, replacement)
        idx, prob = pkg.sample_blocks(to_dev(sc), to_dev(u), g, replacement)
        assert idx.cpu().tolist() == want_i
        assert prob.cpu().numpy().tolist() == want_p


def test_sample_kernel_hand_cases():
    import paper_1703_06065_gb300 as pkg

    device()
    sc = to_dev(np.array([1.0, 2.0, 3.0, 4.0]))
    idx, _ = pkg.sample_blocks(sc, to_dev(np.array([0.95, 0.95, 0.0])), 3, False)
    assert idx.cpu().tolist() == [3, 2, 0]
    idx, _ = pkg.sample_blocks(sc, to_dev(np.array([0.1])), 1, True)
    assert idx.cpu().tolist() == [1]   # x = 1.0 is not > 1.0


@pytest.mark.parametrize("dtype,prec", [("f64", "f64"), ("f32", "f32")])
@pytest.mark.parametrize("m,n,r", [(300, 500, 40), (1000, 777, 129), (64, 64, 1), (517, 263, 0)])
def test_residual_kernel(dtype, prec, m, n, r):
    import paper_1703_06065_gb300 as pkg

    device()
    rg = np.random.default_rng(m + n + r)
    X = rg.standard_normal((m, n))
    P = rg.standard_normal((m, r)) / np.sqrt(max(r, 1))
    Q = rg.standard_normal((r, n))
    if dtype == "f32":
        X, P, Q = X.astype(np.float32), P.astype(np.float32), Q.astype(np.float32)
    X64, P64, Q64 = X.astype(np.float64), P.astype(np.float64), Q.astype(np.float64)
    want_e2 = float(np.sum((X64 - P64 @ Q64) ** 2))
    want_x2 = float(np.sum(X64 ** 2))
    out = pkg.residual(to_dev(X), to_dev(P), to_dev(Q), prec).cpu().numpy()
    # FP64: rounding of r-term dot products; FP32: u32 * sqrt(r) per entry.
    tol = 1e-11 if dtype == "f64" else 2e-5
    assert abs(out[0] - want_e2) <= tol * want_e2
    assert abs(out[1] - want_x2) <= 1e-12 * want_x2
    # bit-identical on repeat (fixed reduction order)
    out2 = pkg.residual(to_dev(X), to_dev(P), to_dev(Q), prec).cpu().numpy()
    assert out2.tobytes() == out.tobytes()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("tA,tB", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_gemm_simt(dtype, tA, tB):
    import paper_1703_06065_gb300 as pkg

    device()
    rg = np.random.default_rng(11 + tA * 2 + tB)
    M, N, K = 193, 301, 259
    A = rg.standard_normal((K, M) if tA else (M, K))
    B = rg.standard_normal((N, K) if tB else (K, N))
    if dtype == "f32":
        A, B = A.astype(np.float32), B.astype(np.float32)
    want = (A.T if tA else A).astype(np.float64) @ (B.T if tB else B).astype(np.float64)
    got = pkg.gemm(to_dev(A), to_dev(B), bool(tA), bool(tB), dtype).double().cpu().numpy()
    tol = 1e-12 if dtype == "f64" else 1e-5
    assert np.max(np.abs(got - want)) <= tol * np.sqrt(K) * np.max(np.abs(want))
