"""The paper's Algorithm 1 on the GPU against the oracle's algorithm1()."""
import numpy as np
import pytest

from _gpu_common import device, to_dev, torch  # noqa: F401
import bcur_inputs as bi
import oracle as orc

pytestmark = pytest.mark.gpu


def _case(kind, seed):
    if kind == "lowrank":
        rg = np.random.default_rng(seed)
        A = rg.standard_normal((300, 4)) @ rg.standard_normal((4, 960))
        return A, bi.uniform_blocks(960, 32)
    if kind == "eda_like":  # 24 subjects x 9929 samples, blocks of 120 (Sec. 4.1 shape)
        p = bi.Problem("eda", 24, 9929, k=5, p=0, q=0, col_off=bi.uniform_blocks(9929, 120),
                       row_off=bi.uniform_blocks(24, 24), g_col=10, g_row=1, seed=seed,
                       storage="f64", recipe=dict(kind="ar1_mixture", rank=5, phi=0.95, noise=0.05))
        return p.matrix(), p.col_off
    rg = np.random.default_rng(seed)
    A = rg.standard_normal((512, 16)) @ rg.standard_normal((16, 1024)) + 0.05 * rg.standard_normal((512, 1024))
    return A, bi.uniform_blocks(1024, 64)


@pytest.mark.parametrize("kind,r,g,dtype", [("lowrank", 12, 6, "f64"), ("noisy", 40, 12, "f64"),
                                            ("noisy", 40, 12, "f32"), ("eda_like", 20, 10, "f64")])
def test_alg1_matches_oracle(kind, r, g, dtype):
    import paper_1703_06065_gb300 as pkg

    device()
    A, off = _case(kind, 3)
    if dtype == "f32":
        A = A.astype(np.float32)
    ur, uc = bi.uniforms(r, 5, 3), bi.uniforms(g, 5, 4)
    ref = orc.algorithm1(A, off, r, g, ur, uc)
    out = pkg.alg1(to_dev(A), off, r, g, to_dev(ur), to_dev(uc))
    assert out["row_idx"].cpu().tolist() == ref["row_idx"]
    tol = 1e-9 if dtype == "f64" else 1e-4
    cs = out["col_scores"].cpu().numpy()
    np.testing.assert_allclose(cs, ref["col_scores"], atol=tol * max(ref["col_scores"]))
    assert abs(cs.sum() - ref["rank_R"]) < 1e3 * tol * r
    if dtype == "f64":
        assert out["col_idx"].cpu().tolist() == ref["col_idx"]
        e = out["err"].cpu().numpy()
        assert abs(e[1] - ref["rel"]) <= 1e-3
        assert abs(e[0] - ref["err"]) <= 1e-6 * max(ref["err"], 1e-12 * e[2]) + 1e-9 * e[2]
        U = out["U"].cpu().numpy()
        np.testing.assert_allclose(U, ref["U"], atol=1e-7 * np.abs(ref["U"]).max())
