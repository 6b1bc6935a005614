"""Diagnostics of Sec. 3.2 on the GPU: block stable rank terms and incoherence,
fed the same factors as the oracle."""
import numpy as np
import pytest

from _gpu_common import device, run_problem, to_dev, torch  # noqa: F401
import bcur_inputs as bi
import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,rtol", [("f64", 1e-9), ("f32", 2e-5)])
@pytest.mark.parametrize("k,h,sizes", [(10, 1024, [32] * 32), (50, 4096, [512] * 8),
                                       (7, 300, [1, 50, 49, 200]), (64, 2000, [1000, 1000])])
def test_block_stable_rank_kernel(dtype, rtol, k, h, sizes):
    import paper_1703_06065_gb300 as pkg

    device()
    rg = np.random.default_rng(k + h)
    F = np.linalg.qr(rg.standard_normal((h, k)))[0]
    F[: sizes[0]] *= 3.0  # make the blocks unequal
    if dtype == "f32":
        F = F.astype(np.float32)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    want = orc.block_stable_rank_terms(F.astype(np.float64), off)
    got = pkg.block_stable_rank(to_dev(np.ascontiguousarray(F.T)), to_dev(off)).cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=rtol)
    sz = np.diff(off)
    assert np.all(got >= 1 - 1e-9) and np.all(got <= np.minimum(sz, k) + 1e-6)


def test_rank_one_block_has_stable_rank_one():
    import paper_1703_06065_gb300 as pkg

    device()
    F = np.zeros((8, 2))
    F[0:2, 0] = [0.6, 0.8]
    F[2:8, 1] = 1 / np.sqrt(6)
    got = pkg.block_stable_rank(to_dev(np.ascontiguousarray(F.T)), to_dev(np.array([0, 2, 8]))).cpu()
    np.testing.assert_allclose(got.numpy(), [1.0, 1.0], rtol=1e-12)


def test_plan_factors_give_the_oracle_diagnostics():
    import paper_1703_06065_gb300 as pkg

    p = bi.plain_fp64_512x1024()
    ref, gpu, plan = run_problem(p)
    Vt, Ut, sig = plan.factors()
    alpha = pkg.block_stable_rank(Vt, to_dev(p.col_off)).cpu().numpy()
    np.testing.assert_allclose(alpha, orc.block_stable_rank_terms(ref["V_k"], p.col_off), rtol=1e-8)
    mu = float(pkg.incoherence(Ut).cpu())
    assert abs(mu - orc.incoherence(ref["U_k"])) <= 1e-8 * mu
    np.testing.assert_allclose(sig.cpu().numpy(), ref["sigma"], rtol=1e-10)
