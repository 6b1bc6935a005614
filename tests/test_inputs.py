"""The seeded input generators (no GPU): the chunked AR(1) recurrence of the
serving workload's device generator against the sequential definition."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from bcur_inputs import generators as G  # noqa: E402


@pytest.mark.parametrize("n,chunk", [(1, 128), (127, 128), (128, 128), (1000, 128), (777, 32)])
def test_chunked_ar1_series_matches_the_recurrence(n, chunk):
    """x_0 = e_0, x_t = phi x_{t-1} + sqrt(1 - phi^2) e_t, evaluated step by
    step in FP64, equals the chunked form (FP32) to FP32 rounding, for lengths
    that are and are not multiples of the chunk."""
    phi = 0.95
    g = torch.Generator().manual_seed(3)
    e = torch.randn(5, n, generator=g)
    x = G.ar1_series_chunked(e, phi, chunk).double().numpy()
    en = e.double().numpy()
    ref = np.empty_like(en)
    ref[:, 0] = en[:, 0]
    c = math.sqrt(1.0 - phi * phi)
    for t in range(1, n):
        ref[:, t] = phi * ref[:, t - 1] + c * en[:, t]
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-5 * max(1.0, np.abs(ref).max()))


def test_chunked_ar1_series_is_stationary():
    """Unit stationary variance: the rows' empirical variance is near 1."""
    g = torch.Generator().manual_seed(4)
    x = G.ar1_series_chunked(torch.randn(64, 20000, generator=g), 0.95)
    v = float(x.var())
    assert abs(v - 1.0) < 0.05, v
