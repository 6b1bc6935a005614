"""The allocation-free residual entry point (bcur_residual_noalloc).

It exists for callers that may not allocate device memory -- code whose GPU
memory is all owned by another framework's pool, request loops that must not
call cudaMalloc/cudaFree, plug-ins handed only input and output pointers.
These tests call it through the C ABI and check it against the ordinary
bcur_residual (which takes a caller-allocated workspace), twice in a row,
since every call reuses the same built-in scratch array.  They cover every
kernel that can serve it: the FP64 and FP32 CUDA-core kernels, the FP32 call
with a tensor-core precision that falls back to the CUDA cores (TF32 cannot
read the row-major Q), and the tensor-core kernel on BF16 P and Q.  The file
is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from _gpu_common import device, to_dev, torch  # noqa: F401

pytestmark = pytest.mark.gpu


def _call(L, X, ldx, P, ldp, Q, ldq, m, n, r, dtype_code, prec_code, out, stream):
    return L.bcur_residual_noalloc(
        ctypes.c_void_p(X.data_ptr()), ldx, ctypes.c_void_p(P.data_ptr() if r else 0), ldp,
        ctypes.c_void_p(Q.data_ptr() if r else 0), ldq, m, n, r, dtype_code, prec_code,
        ctypes.c_void_p(out.data_ptr()), stream)


def _check_twice(L, pkg, want, args, tol):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):  # the second call reuses the scratch the first one left behind
        out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        st = _call(L, *args, out, stream)
        assert st == 0, pkg._lib.STATUS.get(st)
        got = out.cpu().numpy()
        assert abs(got[0] - want[0]) <= tol * want[0], (got, want)
        assert abs(got[1] - want[1]) <= 1e-12 * want[1]


@pytest.mark.parametrize("dtype,prec,tol", [("f64", "f64", 1e-11), ("f32", "f32", 2e-5),
                                            ("f32", "tf32", 2e-5)])
@pytest.mark.parametrize("m,n,r", [(300, 500, 40), (1000, 777, 129)])
def test_noalloc_matches_workspace_residual(dtype, prec, tol, m, n, r):
    import paper_1703_06065_gb300 as pkg
    from paper_1703_06065_gb300 import PREC

    device()
    L = pkg.load()
    rg = np.random.default_rng(m * 7 + r)
    X = rg.standard_normal((m, n))
    P = rg.standard_normal((m, r)) / np.sqrt(r)
    Q = rg.standard_normal((r, n))
    if dtype == "f32":
        X, P, Q = X.astype(np.float32), P.astype(np.float32), Q.astype(np.float32)
    Xd, Pd, Qd = to_dev(X), to_dev(P), to_dev(Q)
    want = pkg.residual(Xd, Pd, Qd, prec).cpu().numpy()
    _check_twice(L, pkg, want, (Xd, n, Pd, r, Qd, n, m, n, r, PREC[dtype], PREC[prec]), tol)


@pytest.mark.parametrize("m,n,r", [(300, 512, 40), (1000, 776, 136)])
def test_noalloc_tensor_core_residual(m, n, r):
    """FP32 X with BF16 P and Q: the tensor-core residual kernel, whose grid
    (at most one CTA per SM) writes one partial pair per CTA into the array.
    n = 776 leaves ragged tiles in both directions."""
    import paper_1703_06065_gb300 as pkg
    from paper_1703_06065_gb300 import PREC

    device()
    L = pkg.load()
    rg = np.random.default_rng(m + 3 * r)
    X = to_dev(rg.standard_normal((m, n)).astype(np.float32))
    P = to_dev(rg.standard_normal((m, r)) / np.sqrt(r), torch.bfloat16)
    Q = to_dev(rg.standard_normal((r, n)), torch.bfloat16)
    want = pkg.residual(X, P, Q, "bf16").cpu().numpy()
    _check_twice(L, pkg, want, (X, n, P, r, Q, n, m, n, r, PREC["bf16"], PREC["bf16"]), 1e-12)


def test_noalloc_refuses_what_tma_cannot_describe():
    """A BF16 operand that is not 16-byte aligned: the tensor-core kernel
    cannot take it and, as bcur_residual does, the call is refused on the host
    with BCUR_ENOTSUP before anything is enqueued."""
    import paper_1703_06065_gb300 as pkg
    from paper_1703_06065_gb300 import PREC

    device()
    L = pkg.load()
    m, n, r = 256, 256, 16
    X = torch.zeros(m, n, device="cuda")
    P = torch.zeros(m * r + 8, dtype=torch.bfloat16, device="cuda")
    Q = torch.zeros(r, n, dtype=torch.bfloat16, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    Pm = P[1:1 + m * r]                        # base 2 bytes past a 16-byte boundary
    st = L.bcur_residual_noalloc(ctypes.c_void_p(X.data_ptr()), n, ctypes.c_void_p(Pm.data_ptr()),
                                 r, ctypes.c_void_p(Q.data_ptr()), n, m, n, r, PREC["bf16"],
                                 PREC["bf16"], ctypes.c_void_p(out.data_ptr()), None)
    assert st == 7  # BCUR_ENOTSUP


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1703_06065_gb300 as pkg

    device()
    L = pkg.load()
    tiny = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(tiny.data_ptr())
    # 257 x 257 tiles of 64 x 64 in FP64 need 66049 > 65536 partial pairs:
    # refused on the host before anything is enqueued.
    n = 64 * 257
    st = L.bcur_residual_noalloc(p, n, p, 1, p, n, n, n, 1, 0, 0, ctypes.c_void_p(out.data_ptr()),
                                 None)
    assert st == 2  # BCUR_ENOMEM
