"""Parity of the tcgen05 tensor-core GEMM (TF32) with the FP32 CUDA-core GEMM
and with FP64 on the host, for every operand layout the library uses."""
import numpy as np
import pytest

from _gpu_common import device, to_dev, torch  # noqa: F401

pytestmark = pytest.mark.gpu

# TF32 keeps 10 explicit mantissa bits: each product carries a relative error
# below 2^-9, and over K random-sign terms the Frobenius-relative error of D
# stays near 2^-10; 5e-3 leaves a wide margin without hiding a wrong layout
# (which gives O(1) errors).
TF32_REL = 5e-3


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("tA,tB", [(0, 1), (0, 0), (1, 1), (1, 0)])
@pytest.mark.parametrize("M,N,K", [(256, 512, 256), (300, 520, 200), (128, 64, 96), (1000, 136, 333)])
def test_tc_gemm_layouts(tA, tB, M, N, K):
    import paper_1703_06065_gb300 as pkg

    device()
    rg = np.random.default_rng(M * 3 + N + K + tA * 7 + tB * 11)
    Kp = (K + 3) // 4 * 4
    A = rg.standard_normal((K, M) if tA else (M, K)).astype(np.float32)
    B = rg.standard_normal((N, K) if tB else (K, N)).astype(np.float32)
    ref = (A.T if tA else A).astype(np.float64) @ (B.T if tB else B).astype(np.float64)
    # leading dimensions must be multiples of 4 floats for TMA: pad columns
    def padded(X):
        cols = (X.shape[1] + 3) // 4 * 4
        Y = np.zeros((X.shape[0], cols), np.float32)
        Y[:, :X.shape[1]] = X
        return Y
    Ad, Bd = to_dev(padded(A)), to_dev(padded(B))
    Mo, No = M, N
    Dt = torch.zeros(Mo, (No + 3) // 4 * 4, dtype=torch.float32, device=Ad.device)
    L = pkg.load()
    import ctypes
    st = L.bcur_gemm(M, N, K, ctypes.c_void_p(Ad.data_ptr()), Ad.shape[1], tA,
                     ctypes.c_void_p(Bd.data_ptr()), Bd.shape[1], tB, ctypes.c_void_p(Dt.data_ptr()),
                     Dt.shape[1], 1, 2, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if tA == 1 or tB == 0:
        # an MN-major TF32 operand: the tensor core reads zeros for it on
        # sm_103a, so the library refuses the call instead of computing it
        assert st == 7, pkg._lib.STATUS.get(st)
        return
    assert st == 0, pkg._lib.STATUS.get(st)
    got = Dt[:, :N].double().cpu().numpy()
    assert _rel(got, ref) < TF32_REL
    # and the CUDA-core FP32 result is much closer
    Ds = torch.zeros_like(Dt)
    st = L.bcur_gemm(M, N, K, ctypes.c_void_p(Ad.data_ptr()), Ad.shape[1], tA,
                     ctypes.c_void_p(Bd.data_ptr()), Bd.shape[1], tB, ctypes.c_void_p(Ds.data_ptr()),
                     Ds.shape[1], 1, 1, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    assert _rel(Ds[:, :N].double().cpu().numpy(), ref) < 1e-5


@pytest.mark.parametrize("tA,tB", [(0, 1), (0, 0), (1, 1), (1, 0)])
@pytest.mark.parametrize("M,N,K", [(256, 512, 256), (300, 520, 200), (1000, 136, 328)])
def test_tc_gemm_bf16_layouts(tA, tB, M, N, K):
    """BF16 operands (products exact in FP32): compare with FP64 on the rounded values."""
    import ctypes

    import paper_1703_06065_gb300 as pkg

    device()
    rg = np.random.default_rng(M + 5 * N + K + tA * 7 + tB * 11)
    A = torch.from_numpy(rg.standard_normal((K, M) if tA else (M, K))).to(torch.bfloat16)
    B = torch.from_numpy(rg.standard_normal((N, K) if tB else (K, N))).to(torch.bfloat16)
    def pad8(X):
        cols = (X.shape[1] + 7) // 8 * 8
        Y = torch.zeros(X.shape[0], cols, dtype=torch.bfloat16)
        Y[:, :X.shape[1]] = X
        return Y.cuda()
    Ad, Bd = pad8(A), pad8(B)
    A64, B64 = A.double().numpy(), B.double().numpy()
    ref = (A64.T if tA else A64) @ (B64.T if tB else B64)
    D = torch.zeros(M, (N + 3) // 4 * 4, dtype=torch.float32, device="cuda")
    L = pkg.load()
    st = L.bcur_gemm(M, N, K, ctypes.c_void_p(Ad.data_ptr()), Ad.shape[1], tA,
                     ctypes.c_void_p(Bd.data_ptr()), Bd.shape[1], tB, ctypes.c_void_p(D.data_ptr()),
                     D.shape[1], 3, 3, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, pkg._lib.STATUS.get(st)
    got = D[:, :N].double().cpu().numpy()
    assert _rel(got, ref) < 1e-5


def test_tc_skinny_long_swapped():
    """M = 60 rows, N = 4096: computed as D^T on the MMA and stored transposed."""
    import paper_1703_06065_gb300 as pkg

    device()
    rg = np.random.default_rng(1)
    A = rg.standard_normal((60, 2048)).astype(np.float32)
    B = rg.standard_normal((4096, 2048)).astype(np.float32)
    got = pkg.gemm(to_dev(A), to_dev(B), False, True, "tf32").double().cpu().numpy()
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    assert _rel(got, ref) < TF32_REL


@pytest.mark.parametrize("m,n,r", [(1024, 768, 256), (517, 300, 136), (300, 4100, 64)])
def test_tc_residual_bf16(m, n, r):
    """Fused residual on tensor cores: X FP32, P and Q BF16 (MN-major Q)."""
    import paper_1703_06065_gb300 as pkg

    device()
    rg = np.random.default_rng(m + 3 * r)
    rp, np_ = (r + 7) // 8 * 8, (n + 7) // 8 * 8
    X = np.zeros((m, np_), np.float32)
    X[:, :n] = rg.standard_normal((m, n))
    P = torch.zeros(m, rp, dtype=torch.bfloat16)
    P[:, :r] = torch.from_numpy(rg.standard_normal((m, r)) / np.sqrt(r)).to(torch.bfloat16)
    Q = torch.zeros(r, np_, dtype=torch.bfloat16)
    Q[:, :n] = torch.from_numpy(rg.standard_normal((r, n))).to(torch.bfloat16)
    P64, Q64 = P.double().numpy(), Q.double().numpy()
    want = float(np.sum((X.astype(np.float64) - P64 @ Q64) ** 2))
    out = pkg.residual(to_dev(X), P.cuda(), Q.cuda(), "bf16").cpu().numpy()
    # BF16 products are exact in FP32; the FP32 accumulation and the FP32
    # squared sums of 32 terms leave about 1e-6.
    assert abs(out[0] - want) <= 1e-5 * want
    out2 = pkg.residual(to_dev(X), P.cuda(), Q.cuda(), "bf16").cpu().numpy()
    assert out.tobytes() == out2.tobytes()


@pytest.mark.parametrize("m,n,r", [(1024, 768, 256), (517, 300, 136)])
def test_tc_residual(m, n, r):
    import paper_1703_06065_gb300 as pkg

    device()
    rg = np.random.default_rng(m + r)
    rp, np_ = (r + 3) // 4 * 4, (n + 3) // 4 * 4
    X = np.zeros((m, np_), np.float32)
    X[:, :n] = rg.standard_normal((m, n))
    P = np.zeros((m, rp), np.float32)
    P[:, :r] = rg.standard_normal((m, r)) / np.sqrt(r)
    Q = np.zeros((r, np_), np.float32)
    Q[:, :n] = rg.standard_normal((r, n))
    want = float(np.sum((X.astype(np.float64) - P.astype(np.float64) @ Q.astype(np.float64)) ** 2))
    out = pkg.residual(to_dev(X), to_dev(P), to_dev(Q), "tf32").cpu().numpy()
    assert abs(out[0] - want) <= 1e-4 * want
    out2 = pkg.residual(to_dev(X), to_dev(P), to_dev(Q), "tf32").cpu().numpy()
    assert out.tobytes() == out2.tobytes()


@pytest.mark.parametrize("tA,tB", [(0, 1), (0, 0), (1, 0)])
def test_tc_gemm_split_precision(tA, tB):
    """Three-term split BF16 keeps ~16 bits: far closer to FP64 than one BF16 term."""
    import paper_1703_06065_gb300 as pkg

    device()
    rg = np.random.default_rng(21 + tA + 2 * tB)
    M, N, K = 384, 520, 456
    A = rg.standard_normal((K, M) if tA else (M, K)).astype(np.float32)
    B = rg.standard_normal((N, K) if tB else (K, N)).astype(np.float32)
    ref = (A.T if tA else A).astype(np.float64) @ (B.T if tB else B).astype(np.float64)
    def split(X):
        t = torch.from_numpy(X).cuda()
        hi = t.to(torch.bfloat16)
        lo = (t - hi.float()).to(torch.bfloat16)
        return hi.contiguous(), lo.contiguous()
    Ah, Al = split(A)
    Bh, Bl = split(B)
    got = pkg.gemm_split(Ah, Al, Bh, Bl, bool(tA), bool(tB)).double().cpu().numpy()
    # hi/lo carries 16 mantissa bits; the dropped lo*lo term and the FP32
    # accumulation leave a Frobenius-relative error near 2^-17.
    assert _rel(got, ref) < 3e-5


@pytest.mark.parametrize("M,N,K", [(256, 512, 256), (300, 520, 200), (60, 4096, 384), (1000, 136, 328)])
def test_tc_gemm_fp8_exact(M, N, K):
    """FP8 e4m3 operands (kind::f8f6f4, both K-major): small integers are exact
    in e4m3 and their products and sums exact in FP32, so the result must equal
    the FP64 product bit for bit.  Other layouts are refused (ENOTSUP)."""
    import ctypes

    import paper_1703_06065_gb300 as pkg

    device()
    f8 = getattr(torch, "float8_e4m3fn", None)
    if f8 is None:
        pytest.skip("torch without float8_e4m3fn")
    rg = np.random.default_rng(M * 3 + N + K)
    A = rg.integers(-8, 9, size=(M, K)).astype(np.float32)
    B = rg.integers(-8, 9, size=(N, K)).astype(np.float32)   # B^T stored: K-major
    def pad16(X):
        cols = (X.shape[1] + 15) // 16 * 16
        Y = np.zeros((X.shape[0], cols), dtype=np.float32)
        Y[:, :X.shape[1]] = X
        return torch.from_numpy(Y).to(f8).cuda()
    Ad, Bd = pad16(A), pad16(B)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    D = torch.zeros(M, (N + 3) // 4 * 4, dtype=torch.float32, device="cuda")
    L = pkg.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.bcur_gemm(M, N, K, ctypes.c_void_p(Ad.data_ptr()), Ad.shape[1], 0,
                     ctypes.c_void_p(Bd.data_ptr()), Bd.shape[1], 1, ctypes.c_void_p(D.data_ptr()),
                     D.shape[1], 5, 5, stream)
    assert st == 0, pkg._lib.STATUS.get(st)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(D[:, :N].double().cpu().numpy(), ref)
    # an MN-major operand is refused rather than read wrongly
    st = L.bcur_gemm(M, N, K, ctypes.c_void_p(Ad.data_ptr()), Ad.shape[1], 0,
                     ctypes.c_void_p(Bd.data_ptr()), Bd.shape[1], 0, ctypes.c_void_p(D.data_ptr()),
                     D.shape[1], 5, 5, stream)
    assert st == 7
