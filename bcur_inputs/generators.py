"""Seeded synthetic inputs for Block CUR workloads.

This module is shared by the FP64 oracle, the tests and the benchmark.  It
only *draws* numbers: matrices with the structure of the paper's workloads,
the Rademacher test matrix Omega of the randomized range finder, and the
uniform variates that drive block sampling.  It holds none of the method's
arithmetic (no leverage scores, no sampling rule, no factorisation of A).

Every random stream is keyed by ``(seed, stream)`` through NumPy's
``SeedSequence`` so that the oracle and the CUDA path see identical inputs.

Workload recipes (all synthetic stand-ins; the paper's EDA and Arcene data
are not available):

* ``small_lowrank``  -- the paper's synthetic family A = U V with iid
  Gaussian factors (Sec. 4.2), plus iid Gaussian noise.
* ``haar_spectrum`` -- A = U diag(sigma) V^T with Haar-random orthonormal
  factors and a power-law spectrum, plus iid Gaussian noise.
* ``ar1_mixture``   -- a biometric-like signal (Sec. 4.1 stand-in): k
  AR(1) time series of unit stationary variance mixed by an m x k Gaussian
  loading matrix, plus iid Gaussian noise.
"""
from __future__ import annotations

import math
import threading
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# Stream identifiers.  Each consumer of randomness draws from its own stream
# so that changing one (e.g. the number of blocks sampled) never shifts
# another.
STREAM_MATRIX = 1
STREAM_OMEGA = 2
STREAM_UCOL = 3
STREAM_UROW = 4
STREAM_SHAPES = 5
STREAM_ARRIVALS = 6


def rng(seed: int, stream: int) -> np.random.Generator:
    """Counter-free, reproducible generator for ``(seed, stream)``."""
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(stream)]))


# ----------------------------------------------------------------------------
# Matrices
# ----------------------------------------------------------------------------

def small_lowrank(m: int, n: int, rank: int, noise: float, seed: int) -> np.ndarray:
    """A = G1 (m x rank) . G2 (rank x n) + noise . N(0,1), FP64."""
    g = rng(seed, STREAM_MATRIX)
    g1 = g.standard_normal((m, rank))
    g2 = g.standard_normal((rank, n))
    a = g1 @ g2
    if noise:
        a = a + noise * g.standard_normal((m, n))
    return a


def haar_orthonormal(g: np.random.Generator, n: int, r: int) -> np.ndarray:
    """n x r matrix with Haar-distributed orthonormal columns.

    QR of a Gaussian matrix with the diagonal-sign correction of Mezzadri
    (2007), which makes the distribution exactly Haar.
    """
    z = g.standard_normal((n, r))
    q, rr = np.linalg.qr(z)
    d = np.sign(np.diag(rr))
    d[d == 0] = 1.0
    return q * d


def haar_spectrum(m: int, n: int, rank: int, decay: float, noise: float, seed: int) -> np.ndarray:
    """A = U diag(i^-decay) V^T + noise . N(0,1) (host, FP64; small sizes)."""
    g = rng(seed, STREAM_MATRIX)
    u = haar_orthonormal(g, m, rank)
    v = haar_orthonormal(g, n, rank)
    sig = np.arange(1, rank + 1, dtype=np.float64) ** (-decay)
    a = (u * sig) @ v.T
    if noise:
        a = a + noise * g.standard_normal((m, n))
    return a


def haar_spectrum_device(m: int, n: int, rank: int, decay: float, noise: float, seed: int,
                         device="cuda", dtype=None):
    """Same recipe as :func:`haar_spectrum`, drawn on a torch device.

    Used for the 32768 x 32768 workload, which is too large to draw on the
    host for every run.  The factors are formed in FP64 and the sum is cast
    to ``dtype`` (default float32) in row panels to bound peak memory.
    """
    import torch

    dtype = dtype or torch.float32
    # The thin Haar factors are drawn and orthonormalised on the host (NumPy),
    # only the m x n product and the noise are formed on the device.
    g = rng(seed, STREAM_MATRIX)
    u = torch.from_numpy(haar_orthonormal(g, m, rank)).to(device)
    v = torch.from_numpy(haar_orthonormal(g, n, rank)).to(device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1000003 + STREAM_MATRIX)
    sig = torch.arange(1, rank + 1, device=device, dtype=torch.float64) ** (-decay)
    us = (u * sig)
    a = torch.empty(m, n, device=device, dtype=dtype)
    panel = 2048
    for i0 in range(0, m, panel):
        i1 = min(m, i0 + panel)
        blk = us[i0:i1] @ v.T
        if noise:
            blk += noise * torch.randn(i1 - i0, n, generator=gen, device=device, dtype=torch.float64)
        a[i0:i1] = blk.to(dtype)
    return a


def _ar1_draw(m: int, n: int, k: int, phi: float, seed: int):
    g = rng(seed, STREAM_MATRIX)
    load = g.standard_normal((m, k)) / math.sqrt(k)
    e = g.standard_normal((k, n))
    x = np.empty((k, n))
    x[:, 0] = e[:, 0]
    c = math.sqrt(1.0 - phi * phi)
    for t in range(1, n):
        x[:, t] = phi * x[:, t - 1] + c * e[:, t]
    return load, x, g


def ar1_factors(m: int, n: int, k: int, phi: float, seed: int):
    """The loading L (m x k) and the AR(1) series X (k x n) of :func:`ar1_mixture`
    (same generator stream, so both recipes share L and X)."""
    load, x, _ = _ar1_draw(m, n, k, phi, seed)
    return load, x


_AR1_CACHE: dict = {}
_GEN_CACHE = threading.local()


def _ar1_mats(phi: float, B: int, nc: int, device):
    """Cached pieces of the chunked AR(1) recurrence, formed on the device:
    T^T (B x B, T = phi^(i - j) on and below the diagonal), S^T (S = phi^(B (i - j))
    over chunks; lower-triangular Toeplitz, so the leading nc x nc block of a
    larger one is the same) and phi^(i + 1)."""
    import torch

    key = (float(phi), B, str(device))
    got = _AR1_CACHE.get(key)
    if got is None or got[1].shape[0] < nc:
        size = max(nc, 128 if got is None else 2 * got[1].shape[0])
        i = torch.arange(B, device=device, dtype=torch.float32)
        d = i.view(B, 1) - i.view(1, B)
        T = torch.where(d >= 0, torch.pow(phi, d.clamp(min=0)), torch.zeros_like(d))
        jj = torch.arange(size, device=device, dtype=torch.float32)
        dj = jj.view(size, 1) - jj.view(1, size)
        S = torch.where(dj >= 0, torch.pow(phi ** B, dj.clamp(min=0)), torch.zeros_like(dj))
        got = (T.t().contiguous(), S.t().contiguous(), torch.pow(phi, i + 1))
        _AR1_CACHE[key] = got
    return got[0], got[1][:nc, :nc], got[2]


def ar1_series_chunked(e, phi: float, chunk: int = 128):
    """The AR(1) rows x_0 = e_0, x_t = phi x_{t-1} + sqrt(1 - phi^2) e_t of a
    k x n innovation matrix e (torch, any device), computed as a chunked linear
    recurrence: inside each chunk of `chunk` steps the solution from a zero
    start is one product with the lower-triangular matrix of powers
    phi^(i - j); the chunks' end values are joined by a second small product
    over chunks, and each chunk adds its predecessor's end value times
    phi^(i + 1).  Two matrix products in place of a sequential scan; exact up
    to FP32 rounding (no truncation)."""
    import torch

    k, n = e.shape
    B = chunk
    nc = (n + B - 1) // B
    Tt, St, pw = _ar1_mats(phi, B, nc, e.device)
    src = torch.zeros(k, nc * B, device=e.device, dtype=torch.float32)
    src[:, :n].copy_(e).mul_(math.sqrt(1.0 - phi * phi))
    src[:, 0] = e[:, 0]
    y = (src.view(k * nc, B) @ Tt).view(k, nc, B)       # each chunk from a zero start
    z = y[:, :, B - 1] @ St                             # chunk end values, k x nc
    y[:, 1:, :].addcmul_(z[:, :-1].unsqueeze(2), pw.view(1, 1, B))
    return y.view(k, nc * B)[:, :n]


def _device_generator(device):
    """One reusable torch generator per thread and device (reseeded per use)."""
    import torch

    gens = getattr(_GEN_CACHE, "gens", None)
    if gens is None:
        gens = _GEN_CACHE.gens = {}
    key = str(device)
    g = gens.get(key)
    if g is None:
        g = gens[key] = torch.Generator(device=device)
    return g


def ar1_mixture_stream(m: int, n: int, k: int, phi: float, noise: float, seed: int,
                       device="cuda", out=None):
    """The biometric-like recipe drawn entirely on the device (the serving
    workload, where every request's matrix is drawn at admission): L and the
    innovations from a seeded torch generator, the AR(1) series by
    :func:`ar1_series_chunked`, A = noise * N(0,1) + L X.  FP32."""
    import torch

    gen = _device_generator(device)
    gen.manual_seed(int(seed) * 1000003 + STREAM_MATRIX)
    L = torch.randn(m, k, generator=gen, device=device).mul_(1.0 / math.sqrt(k))
    e = torch.randn(k, n, generator=gen, device=device)
    x = ar1_series_chunked(e, phi)
    # A = noise * N(0,1) + L x, formed in place (out: a preallocated m x n buffer)
    a = torch.empty(m, n, device=device) if out is None else out
    if noise:
        a.normal_(0.0, noise, generator=gen)
    else:
        a.zero_()
    # the rank-k product on tensor cores with TF32 inputs and FP32 accumulation:
    # A is still exactly rank k plus noise (the product of TF32-rounded
    # factors); an FP32 product cost about as much as decomposing the request
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        a.addmm_(L, x)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return a


def request_inputs_device(p: "Problem", device="cuda", out=None):
    """Every input of one serving request drawn on the device from its seed:
    A (the biometric recipe, :func:`ar1_mixture_stream`), the Rademacher test
    matrix as an l x n panel (FP32) and the column / row uniforms (FP64 in
    [0, 1))."""
    import torch

    r = p.recipe
    A = ar1_mixture_stream(p.m, p.n, r["rank"], r["phi"], r["noise"], p.seed, device=device,
                           out=out)
    gen = _device_generator(device)
    gen.manual_seed(int(p.seed) * 1000003 + STREAM_OMEGA)
    om = torch.empty(p.l, p.n, device=device).bernoulli_(0.5, generator=gen).mul_(2.0).sub_(1.0)
    u = torch.rand(p.g_col + p.g_row, generator=gen, device=device, dtype=torch.float64)
    return A, om, u[:p.g_col], u[p.g_col:]


def ar1_mixture_device(m: int, n: int, k: int, phi: float, noise: float, seed: int,
                       device="cuda", dtype=None):
    """The biometric-like recipe drawn on a torch device: L and X as in
    :func:`ar1_mixture` (host, small), the product and the noise on the device
    (noise from a seeded torch generator, so it differs from the host recipe's
    noise draw; the distribution is the same)."""
    import torch

    dtype = dtype or torch.float32
    load, x = ar1_factors(m, n, k, phi, seed)
    L = torch.from_numpy(load).to(device=device, dtype=torch.float32)
    X = torch.from_numpy(x).to(device=device, dtype=torch.float32)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1000003 + STREAM_MATRIX)
    a = L @ X
    if noise:
        a += noise * torch.randn(m, n, generator=gen, device=device, dtype=torch.float32)
    return a.to(dtype)


def ar1_mixture(m: int, n: int, k: int, phi: float, noise: float, seed: int) -> np.ndarray:
    """Biometric-like matrix: L (m x k, N(0,1)/sqrt(k)) . X (k x n AR(1)) + noise.

    Each row of X follows x_t = phi x_{t-1} + sqrt(1 - phi^2) e_t with
    x_0 ~ N(0,1), so every series has unit stationary variance.
    """
    load, x, g = _ar1_draw(m, n, k, phi, seed)
    a = load @ x
    if noise:
        a = a + noise * g.standard_normal((m, n))
    return a


# ----------------------------------------------------------------------------
# Random variates the method consumes
# ----------------------------------------------------------------------------

def rademacher(n: int, l: int, seed: int) -> np.ndarray:
    """Omega (n x l) with iid +-1 entries, FP64 (exact in every precision)."""
    g = rng(seed, STREAM_OMEGA)
    return (g.integers(0, 2, size=(n, l), dtype=np.int8).astype(np.float64) * 2.0 - 1.0)


def uniforms(count: int, seed: int, stream: int) -> np.ndarray:
    """``count`` doubles uniform on [0, 1) with 53 random bits each."""
    return rng(seed, stream).random(count)


# ----------------------------------------------------------------------------
# Block partitions
# ----------------------------------------------------------------------------

def uniform_blocks(n: int, s: int) -> np.ndarray:
    """Offsets of contiguous blocks of ``s`` indices; G = ceil(n/s), last may be short."""
    G = -(-n // s)
    off = np.minimum(np.arange(G + 1, dtype=np.int64) * s, n)
    return off


def blocks_to_sample(k: int, s: int, G: int, other: int = None) -> int:
    """Number of blocks per side for the batched workloads:
    min(ceil(2k/s)+1, ceil(G/2)), and (given the length `other` of the other
    side: m for column blocks, n for row blocks) at most floor(other/(2s)),
    at least 1, so that C (m x c) and R (r x n) stay tall, c <= m/2 and
    r <= n/2."""
    g = min(-(-2 * k // s) + 1, -(-G // 2))
    if other is not None:
        g = min(g, max(1, other // (2 * s)))
    return int(g)


# ----------------------------------------------------------------------------
# Workload descriptions
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    """One Block CUR problem: a matrix recipe plus the method's parameters."""
    name: str
    m: int
    n: int
    k: int
    p: int
    q: int
    col_off: np.ndarray
    row_off: np.ndarray
    g_col: int
    g_row: int
    seed: int
    storage: str = "f64"          # "f64" or "f32"
    replacement: bool = False
    recipe: dict = field(default_factory=dict)

    @property
    def l(self) -> int:
        return self.k + self.p

    def matrix(self) -> np.ndarray:
        """The stored matrix (host), in its storage precision."""
        r = self.recipe
        kind = r["kind"]
        if kind == "small_lowrank":
            a = small_lowrank(self.m, self.n, r["rank"], r["noise"], self.seed)
        elif kind == "haar_spectrum":
            a = haar_spectrum(self.m, self.n, r["rank"], r["decay"], r["noise"], self.seed)
        elif kind == "ar1_mixture":
            a = ar1_mixture(self.m, self.n, r["rank"], r["phi"], r["noise"], self.seed)
        else:
            raise ValueError(kind)
        return a.astype(np.float32) if self.storage == "f32" else a

    def matrix_device(self, device="cuda"):
        """The stored matrix drawn on a device (the large workloads)."""
        r = self.recipe
        kind = r["kind"]
        if kind == "ar1_mixture":
            return ar1_mixture_device(self.m, self.n, r["rank"], r["phi"], r["noise"], self.seed,
                                      device=device)
        if kind == "haar_spectrum":
            return haar_spectrum_device(self.m, self.n, r["rank"], r["decay"], r["noise"],
                                        self.seed, device=device)
        raise ValueError(kind)

    def omega(self) -> np.ndarray:
        return rademacher(self.n, self.l, self.seed)

    def u_col(self) -> np.ndarray:
        return uniforms(self.g_col, self.seed, STREAM_UCOL)

    def u_row(self) -> np.ndarray:
        return uniforms(self.g_row, self.seed, STREAM_UROW)


def plain_fp64_512x1024(seed: int = 0) -> Problem:
    """512 x 1024 rank-10 Gaussian product + 0.01 noise; 32 column / 16 row blocks of 32."""
    return Problem("plain_fp64_512x1024", 512, 1024, k=10, p=10, q=2,
                   col_off=uniform_blocks(1024, 32), row_off=uniform_blocks(512, 32),
                   g_col=8, g_row=6, seed=seed, storage="f64",
                   recipe=dict(kind="small_lowrank", rank=10, noise=0.01))


def fp32_32768(seed: int = 1, k: int = 50, p: int = 10, q: int = 2) -> Problem:
    """32768^2 Haar rank-200 spectrum i^-1.5 + 1e-4 noise; 64+64 blocks of 512; 16+16 sampled."""
    n = 32768
    return Problem("fp32_32768", n, n, k=k, p=p, q=q,
                   col_off=uniform_blocks(n, 512), row_off=uniform_blocks(n, 512),
                   g_col=16, g_row=16, seed=seed, storage="f32",
                   recipe=dict(kind="haar_spectrum", rank=200, decay=1.5, noise=1e-4))


def precision_32768(seed: int = 1) -> Problem:
    """The 32768^2 matrix of :func:`fp32_32768` with k = 100, p = 20, q = 3 (the
    precision study: BF16 sketch, error against FP64 reported per stage)."""
    p = fp32_32768(seed=seed, k=100, p=20, q=3)
    p.name = "precision_32768"
    return p


def scaled_haar(m: int, n: int, s: int, k: int, p: int, q: int, g_col: int, g_row: int,
                seed: int, storage: str = "f32", rank: int = 200, noise: float = 1e-4) -> Problem:
    """The Haar-spectrum recipe at an arbitrary (smaller) size, for parity tests."""
    return Problem(f"haar_{m}x{n}_s{s}", m, n, k=k, p=p, q=q,
                   col_off=uniform_blocks(n, s), row_off=uniform_blocks(m, s),
                   g_col=g_col, g_row=g_row, seed=seed, storage=storage,
                   recipe=dict(kind="haar_spectrum", rank=min(rank, m, n), decay=1.5, noise=noise))


def host_sample(full: Problem, factor: int = 4) -> Problem:
    """A bounded stand-in of a large single-matrix workload for timing the host
    oracle: the same recipe at 1/factor the size per side, blocks of the same
    width, and g scaled so that c/n and r/m stay as in the full problem.
    Problems of at most 8192 x 8192 are returned unchanged."""
    if full.m <= 8192 and full.n <= 8192:
        return full
    m, n = full.m // factor, full.n // factor
    s = int(full.col_off[1])
    gs = max(1, full.g_col // factor)
    r = full.recipe
    return scaled_haar(m, n, s, k=full.k, p=full.p, q=full.q, g_col=gs, g_row=gs, seed=full.seed,
                       rank=min(r.get("rank", 200), m), noise=r.get("noise", 1e-4))


def _biometric(g: np.random.Generator, name: str, seed: int, m_range=(256, 4096),
               n_range=(1024, 16384), k_range=(5, 50), blocks=(16, 32, 64, 128, 256)) -> Problem:
    s = int(g.choice(list(blocks)))
    # at least two blocks per side: with one, the draw is forced and C or R is all of A
    m = max(int(g.integers(m_range[0], m_range[1] + 1)) // s * s, 2 * s)
    n = max(int(g.integers(n_range[0], n_range[1] + 1)) // s * s, 2 * s)
    k = int(g.integers(k_range[0], k_range[1] + 1))
    Gc, Gr = n // s, m // s
    return Problem(name, m, n, k=k, p=10, q=2,
                   col_off=uniform_blocks(n, s), row_off=uniform_blocks(m, s),
                   g_col=blocks_to_sample(k, s, Gc, m), g_row=blocks_to_sample(k, s, Gr, n),
                   seed=seed, storage="f32",
                   recipe=dict(kind="ar1_mixture", rank=k, phi=0.95, noise=0.05))


def batched_biometric(count: int = 512, seed: int = 3, m_range=(256, 4096), n_range=(1024, 16384),
                      k_range=(5, 50), blocks=(16, 32, 64, 128, 256)) -> List[Problem]:
    """Uneven batch: m~U[256,4096], n~U[1024,16384] (rounded down to s, at least 2s),
    s in {16..256}, k~U[5,50].

    The ranges can be narrowed for test-sized batches; the defaults are the
    512-matrix biometric workload."""
    g = rng(seed, STREAM_SHAPES)
    return [_biometric(g, f"bio_{i}", seed * 100003 + i, m_range, n_range, k_range, blocks)
            for i in range(count)]


@dataclass
class Request:
    """One decomposition request of the serving workload."""
    rid: int
    arrival: float          # seconds after the start of the run
    problem: Problem
    heavy: bool


def serving_requests(rate: float = 2000.0, duration: float = 60.0, seed: int = 4,
                     heavy_frac: float = 0.1, heavy_n: int = 16384,
                     **light_ranges) -> List[Request]:
    """Poisson arrivals at `rate` per second for `duration` seconds: a fraction
    `heavy_frac` of heavy_n^2 matrices (16384 by default; blocks of 256,
    k = 64, 2 + 2 blocks drawn), the rest drawn like the members of the
    biometric batch (`light_ranges` narrows their shapes for tests)."""
    ga = rng(seed, STREAM_ARRIVALS)
    gs = rng(seed, STREAM_SHAPES)
    out, t, i = [], 0.0, 0
    while True:
        t += float(ga.exponential(1.0 / rate))
        if t >= duration:
            break
        rseed = seed * 1000003 + i
        if float(gs.random()) < heavy_frac:
            n = heavy_n
            p = Problem(f"heavy_{i}", n, n, k=64, p=10, q=2, col_off=uniform_blocks(n, 256),
                        row_off=uniform_blocks(n, 256), g_col=2, g_row=2, seed=rseed,
                        storage="f32", recipe=dict(kind="ar1_mixture", rank=64, phi=0.95,
                                                   noise=0.05))
            out.append(Request(i, t, p, True))
        else:
            out.append(Request(i, t, _biometric(gs, f"req_{i}", rseed, **light_ranges), False))
        i += 1
    return out
