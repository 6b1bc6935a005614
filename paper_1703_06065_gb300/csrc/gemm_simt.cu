// Dense GEMM on CUDA cores for FP64 and FP32 (sm_103a).
//
// This is the "plain" arithmetic path: every multiply-add is an FP32 or FP64
// FMA, so results match the oracle to the rounding of the working precision.
// The tensor-core path (gemm_tc.cu) is checked against it.
//
// Tile: BM x BN output per CTA, BK-deep K slices staged in shared memory,
// each of the 256 threads owning a TM x TN register micro-tile.  The next K
// slice is prefetched into registers while the current one is consumed.
#include "kernels.h"

namespace bcur {

template <typename T> struct SimtCfg;
template <> struct SimtCfg<float> { static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8; };
template <> struct SimtCfg<double> { static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4; };

template <typename T>
__device__ __forceinline__ void k_range(const GemmDesc& d, int64_t m0, int64_t n0, int z,
                                        int64_t& lo, int64_t& hi) {
  constexpr int BM = SimtCfg<T>::BM, BN = SimtCfg<T>::BN, BK = SimtCfg<T>::BK;
  lo = 0;
  hi = d.K;
  if (d.ksplit > 1) {
    int64_t chunk = ((d.K + d.ksplit - 1) / d.ksplit + BK - 1) / BK * BK;
    lo = (int64_t)z * chunk;
    hi = min(d.K, lo + chunk);
  }
  if (d.triA == 1) hi = min(hi, m0 + BM);
  if (d.triA == 2) lo = max(lo, m0);
  if (d.triB == 1) lo = max(lo, n0);
  if (d.triB == 2) hi = min(hi, n0 + BN);
}

template <typename T, bool RESID>
__global__ void __launch_bounds__(256) gemm_simt_kernel(GemmDesc d) {
  constexpr int BM = SimtCfg<T>::BM, BN = SimtCfg<T>::BN, BK = SimtCfg<T>::BK;
  constexpr int TM = SimtCfg<T>::TM, TN = SimtCfg<T>::TN;
  constexpr int NT = 256;
  constexpr int TX = BN / TN;
  constexpr int A_PER = BM * BK / NT;
  constexpr int B_PER = BN * BK / NT;
  static_assert((BM / TM) * (BN / TN) == NT, "thread layout");

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int z = blockIdx.z;
  if (!RESID && d.out_lower && m0 + BM - 1 < n0) return;

  const int64_t zb = (d.ksplit > 1) ? 0 : z;
  const T* A = (const T*)d.A + zb * d.sA;
  const T* B = (const T*)d.B + zb * d.sB;
  int64_t lo, hi;
  k_range<T>(d, m0, n0, z, lo, hi);

  __shared__ __align__(16) T As[BK][BM];
  __shared__ __align__(16) T Bs[BK][BN];
  T acc[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[r][c] = T(0);

  T ra[A_PER], rb[B_PER];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      const int idx = tid + e * NT;
      int i, kk;
      if (!d.transA) { kk = idx % BK; i = idx / BK; } else { i = idx % BM; kk = idx / BM; }
      const int64_t gi = m0 + i, gk = k0 + kk;
      T v = T(0);
      if (gi < d.M && gk < hi) v = d.transA ? A[gk * d.lda + gi] : A[gi * d.lda + gk];
      ra[e] = v;
    }
#pragma unroll
    for (int e = 0; e < B_PER; ++e) {
      const int idx = tid + e * NT;
      int j, kk;
      if (!d.transB) { j = idx % BN; kk = idx / BN; } else { kk = idx % BK; j = idx / BK; }
      const int64_t gj = n0 + j, gk = k0 + kk;
      T v = T(0);
      if (gj < d.N && gk < hi) v = d.transB ? B[gj * d.ldb + gk] : B[gk * d.ldb + gj];
      rb[e] = v;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      const int idx = tid + e * NT;
      int i, kk;
      if (!d.transA) { kk = idx % BK; i = idx / BK; } else { i = idx % BM; kk = idx / BM; }
      As[kk][i] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < B_PER; ++e) {
      const int idx = tid + e * NT;
      int j, kk;
      if (!d.transB) { j = idx % BN; kk = idx / BN; } else { kk = idx % BK; j = idx / BK; }
      Bs[kk][j] = rb[e];
    }
  };

  if (lo < hi) {
    load(lo);
    for (int64_t k0 = lo; k0 < hi; k0 += BK) {
      store();
      __syncthreads();
      if (k0 + BK < hi) load(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[TM], b[TN];
#pragma unroll
        for (int r = 0; r < TM; ++r) a[r] = As[kk][ty * TM + r];
#pragma unroll
        for (int c = 0; c < TN; ++c) b[c] = Bs[kk][tx * TN + c];
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
          for (int c = 0; c < TN; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
      }
      __syncthreads();
    }
  }

  const T alpha = (T)d.alpha;
  if constexpr (!RESID) {
    T* D = (T*)d.D + (int64_t)z * d.sD;
    const T beta = (T)d.beta;
#pragma unroll
    for (int r = 0; r < TM; ++r) {
      const int64_t gi = m0 + ty * TM + r;
      if (gi >= d.M) continue;
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        const int64_t gj = n0 + tx * TN + c;
        if (gj >= d.N || (d.out_lower && gi < gj)) continue;
        T v = alpha * acc[r][c];
        if (d.beta != 0.0) v = fma(beta, D[gi * d.ldd + gj], v);
        D[gi * d.ldd + gj] = v;
      }
    }
  } else {
    const T* X = (const T*)d.X;
    double e2 = 0.0, x2 = 0.0;
#pragma unroll
    for (int r = 0; r < TM; ++r) {
      const int64_t gi = m0 + ty * TM + r;
      if (gi >= d.M) continue;
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        const int64_t gj = n0 + tx * TN + c;
        if (gj >= d.N) continue;
        const double x = (double)X[gi * d.ldx + gj];
        const double v = x - (double)(alpha * acc[r][c]);
        e2 = fma(v, v, e2);
        x2 = fma(x, x, x2);
      }
    }
    // Fixed-order block reduction: xor-tree inside each warp, then warps in order.
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e2 += __shfl_xor_sync(0xffffffffu, e2, o);
      x2 += __shfl_xor_sync(0xffffffffu, x2, o);
    }
    __shared__ double red[2][NT / 32];
    if ((tid & 31) == 0) { red[0][tid >> 5] = e2; red[1][tid >> 5] = x2; }
    __syncthreads();
    if (tid == 0) {
      double se = 0.0, sx = 0.0;
      for (int w = 0; w < NT / 32; ++w) { se += red[0][w]; sx += red[1][w]; }
      const int64_t bid = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
      d.partials[2 * bid] = se;
      d.partials[2 * bid + 1] = sx;
    }
  }
}

template <typename T>
bcur_status_t gemm_simt(const GemmDesc& d, cudaStream_t s) {
  constexpr int BM = SimtCfg<T>::BM, BN = SimtCfg<T>::BN;
  if (d.M <= 0 || d.N <= 0) return BCUR_OK;
  const int64_t gx = ceil_div(d.N, BN), gy = ceil_div(d.M, BM);
  const int gz = d.ksplit > 1 ? d.ksplit : d.batch;
  if (gy > 65535 || gz > 65535 || gz < 1) return BCUR_EINVAL;
  if (d.ksplit > 1 && d.batch > 1) return BCUR_EINVAL;
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)gz);
  gemm_simt_kernel<T, false><<<grid, 256, 0, s>>>(d);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

template <typename T>
int64_t gemm_simt_resid_ctas(int64_t M, int64_t N) {
  return ceil_div(N, SimtCfg<T>::BN) * ceil_div(M, SimtCfg<T>::BM);
}

template <typename T>
bcur_status_t gemm_simt_resid(const GemmDesc& d, cudaStream_t s, int64_t* n_partials) {
  constexpr int BM = SimtCfg<T>::BM, BN = SimtCfg<T>::BN;
  const int64_t gx = ceil_div(d.N, BN), gy = ceil_div(d.M, BM);
  *n_partials = gx * gy;
  if (d.M <= 0 || d.N <= 0) return BCUR_OK;
  if (gy > 65535 || d.batch != 1 || d.ksplit != 1) return BCUR_EINVAL;
  dim3 grid((unsigned)gx, (unsigned)gy, 1);
  gemm_simt_kernel<T, true><<<grid, 256, 0, s>>>(d);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

template bcur_status_t gemm_simt<float>(const GemmDesc&, cudaStream_t);
template bcur_status_t gemm_simt<double>(const GemmDesc&, cudaStream_t);
template bcur_status_t gemm_simt_resid<float>(const GemmDesc&, cudaStream_t, int64_t*);
template bcur_status_t gemm_simt_resid<double>(const GemmDesc&, cudaStream_t, int64_t*);
template int64_t gemm_simt_resid_ctas<float>(int64_t, int64_t);
template int64_t gemm_simt_resid_ctas<double>(int64_t, int64_t);

}  // namespace bcur
