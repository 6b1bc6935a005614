// Small and memory-bound kernels of the Block CUR hot path (sm_103a):
// block leverage scores (Def. 2), inverse-CDF block sampling (Alg. 1 step 2),
// block gathers for C and R (Alg. 1), the FP64 Cholesky of small Gram
// matrices used by Cholesky-QR, the diagonal-block factorisation of the
// blocked Cholesky, a one-sided Jacobi SVD for the l x l projected factor,
// and fixed-order FP64 reductions.
#include <float.h>

#include <algorithm>

#include <cuda_fp8.h>

#include <cooperative_groups.h>

#include "kernels.h"
#include "leaf.cuh"

namespace bcur {

// ---------------------------------------------------------------------------
// Fixed-order reductions
// ---------------------------------------------------------------------------
template <typename T>
__global__ void reduce_splits_kernel(const T* part, int nsplit, int64_t stride, int64_t count,
                                     double* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  double s = 0.0;
  for (int z = 0; z < nsplit; ++z) s += (double)part[(int64_t)z * stride + e];
  out[e] = s;
}

template <typename T>
bcur_status_t reduce_splits_f64(const T* part, int nsplit, int64_t stride, int64_t count,
                                double* out, cudaStream_t s) {
  if (count <= 0) return BCUR_OK;
  reduce_splits_kernel<T><<<(unsigned)ceil_div(count, 256), 256, 0, s>>>(part, nsplit, stride,
                                                                          count, out);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void finish_residual_kernel(const double* partials, int64_t n, double* out, int mode,
                                       int* flag) {
  if (mode == 3 && *flag == 0) return;
  double e2 = 0.0, x2 = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    e2 += partials[2 * i];
    x2 += partials[2 * i + 1];
  }
  e2 = warp_sum(e2);
  x2 = warp_sum(x2);
  __shared__ double r[2][32];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { r[0][w] = e2; r[1][w] = x2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double se = 0.0, sx = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { se += r[0][i]; sx += r[1][i]; }
    if (mode != 1) {
      const double e = sqrt(se), a = sqrt(sx);
      out[0] = e;
      out[1] = a > 0.0 ? e / a : 0.0;
      out[2] = a;
      if (mode == 2) *flag = residual_needs_refine(out[1]) ? 1 : 0;
    } else {
      out[0] = se;
      out[1] = sx;
    }
  }
}

bcur_status_t finish_residual(const double* partials, int64_t n, double* out, int mode,
                              cudaStream_t s, int* flag) {
  if (mode >= 2 && !flag) return BCUR_EINVAL;
  finish_residual_kernel<<<1, 1024, 0, s>>>(partials, n, out, mode, flag);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

__global__ void select_result_kernel(const double* r0, const double* r1, const int* flag,
                                     double* out) {
  const int i = threadIdx.x;
  if (i < 3) out[i] = *flag ? r1[i] : r0[i];
}

bcur_status_t select_result(const double* r0, const double* r1, const int* flag, double* out,
                            cudaStream_t s) {
  select_result_kernel<<<1, 32, 0, s>>>(r0, r1, flag, out);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

// ---------------------------------------------------------------------------
// Small FP64 Cholesky with the drop rule, and its inverse
// ---------------------------------------------------------------------------
template <typename T>
__global__ void chol_small_kernel(const double* G, int w, double tol_rel, double* L64,
                                  double* Linv64, T* LinvT, int* kept) {
  extern __shared__ double S[];
  chol_small_body<T>(G, w, w, tol_rel, L64, Linv64, LinvT, kept, S);
}

template <typename T>
bcur_status_t chol_small(const double* G, int w, double tol_rel, double* L64, double* Linv64,
                         T* LinvT, int* kept, cudaStream_t s) {
  if (w < 1 || w > 128) return BCUR_EINVAL;
  const size_t smem = (size_t)w * (w + 1) * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    BCUR_CUDA_TRY(cudaFuncSetAttribute(chol_small_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024));
    attr_set = true;
  }
  chol_small_kernel<T><<<1, 256, smem, s>>>(G, w, tol_rel, L64, Linv64, LinvT, kept);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

__global__ void trmm_small_kernel(const double* La, const double* Lb, int w, double* Lc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= w * w) return;
  const int i = e / w, j = e % w;
  double acc = 0.0;
  if (j <= i)
    for (int k = j; k <= i; ++k) acc += La[i * w + k] * Lb[k * w + j];
  Lc[e] = acc;
}

bcur_status_t trmm_small_f64(const double* La, const double* Lb, int w, double* Lc,
                             cudaStream_t s) {
  trmm_small_kernel<<<(unsigned)ceil_div((int64_t)w * w, 256), 256, 0, s>>>(La, Lb, w, Lc);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi SVD of a small square matrix, one CTA.
// Columns of X are rotated pairwise until mutually orthogonal: X J = U Sigma,
// so X = U Sigma J^T.  Pairs follow a round-robin tournament so that each
// round's rotations are disjoint and run in parallel, one warp per pair.
// ---------------------------------------------------------------------------
template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = 1.1920928955078125e-07; };
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };

__device__ __forceinline__ int rr_player(int pos, int round, int wp) {
  return pos == 0 ? 0 : ((pos - 1 + round) % (wp - 1)) + 1;
}

template <typename T>
__global__ void jacobi_svd_kernel(const double* X, int ws, T* Ut, T* W, double* sigma, T* J,
                                  int* status, const int* wdim) {
  extern __shared__ unsigned char smem_raw[];
  // ws: the stride of the stored w x w matrices; w: the leading block that is
  // factored (a batch entry's own width when wdim is given; the rest of the
  // stored matrix is zero and its outputs are written as zeros)
  const int64_t b = blockIdx.x;
  const int w = wdim ? min(ws, max(1, wdim[b])) : ws;
  T* Xs = reinterpret_cast<T*>(smem_raw);  // column-major: column p at Xs[p * w]
  const int wp = w + (w & 1);
  {  // batch: one matrix per CTA
    const int64_t wsp = ws + (ws & 1);
    X += b * ws * ws;
    if (Ut) Ut += b * ws * ws;
    if (W) W += b * ws * ws;
    sigma += b * ws;
    J += b * wsp * wsp;
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  for (int e = tid; e < wp * w; e += blockDim.x) {
    const int p = e / w, i = e % w;
    Xs[e] = (p < w) ? (T)X[i * ws + p] : T(0);
  }
  for (int e = tid; e < wp * wp; e += blockDim.x) J[e] = (e / wp == e % wp) ? T(1) : T(0);
  __shared__ int s_rot;
  __shared__ int s_order[128];
  __shared__ double s_sig[128];
  __syncthreads();
  const T tol = (T)(8.0 * Eps<T>::v);
  const int max_sweeps = 40;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < wp - 1; ++round) {
      for (int pr = warp; pr < wp / 2; pr += nwarps) {
        int p = rr_player(pr, round, wp), q = rr_player(wp - 1 - pr, round, wp);
        if (p > q) { const int t = p; p = q; q = t; }
        T* xp = Xs + (int64_t)p * w;
        T* xq = Xs + (int64_t)q * w;
        T a = 0, b = 0, g = 0;
        for (int i = lane; i < w; i += 32) {
          const T u = xp[i], v = xq[i];
          a += u * u;
          b += v * v;
          g += u * v;
        }
        a = warp_sum(a);
        b = warp_sum(b);
        g = warp_sum(g);
        if (g != T(0) && a > T(0) && b > T(0) && fabs(g) > tol * sqrt(a * b)) {
          const T zeta = (b - a) / (T(2) * g);
          const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          const T c = T(1) / sqrt(T(1) + t * t);
          const T sn = c * t;
          for (int i = lane; i < w; i += 32) {
            const T u = xp[i], v = xq[i];
            xp[i] = c * u - sn * v;
            xq[i] = sn * u + c * v;
          }
          T* jp = J + (int64_t)p * wp;
          T* jq = J + (int64_t)q * wp;
          for (int i = lane; i < wp; i += 32) {
            const T u = jp[i], v = jq[i];
            jp[i] = c * u - sn * v;
            jq[i] = sn * u + c * v;
          }
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    if (s_rot == 0) break;
    __syncthreads();
  }
  // singular values and descending order (stable insertion sort)
  for (int p = warp; p < wp; p += nwarps) {
    double a = 0.0;
    for (int i = lane; i < w; i += 32) a += (double)Xs[p * w + i] * (double)Xs[p * w + i];
    a = warp_sum(a);
    if (lane == 0) s_sig[p] = sqrt(a);
  }
  __syncthreads();
  if (tid == 0) {
    for (int p = 0; p < wp; ++p) s_order[p] = p;
    for (int p = 1; p < wp; ++p) {
      const int v = s_order[p];
      int j = p - 1;
      while (j >= 0 && s_sig[s_order[j]] < s_sig[v]) { s_order[j + 1] = s_order[j]; --j; }
      s_order[j + 1] = v;
    }
    if (sweep == max_sweeps && status) atomicCAS(status, 0, (int)BCUR_ETIMEOUT);
  }
  __syncthreads();
  for (int e = tid; e < ws * ws; e += blockDim.x) {
    const int i = e / ws, t = e % ws;
    const bool in = i < w && t < w;
    const int p = in ? s_order[t] : 0;
    const double sg = in ? s_sig[p] : 0.0;
    if (Ut) Ut[e] = (in && sg > 0.0) ? (T)((double)Xs[p * w + i] / sg) : T(0);
    if (W) W[e] = in ? J[(int64_t)p * wp + i] : T(i == t ? 1 : 0);
  }
  for (int t = tid; t < ws; t += blockDim.x) sigma[t] = t < w ? s_sig[s_order[t]] : 0.0;
}

template <typename T>
bcur_status_t jacobi_svd_small(const double* X, int w, T* Ut, T* W, double* sigma, T* jwork,
                               int* status, cudaStream_t s) {
  if (w < 1 || w > 128) return BCUR_EINVAL;
  const int wp = w + (w & 1);
  const size_t smem = (size_t)wp * w * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    BCUR_CUDA_TRY(cudaFuncSetAttribute(jacobi_svd_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024));
    attr_set = true;
  }
  const int warps = wp / 2 < 32 ? (wp / 2 < 1 ? 1 : wp / 2) : 32;
  jacobi_svd_kernel<T><<<1, warps * 32, smem, s>>>(X, w, Ut, W, sigma, jwork, status, nullptr);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

template <typename T>
bcur_status_t jacobi_svd_batched(const double* X, int w, T* Ut, T* W, double* sigma, T* jwork,
                                 int* status, int batch, cudaStream_t s, const int* wdim) {
  if (w < 2 || w > 128 || (w & 1) || batch < 1) return BCUR_EINVAL;
  const size_t smem = (size_t)w * w * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    BCUR_CUDA_TRY(cudaFuncSetAttribute(jacobi_svd_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024));
    attr_set = true;
  }
  const int warps = w / 2 < 32 ? w / 2 : 32;
  jacobi_svd_kernel<T><<<batch, warps * 32, smem, s>>>(X, w, Ut, W, sigma, jwork, status, wdim);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}
template bcur_status_t jacobi_svd_batched<float>(const double*, int, float*, float*, double*,
                                                 float*, int*, int, cudaStream_t, const int*);

// ---------------------------------------------------------------------------
// Blocked Cholesky pieces (working precision T)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void max_diag_kernel(const T* G, int64_t w, int64_t ldg, T* out, const int* run) {
  if (run && *run == 0) return;
  T mx = T(0);
  for (int64_t i = threadIdx.x; i < w; i += blockDim.x) mx = fmax(mx, G[i * ldg + i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ T r[32];
  if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    T m2 = T(0);
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m2 = fmax(m2, r[i]);
    *out = m2;
  }
}

template <typename T>
bcur_status_t max_diag(const T* G, int64_t w, int64_t ldg, T* out, cudaStream_t s,
                       const int* run) {
  max_diag_kernel<T><<<1, 1024, 0, s>>>(G, w, ldg, out, run);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

// Factor the diagonal block G[j0:j0+NB, j0:j0+NB] (lower part, already
// updated by the trailing updates) as L L^T with the drop rule, and write L
// and L^{-1} into the same block position of L and Linv (zeros above the
// diagonal); the arithmetic is potrf_leaf's.
template <typename T, int NB>
__global__ void __launch_bounds__(256) potrf_diag_kernel(const T* G, int64_t ldg, T* L, int64_t ldl,
                                                         T* Linv, int64_t ldi, int64_t j0,
                                                         const T* maxdiag, double tol_rel,
                                                         int* kept) {
  constexpr int TPR = 256 / NB;
  constexpr int LD = NB + TPR;
  extern __shared__ unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);  // NB x LD: L
  T* X = S + NB * LD;                      // NB x LD: L^{-1}
  const T tol = (T)(tol_rel * (double)(*maxdiag));
  const int nk = potrf_leaf<T, NB>(G + j0 * ldg + j0, ldg, S, X, tol);
  const int tid = threadIdx.x;
  const int i = tid / TPR, h = tid % TPR;
  for (int c = h; c < NB; c += TPR) {
    L[(j0 + i) * ldl + j0 + c] = (c <= i) ? S[i * LD + c] : T(0);
    Linv[(j0 + i) * ldi + j0 + c] = (c <= i) ? X[i * LD + c] : T(0);
  }
  if (tid == 0) atomicAdd(kept, nk);
}

template <typename T, int NB>
bcur_status_t potrf_diag_nb(T* G, int64_t ldg, T* L, int64_t ldl, T* Linv, int64_t ldi,
                            int64_t j0, const T* maxdiag, double tol_rel, int* kept,
                            cudaStream_t s) {
  const size_t smem = 2 * (size_t)NB * (NB + 256 / NB) * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    BCUR_CUDA_TRY(cudaFuncSetAttribute(potrf_diag_kernel<T, NB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  potrf_diag_kernel<T, NB><<<1, 256, smem, s>>>(G, ldg, L, ldl, Linv, ldi, j0, maxdiag, tol_rel,
                                                kept);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

template <typename T>
bcur_status_t potrf_diag(T* G, int64_t ldg, T* L, int64_t ldl, T* Linv, int64_t ldi, int64_t j0,
                         int nb, const T* maxdiag, double tol_rel, int* kept, cudaStream_t s) {
  if (nb == 128) return potrf_diag_nb<T, 128>(G, ldg, L, ldl, Linv, ldi, j0, maxdiag, tol_rel, kept, s);
  if (nb == 64) return potrf_diag_nb<T, 64>(G, ldg, L, ldl, Linv, ldi, j0, maxdiag, tol_rel, kept, s);
  return BCUR_EINVAL;
}

// ---------------------------------------------------------------------------
// One 64-column step of the blocked Cholesky G = L L^T (FP32, w x w, ld w,
// w a multiple of 64), left-looking inside the outer panel that starts at
// column J0 (the columns J0.. of G already carry the updates of the earlier
// outer panels).  With j1 = j0 + 64 and K = j0 - J0:
//   D  = G[j0:j1, j0:j1] - L[j0:j1, J0:j0] L[j0:j1, J0:j0]^T
//   L_jj = chol(D) with the drop rule, X = L_jj^{-1}        (leaf64_core)
//   L[R, j0:j1] = (G[R, j0:j1] - L[R, J0:j0] L[j0:j1, J0:j0]^T) X^T
// for the 64-row blocks R below j1.  CTA b handles rows j0 + 64 b; every CTA
// factors D itself (the same arithmetic in each, so every copy of X is the
// same), CTA 0 writes L_jj and X into L and Linv and adds its kept pivots.
// One launch per step replaces the leaf, panel solve, split and inner
// trailing update of the right-looking order; the products are exact FP32.
// ---------------------------------------------------------------------------
namespace {
constexpr int kStepLD = 68;   // leaf tiles S and X; k-major product tiles
constexpr int kStepKC = 32;   // K chunk of the products

// acc += A B^T for 64 x 64 outputs, A = 64 rows of Ab, B = 64 rows of Bb (row
// major, ld), K a multiple of 32.  The K chunk goes to shared memory k-major
// (As[k][row], ld 68) so that thread (ty, tx) = (tid / 16, tid % 16), which
// holds rows 4 ty.. and columns 4 tx.., reads two float4 per k.  The next
// chunk is loaded into registers while the current one is multiplied.
__device__ void step_prod64(const float* Ab, const float* Bb, int64_t ld, int K, float (&acc)[4][4],
                            float* As, float* Bs) {
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  if (K <= 0) return;
  float ra[8], rb[8];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q, r = e >> 5, c = e & 31;
      ra[q] = Ab[(int64_t)r * ld + k0 + c];
      rb[q] = Bb[(int64_t)r * ld + k0 + c];
    }
  };
  fetch(0);
  for (int k0 = 0; k0 < K; k0 += kStepKC) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q, r = e >> 5, c = e & 31;
      As[c * kStepLD + r] = ra[q];
      Bs[c * kStepLD + r] = rb[q];
    }
    __syncthreads();
    if (k0 + kStepKC < K) fetch(k0 + kStepKC);
#pragma unroll 8
    for (int k = 0; k < kStepKC; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&As[k * kStepLD + 4 * ty]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[k * kStepLD + 4 * tx]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
}
}  // namespace

__global__ void __launch_bounds__(256) chol_step_kernel(const float* G, int64_t w, float* L,
                                                        float* Linv, int64_t J0, int64_t j0,
                                                        const float* maxdiag, double tol_rel,
                                                        int* kept, const int* run) {
  // a gated step (run reads 0) does nothing; the flag was written before the
  // first step of the factorisation was launched, so every CTA of every step
  // reads the same value
  if (run && *run == 0) return;
  extern __shared__ __align__(16) float step_smem[];
  float* S = step_smem;                     // 64 x 68: D, then L_jj; then X^T
  float* X = S + 64 * kStepLD;              // 64 x 68: L_jj^{-1}
  float* As = X + 64 * kStepLD;             // 32 x 68 (k-major)
  float* Bs = As + kStepKC * kStepLD;       // 32 x 68
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int K = (int)(j0 - J0);
  // Columns J0 .. j0-64 of L were written by the steps before the previous
  // one, the last 64 by the previous step.  Launched as a programmatic
  // dependent of the previous step, this kernel forms the products over the
  // older columns while that step is still running, then waits for it
  // (griddepcontrol.wait: the previous grid has completed and its writes are
  // visible; a no-op for an ordinary launch) and adds the last 64 columns.
  // The next step may start once every CTA of this one has passed the wait,
  // so that its early products only read columns complete by then.
  const int K0 = K >= 64 ? K - 64 : 0;
  const float* Ljj = L + j0 * w + J0;       // rows j0.., columns J0..j0
  const int64_t r0 = j0 + 64 * (int64_t)blockIdx.x;
  float acc[4][4] = {};
  float accp[4][4] = {};
  step_prod64(Ljj, Ljj, w, K0, acc, As, Bs);
  if (blockIdx.x != 0) step_prod64(L + r0 * w + J0, Ljj, w, K0, accp, As, Bs);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  step_prod64(Ljj + K0, Ljj + K0, w, K - K0, acc, As, Bs);
  const float tol = (float)(tol_rel * (double)(*maxdiag));
  // D, every CTA
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = 4 * ty + i;
    const float4 g = *reinterpret_cast<const float4*>(&G[(j0 + r) * w + j0 + 4 * tx]);
    const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 4 * tx + j;
      S[r * kStepLD + c] = (c <= r) ? gv[j] - acc[i][j] : 0.f;
      X[r * kStepLD + c] = 0.f;
    }
  }
  __syncthreads();
  const int nk = leaf64_core(S, X, tol);
  if (blockIdx.x == 0) {
    for (int e = tid; e < 64 * 64; e += 256) {
      const int r = e >> 6, c = e & 63;
      L[(j0 + r) * w + j0 + c] = (c <= r) ? S[r * kStepLD + c] : 0.f;
      Linv[(j0 + r) * w + j0 + c] = (c <= r) ? X[r * kStepLD + c] : 0.f;
    }
    if (tid == 0) atomicAdd(kept, nk);
    return;
  }
  // the panel rows of this CTA
  step_prod64(L + r0 * w + J0 + K0, Ljj + K0, w, K - K0, accp, As, Bs);
  // P^T (k-major over As and Bs, 64 x 68) and X^T (over S, no longer needed)
  float* PT = As;
  float* XT = S;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = 4 * ty + i;
    const float4 g = *reinterpret_cast<const float4*>(&G[(r0 + r) * w + j0 + 4 * tx]);
    const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) PT[(4 * tx + j) * kStepLD + r] = gv[j] - accp[i][j];
  }
  for (int e = tid; e < 64 * 64; e += 256) {
    const int c = e >> 6, t = e & 63;
    XT[t * kStepLD + c] = X[c * kStepLD + t];
  }
  __syncthreads();
  // L[R, j0:j1] = P X^T (X lower: X[c][t] = 0 for t > c)
  float o[4][4] = {};
#pragma unroll 8
  for (int t = 0; t < 64; ++t) {
    const float4 a = *reinterpret_cast<const float4*>(&PT[t * kStepLD + 4 * ty]);
    const float4 b = *reinterpret_cast<const float4*>(&XT[t * kStepLD + 4 * tx]);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) o[i][j] = fmaf(av[i], bv[j], o[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
    *reinterpret_cast<float4*>(&L[(r0 + 4 * ty + i) * w + j0 + 4 * tx]) =
        make_float4(o[i][0], o[i][1], o[i][2], o[i][3]);
}

size_t chol_step_smem() {
  return (size_t)(2 * 64 * kStepLD + 2 * kStepKC * kStepLD) * sizeof(float);
}

bcur_status_t chol_step(const float* G, int64_t w, float* L, float* Linv, int64_t J0, int64_t j0,
                        const float* maxdiag, double tol_rel, int* kept, cudaStream_t s,
                        const int* run) {
  if (w % 64 != 0 || j0 % 64 != 0 || J0 > j0 || (j0 - J0) % 64 != 0 || j0 + 64 > w)
    return BCUR_EINVAL;
  static bool attr_set = false;
  if (!attr_set) {
    BCUR_CUDA_TRY(cudaFuncSetAttribute(chol_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)chol_step_smem()));
    attr_set = true;
  }
  const unsigned blocks = (unsigned)((w - j0) / 64);
  // A step after the first of an outer panel follows the previous step in the
  // stream: it is launched as that step's programmatic dependent (see the
  // kernel); the first step of a panel follows other work and waits for it.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = chol_step_smem();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = j0 > J0 ? 1 : 0;
  BCUR_CUDA_TRY(cudaLaunchKernelEx(&cfg, chol_step_kernel, G, w, L, Linv, J0, j0, maxdiag, tol_rel,
                                   kept, run));
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

// ---------------------------------------------------------------------------
// Block leverage scores (Def. 2): one thread-block cluster of kScoreCtas CTAs
// per block g.  CTA q of the cluster sums F[j, t]^2 over its slice of the
// block's columns j (every row t; consecutive threads on consecutive j
// within a row piece, so each piece is a coalesced read) in FP64; the CTA's partial is formed
// in a fixed order (per thread, xor-tree per warp, warps in order), and CTA 0
// adds the cluster's partials in rank order through distributed shared
// memory, so the score does not depend on scheduling.
// ---------------------------------------------------------------------------
constexpr int kScoreCtas = 8;

template <typename T>
__global__ void __cluster_dims__(kScoreCtas, 1, 1) __launch_bounds__(256)
    block_scores_kernel(const T* Ft, int k, int64_t ldf, const int64_t* off, int G,
                        double* scores, int* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  for (int g = blockIdx.y; g < G; g += gridDim.y) {
  const int64_t j0 = off[g], size = off[g + 1] - off[g];
  const int64_t chunk = (size + kScoreCtas - 1) / kScoreCtas;
  const int64_t a = j0 + q * chunk, b = min(j0 + size, a + chunk);
  // the slice's k x len elements spread over all threads (a narrow slice
  // still gives every thread several independent loads in flight)
  const int len = b > a ? (int)(b - a) : 0;
  const int total = k * len;
  double acc = 0.0;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int t = e / len, j = e - t * len;
    const double v = (double)Ft[(int64_t)t * ldf + a + j];
    acc = fma(v, v, acc);
  }
  acc = warp_sum(acc);
  __shared__ double r[32];
  __shared__ double part;
  if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += r[w];
    part = sum;
  }
  cluster.sync();  // every CTA's partial is written
  if (q == 0 && threadIdx.x == 0) {
    double sum = 0.0;
    for (int c = 0; c < kScoreCtas; ++c) sum += *cluster.map_shared_rank(&part, c);
    scores[g] = sum;
    if (!isfinite(sum)) dev_set_status(status, (int)BCUR_ENONFINITE);
  }
  cluster.sync();  // the partials stay alive until CTA 0 has read them
  }
}

template <typename T>
bcur_status_t block_scores(const T* Ft, int k, int64_t h, int64_t ldf, const int64_t* off, int G,
                           double* scores, int* status, cudaStream_t s) {
  (void)h;
  if (G <= 0) return BCUR_OK;
  block_scores_kernel<T><<<dim3(kScoreCtas, (unsigned)std::min(G, 32768)), 256, 0, s>>>(
      Ft, k, ldf, off, G, scores, status);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

// mu = (m / k) max_i ||U_k^T e_i||^2 (Sec. 3.2): each thread forms the FP64
// squared norms of its columns of the panel U_k^T; the maximum is taken with
// an atomic max on the bit pattern (non-negative doubles order like their
// bits), so the result does not depend on the order.
template <typename T>
__global__ void incoherence_kernel(const T* Ut, int k, int64_t m, int64_t ld,
                                   unsigned long long* out_bits) {
  double mx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int t = 0; t < k; ++t) {
      const double v = (double)Ut[(int64_t)t * ld + i];
      acc = fma(v, v, acc);
    }
    mx = fmax(mx, acc);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out_bits, (unsigned long long)__double_as_longlong(mx));
}

__global__ void incoherence_finish_kernel(const unsigned long long* bits, double scale,
                                          double* out) {
  *out = scale * __longlong_as_double((long long)*bits);
}

template <typename T>
bcur_status_t incoherence(const T* Ut, int k, int64_t m, int64_t ld, double* out, void* scratch,
                          cudaStream_t s) {
  if (k < 1 || m < 1 || ld < m) return BCUR_EINVAL;
  unsigned long long* bits = static_cast<unsigned long long*>(scratch);
  BCUR_CUDA_TRY(cudaMemsetAsync(bits, 0, sizeof(*bits), s));
  const int blocks = (int)std::min<int64_t>((m + 255) / 256, 1024);
  incoherence_kernel<T><<<blocks, 256, 0, s>>>(Ut, k, m, ld, bits);
  BCUR_LAUNCH_CHECK();
  incoherence_finish_kernel<<<1, 1, 0, s>>>(bits, (double)m / (double)k, out);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}
template bcur_status_t incoherence<float>(const float*, int, int64_t, int64_t, double*, void*,
                                          cudaStream_t);
template bcur_status_t incoherence<double>(const double*, int, int64_t, int64_t, double*, void*,
                                           cudaStream_t);

// ---------------------------------------------------------------------------
// Inverse-CDF sampling, one thread: the arithmetic must be the sequential
// FP64 order of the oracle, so every add / multiply is an explicit
// round-to-nearest intrinsic (no contraction into FMA).
// ---------------------------------------------------------------------------
__global__ void sample_kernel(const double* scores, int G, const double* u, int g,
                              int replacement, int32_t* idx, double* prob) {
  extern __shared__ unsigned char remaining[];
  if (threadIdx.x != 0) return;
  sample_seq(scores, G, u, g, replacement, idx, prob, remaining);
}

bcur_status_t sample_blocks(const double* scores, int G, const double* u, int g, int replacement,
                            int32_t* idx, double* prob, cudaStream_t s) {
  if (G < 1 || G > 32768 || g < 0 || (!replacement && g > G)) return BCUR_EINVAL;
  if (g == 0) return BCUR_OK;
  sample_kernel<<<1, 32, G, s>>>(scores, G, u, g, replacement, idx, prob);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

// ---------------------------------------------------------------------------
// Block index expansion and gathers
// ---------------------------------------------------------------------------
__global__ void expand_blocks_kernel(const int32_t* idx, int g, const int64_t* off, int G,
                                     int64_t cap, int64_t* map, int64_t* count) {
  int64_t base = 0;
  for (int t = 0; t < g; ++t) {
    const int b = idx[t];
    const bool ok = (b >= 0 && b < G);
    const int64_t start = ok ? off[b] : 0;
    const int64_t size = ok ? off[b + 1] - off[b] : 0;
    for (int64_t e = threadIdx.x; e < size; e += blockDim.x)
      if (base + e < cap) map[base + e] = start + e;
    base += size;
  }
  for (int64_t e = base + threadIdx.x; e < cap; e += blockDim.x) map[e] = -1;
  if (threadIdx.x == 0) *count = base < cap ? base : cap;
}

bcur_status_t expand_blocks(const int32_t* idx, int g, const int64_t* off, int G, int64_t cap,
                            int64_t* map, int64_t* count, cudaStream_t s) {
  expand_blocks_kernel<<<1, 512, 0, s>>>(idx, g, off, G, cap, map, count);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

template <typename T>
__global__ void gather_cols_kernel(const T* A, int64_t lda, int64_t m, const int64_t* map,
                                   int64_t cap, T* Cp, int64_t ldp) {
  __shared__ T tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  const int x = threadIdx.x;
  const int64_t cc = c0 + x;
  const int64_t col = cc < cap ? map[cc] : -1;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t i = i0 + y;
    tile[y][x] = (col >= 0 && i < m) ? A[i * lda + col] : T(0);
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t c = c0 + y, i = i0 + x;
    if (c < cap && i < m) Cp[c * ldp + i] = tile[x][y];
  }
}

template <typename T>
bcur_status_t gather_cols_t(const T* A, int64_t lda, int64_t m, const int64_t* map, int64_t cap,
                            T* Cp, int64_t ldp, cudaStream_t s) {
  if (cap <= 0 || m <= 0) return BCUR_OK;
  if (ceil_div(cap, 32) > 65535) return BCUR_EINVAL;
  dim3 grid((unsigned)ceil_div(m, 32), (unsigned)ceil_div(cap, 32));
  gather_cols_kernel<T><<<grid, dim3(32, 8), 0, s>>>(A, lda, m, map, cap, Cp, ldp);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

template <typename T>
__global__ void gather_rows_kernel(const T* A, int64_t lda, int64_t n, const int64_t* map,
                                   T* R, int64_t ldr) {
  const int64_t rr = blockIdx.y;
  const int64_t row = map[rr];
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    R[rr * ldr + j] = row >= 0 ? A[row * lda + j] : T(0);
}

template <typename T>
bcur_status_t gather_rows(const T* A, int64_t lda, int64_t n, const int64_t* map, int64_t cap,
                          T* R, int64_t ldr, cudaStream_t s) {
  if (cap <= 0 || n <= 0) return BCUR_OK;
  if (cap > 65535) return BCUR_EINVAL;
  const int64_t gx = ceil_div(n, 256) < 8 ? ceil_div(n, 256) : 8;
  gather_rows_kernel<T><<<dim3((unsigned)gx, (unsigned)cap), 256, 0, s>>>(A, lda, n, map, R, ldr);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

// ---------------------------------------------------------------------------
// Elementwise helpers
// ---------------------------------------------------------------------------
template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin* in, Tout* out, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (Tout)in[e];
}

template <typename Tin, typename Tout>
bcur_status_t convert(const Tin* in, Tout* out, int64_t count, cudaStream_t s) {
  if (count <= 0) return BCUR_OK;
  const int64_t blocks = ceil_div(count, 256) < 4096 ? ceil_div(count, 256) : 4096;
  convert_kernel<Tin, Tout><<<(unsigned)blocks, 256, 0, s>>>(in, out, count);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

template <typename T>
bcur_status_t copy2d(const T* src, int64_t lds, T* dst, int64_t ldd, int64_t rows, int64_t cols,
                     cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return BCUR_OK;
  BCUR_CUDA_TRY(cudaMemcpy2DAsync(dst, ldd * sizeof(T), src, lds * sizeof(T), cols * sizeof(T),
                                  rows, cudaMemcpyDeviceToDevice, s));
  return BCUR_OK;
}

// Copy of `bytes` bytes by the SMs: 16 bytes per thread and step, many
// loads in flight per SM.  Used to bring a page-locked host buffer that is
// mapped into the device's address space into device memory with the SMs
// reading it over the host link (the copy engines are the alternative).
__global__ void __launch_bounds__(256) copy_bytes_kernel(const uint4* __restrict__ src,
                                                         uint4* __restrict__ dst, int64_t n16) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    const uint4 a = __ldcs(src + i), b = __ldcs(src + i + stride);
    const uint4 c = __ldcs(src + i + 2 * stride), d = __ldcs(src + i + 3 * stride);
    __stcs(dst + i, a);
    __stcs(dst + i + stride, b);
    __stcs(dst + i + 2 * stride, c);
    __stcs(dst + i + 3 * stride, d);
  }
  for (; i < n16; i += stride) __stcs(dst + i, __ldcs(src + i));
}

bcur_status_t copy_bytes_sm(const void* src, void* dst, size_t bytes, int sms, cudaStream_t s) {
  if (((uintptr_t)src | (uintptr_t)dst | bytes) & 15) return BCUR_EINVAL;
  const int64_t n16 = (int64_t)(bytes / 16);
  if (n16 == 0) return BCUR_OK;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(4 * (int64_t)sms,
                                                                 (n16 + 255) / 256));
  copy_bytes_kernel<<<blocks, 256, 0, s>>>(static_cast<const uint4*>(src),
                                           static_cast<uint4*>(dst), n16);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

bcur_status_t fill_zero(void* p, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return BCUR_OK;
  BCUR_CUDA_TRY(cudaMemsetAsync(p, 0, bytes, s));
  return BCUR_OK;
}

// Zero `head` bytes at p, then n16 16-byte words, then `tail` bytes, unless
// *run reads 0.
__global__ void fill_zero_if_kernel(unsigned char* p, int head, int64_t n16, int tail,
                                    const int* run) {
  if (*run == 0) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < head) p[t] = 0;
  uint4* w = reinterpret_cast<uint4*>(p + head);
  for (int64_t i = t; i < n16; i += (int64_t)gridDim.x * blockDim.x) w[i] = make_uint4(0u, 0u, 0u, 0u);
  if (t < tail) p[head + 16 * n16 + t] = 0;
}

bcur_status_t fill_zero_if(void* p, size_t bytes, const int* run, cudaStream_t s) {
  if (!run) return fill_zero(p, bytes, s);
  if (bytes == 0) return BCUR_OK;
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const int head = (int)std::min<size_t>(bytes, (16 - (a & 15)) & 15);
  const int64_t n16 = (int64_t)((bytes - head) / 16);
  const int tail = (int)(bytes - head - 16 * (size_t)n16);
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(n16, 256), 1024));
  fill_zero_if_kernel<<<(unsigned)blocks, 256, 0, s>>>(static_cast<unsigned char*>(p), head, n16,
                                                       tail, run);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

// ---------------------------------------------------------------------------
// Block stable rank (Sec. 3.2): per column block g of a factor F (given as its
// panel F^T, k x h), ratio_g = ||F_g||_F^2 / ||F_g||_2^2 with F_g the rows of F
// in block g.  The k x k Gram F_g^T F_g is formed in FP64 (one CTA per block);
// its largest eigenvalue (= ||F_g||_2^2) comes from the batched one-sided Jacobi
// kernel above, its trace is ||F_g||_F^2.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void block_gram_kernel(const T* Ft, int k, int64_t ldf, const int64_t* off,
                                  double* gram) {
  const int g = blockIdx.x;
  const int64_t j0 = off[g], j1 = off[g + 1];
  double* out = gram + (int64_t)g * k * k;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, b = e % k;
    double acc = 0.0;
    if (b <= a)
      for (int64_t j = j0; j < j1; ++j) acc = fma((double)Ft[a * ldf + j], (double)Ft[b * ldf + j], acc);
    out[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, b = e % k;
    if (b > a) out[e] = out[b * k + a];
  }
}

__global__ void stable_rank_finish_kernel(const double* gram, const double* sigma, int k, int G,
                                          double* ratio) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const double* Gg = gram + (int64_t)g * k * k;
  double tr = 0.0;
  for (int a = 0; a < k; ++a) tr += Gg[a * k + a];
  const double lmax = sigma[(int64_t)g * k];  // singular values of an SPD Gram = eigenvalues
  ratio[g] = (tr > 0.0 && lmax > 0.0) ? tr / lmax : nan("");
}

template <typename T>
bcur_status_t block_stable_rank(const T* Ft, int k, int64_t ldf, const int64_t* off, int G,
                                double* ratio, void* ws, size_t ws_bytes, cudaStream_t s) {
  const int kp = k + (k & 1);
  const size_t need = ((size_t)G * k * k + (size_t)G * k) * sizeof(double) +
                      (size_t)G * kp * kp * sizeof(double);
  if (!ws || ws_bytes < need) return BCUR_ENOMEM;
  if (k < 1 || k > 128 || G < 1) return BCUR_EINVAL;
  double* gram = static_cast<double*>(ws);
  double* sig = gram + (size_t)G * k * k;
  double* jw = sig + (size_t)G * k;
  block_gram_kernel<T><<<G, 256, 0, s>>>(Ft, k, ldf, off, gram);
  BCUR_LAUNCH_CHECK();
  const size_t smem = (size_t)kp * k * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    BCUR_CUDA_TRY(cudaFuncSetAttribute(jacobi_svd_kernel<double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024));
    attr_set = true;
  }
  const int warps = kp / 2 < 32 ? (kp / 2 < 1 ? 1 : kp / 2) : 32;
  jacobi_svd_kernel<double><<<G, warps * 32, smem, s>>>(gram, k, nullptr, nullptr, sig, jw,
                                                        nullptr, nullptr);
  BCUR_LAUNCH_CHECK();
  stable_rank_finish_kernel<<<(G + 127) / 128, 128, 0, s>>>(gram, sig, k, G, ratio);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

size_t block_stable_rank_workspace(int k, int G) {
  const int kp = k + (k & 1);
  return ((size_t)G * k * k + (size_t)G * k + (size_t)G * kp * kp) * sizeof(double);
}

// ---------------------------------------------------------------------------
// Row scaling X[i][:] *= s[i] (FP64 scale factors)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void scale_rows_by_kernel(T* X, int64_t rows, int64_t cols, int64_t ld, const double* sc) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    X[i * ld + j] = (T)((double)X[i * ld + j] * sc[i]);
  }
}

template <typename T>
bcur_status_t scale_rows_by(T* X, int64_t rows, int64_t cols, int64_t ld, const double* sc,
                            cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return BCUR_OK;
  const int64_t blocks = std::min<int64_t>(ceil_div(rows * cols, 256), 4096);
  scale_rows_by_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(X, rows, cols, ld, sc);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}
template bcur_status_t scale_rows_by<float>(float*, int64_t, int64_t, int64_t, const double*, cudaStream_t);
template bcur_status_t scale_rows_by<double>(double*, int64_t, int64_t, int64_t, const double*, cudaStream_t);

// ---------------------------------------------------------------------------
// FP32 -> FP8 e4m3, one scale per row
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) quant_rows_e4m3_kernel(const float* X, int64_t ldx,
                                                              int64_t rows, int64_t cols,
                                                              const float* pre, uint8_t* Q,
                                                              int64_t ldq, float* scale) {
  __shared__ float red[8];
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const float* xr = X + r * ldx;
    float mx = 0.f;
    for (int64_t j = threadIdx.x; j < cols; j += blockDim.x)
      mx = fmaxf(mx, fabsf(xr[j] * (pre ? pre[j] : 1.f)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    float amax = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) amax = fmaxf(amax, red[i]);
    const float sc = amax > 0.f ? amax / 448.f : 1.f;
    const float inv = 1.f / sc;
    if (threadIdx.x == 0) scale[r] = sc;
    uint8_t* qr = Q + r * ldq;
    for (int64_t j = threadIdx.x; j < cols; j += blockDim.x)
      qr[j] = (uint8_t)__nv_cvt_float_to_fp8(xr[j] * (pre ? pre[j] : 1.f) * inv, __NV_SATFINITE,
                                             __NV_E4M3);
    __syncthreads();
  }
}

bcur_status_t quant_rows_e4m3(const float* X, int64_t ldx, int64_t rows, int64_t cols,
                              const float* pre, uint8_t* Q, int64_t ldq, float* scale,
                              cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return BCUR_OK;
  const unsigned grid = (unsigned)std::min<int64_t>(rows, 1 << 20);
  quant_rows_e4m3_kernel<<<grid, 256, 0, s>>>(X, ldx, rows, cols, pre, Q, ldq, scale);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

// ---------------------------------------------------------------------------
// FP32 -> FP8 e4m3, one scale per 128 x 128 block, written twice (row-major
// and transposed, so that both products with A read K-major operands).  One
// CTA per block: the block's amax (fixed-order reduction), scale = amax / 448
// (1 for an all-zero block), then the quantised bytes through a shared tile.
// Interior blocks with 16-byte aligned rows move four elements per access.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) quant_blocks_e4m3_kernel(const float* X, int64_t ldx,
                                                                int64_t rows, int64_t cols,
                                                                uint8_t* Q, int64_t ldq,
                                                                uint8_t* QT, int64_t ldqt,
                                                                float* scale, int64_t lds,
                                                                int vec) {
  __shared__ __align__(16) uint8_t tile[128][132];
  __shared__ float red[8];
  const int64_t r0 = (int64_t)blockIdx.y * 128, c0 = (int64_t)blockIdx.x * 128;
  const int tid = threadIdx.x;
  const bool whole = vec && r0 + 128 <= rows && c0 + 128 <= cols;
  float mx = 0.f;
  if (whole) {
    for (int e = tid; e < 128 * 32; e += 256) {
      const int i = e >> 5, j4 = (e & 31) * 4;
      const float4 v = *reinterpret_cast<const float4*>(X + (r0 + i) * ldx + c0 + j4);
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
  } else {
    for (int e = tid; e < 128 * 128; e += 256) {
      const int i = e >> 7, j = e & 127;
      if (r0 + i < rows && c0 + j < cols) mx = fmaxf(mx, fabsf(X[(r0 + i) * ldx + c0 + j]));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  float amax = 0.f;
  for (int i = 0; i < 8; ++i) amax = fmaxf(amax, red[i]);
  const float sc = amax > 0.f ? amax / 448.f : 1.f;
  const float inv = 1.f / sc;
  if (tid == 0) scale[(int64_t)blockIdx.y * lds + blockIdx.x] = sc;
  auto q8 = [&](float x) {
    return (uint8_t)__nv_cvt_float_to_fp8(x * inv, __NV_SATFINITE, __NV_E4M3);
  };
  if (whole) {
    for (int e = tid; e < 128 * 32; e += 256) {
      const int i = e >> 5, j4 = (e & 31) * 4;
      const float4 v = *reinterpret_cast<const float4*>(X + (r0 + i) * ldx + c0 + j4);
      const uint8_t b0 = q8(v.x), b1 = q8(v.y), b2 = q8(v.z), b3 = q8(v.w);
      tile[i][j4] = b0; tile[i][j4 + 1] = b1; tile[i][j4 + 2] = b2; tile[i][j4 + 3] = b3;
      *reinterpret_cast<uint32_t*>(Q + (r0 + i) * ldq + c0 + j4) =
          (uint32_t)b0 | ((uint32_t)b1 << 8) | ((uint32_t)b2 << 16) | ((uint32_t)b3 << 24);
    }
  } else {
    for (int e = tid; e < 128 * 128; e += 256) {
      const int i = e >> 7, j = e & 127;
      const bool in = r0 + i < rows && c0 + j < cols;
      const uint8_t b = in ? q8(X[(r0 + i) * ldx + c0 + j]) : (uint8_t)0;
      tile[i][j] = b;
      if (in) Q[(r0 + i) * ldq + c0 + j] = b;
    }
  }
  __syncthreads();
  if (whole) {
    for (int e = tid; e < 128 * 32; e += 256) {
      const int j = e >> 5, i4 = (e & 31) * 4;
      *reinterpret_cast<uint32_t*>(QT + (c0 + j) * ldqt + r0 + i4) =
          (uint32_t)tile[i4][j] | ((uint32_t)tile[i4 + 1][j] << 8) |
          ((uint32_t)tile[i4 + 2][j] << 16) | ((uint32_t)tile[i4 + 3][j] << 24);
    }
  } else {
    for (int e = tid; e < 128 * 128; e += 256) {
      const int j = e >> 7, i = e & 127;
      if (c0 + j < cols && r0 + i < rows) QT[(c0 + j) * ldqt + r0 + i] = tile[i][j];
    }
  }
}

bcur_status_t quant_blocks_e4m3(const float* X, int64_t ldx, int64_t rows, int64_t cols,
                                uint8_t* Q, int64_t ldq, uint8_t* QT, int64_t ldqt, float* scale,
                                cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return BCUR_OK;
  const int64_t gr = ceil_div(rows, 128), gc = ceil_div(cols, 128);
  if (gr > 65535 || gc > INT32_MAX) return BCUR_EINVAL;
  const int vec = (ldx % 4 == 0) && (ldq % 4 == 0) && (ldqt % 4 == 0) &&
                  ((uintptr_t)X % 16 == 0) && ((uintptr_t)Q % 4 == 0) && ((uintptr_t)QT % 4 == 0);
  quant_blocks_e4m3_kernel<<<dim3((unsigned)gc, (unsigned)gr), 256, 0, s>>>(
      X, ldx, rows, cols, Q, ldq, QT, ldqt, scale, gc, vec);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

__global__ void transpose_u8_kernel(const uint8_t* Q, int64_t ldq, int64_t rows, int64_t cols,
                                    uint8_t* T, int64_t ldt) {
  __shared__ uint8_t tile[64][65];
  const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int i = e / 64, j = e % 64;
    tile[i][j] = (r0 + i < rows && c0 + j < cols) ? Q[(r0 + i) * ldq + c0 + j] : (uint8_t)0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int j = e / 64, i = e % 64;
    if (c0 + j < cols && r0 + i < rows) T[(c0 + j) * ldt + r0 + i] = tile[i][j];
  }
}

bcur_status_t transpose_u8(const uint8_t* Q, int64_t ldq, int64_t rows, int64_t cols, uint8_t* T,
                           int64_t ldt, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return BCUR_OK;
  if (ceil_div(rows, 64) > 65535) return BCUR_EINVAL;
  dim3 grid((unsigned)ceil_div(cols, 64), (unsigned)ceil_div(rows, 64));
  transpose_u8_kernel<<<grid, 256, 0, s>>>(Q, ldq, rows, cols, T, ldt);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

// ---------------------------------------------------------------------------
// FP32 -> BF16 hi/lo pairs
// ---------------------------------------------------------------------------
__global__ void split_bf16_kernel(const float* X, int64_t ldx, int64_t rows, int64_t cols,
                                  __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo, int vec4,
                                  int write_hi, const int* run_flag) {
  if (run_flag && *run_flag == 0) return;
  for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
    const float* xr = X + r * ldx;
    __nv_bfloat16* hr = hi + r * ldo;
    __nv_bfloat16* lr = lo ? lo + r * ldo : nullptr;
    if (vec4) {
      const int64_t n4 = cols / 4;
      for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n4;
           c += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = reinterpret_cast<const float4*>(xr)[c];
        const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y);
        const __nv_bfloat162 h23 = __floats2bfloat162_rn(v.z, v.w);
        if (write_hi) {
          reinterpret_cast<__nv_bfloat162*>(hr)[2 * c] = h01;
          reinterpret_cast<__nv_bfloat162*>(hr)[2 * c + 1] = h23;
        }
        if (lr) {
          const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
          reinterpret_cast<__nv_bfloat162*>(lr)[2 * c] = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
          reinterpret_cast<__nv_bfloat162*>(lr)[2 * c + 1] =
              __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
        }
      }
    } else {
      for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cols;
           c += (int64_t)gridDim.x * blockDim.x) {
        const float v = xr[c];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        if (write_hi) hr[c] = h;
        if (lr) lr[c] = __float2bfloat16_rn(v - __bfloat162float(h));
      }
    }
  }
}

bcur_status_t split_bf16(const float* X, int64_t ldx, int64_t rows, int64_t cols,
                         __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo, cudaStream_t s,
                         bool write_hi, const int* run_flag) {
  if (rows <= 0 || cols <= 0) return BCUR_OK;
  if (!hi && write_hi) return BCUR_EINVAL;
  if (!hi) hi = lo;  // not written; keeps the address arithmetic valid
  if (!hi) return BCUR_OK;
  const int vec4 = (cols % 4 == 0) && (ldx % 4 == 0) && (ldo % 4 == 0) &&
                   ((uintptr_t)X % 16 == 0) && ((uintptr_t)hi % 8 == 0) &&
                   (!lo || (uintptr_t)lo % 8 == 0);
  const int64_t per_row = vec4 ? cols / 4 : cols;
  const int64_t gx = std::min<int64_t>(ceil_div(per_row, 256), 64);
  const int64_t gy = std::min<int64_t>(rows, 65535 / std::max<int64_t>(1, 1));
  split_bf16_kernel<<<dim3((unsigned)gx, (unsigned)std::min<int64_t>(gy, 8192)), 256, 0, s>>>(
      X, ldx, rows, cols, hi, lo, ldo, vec4, write_hi ? 1 : 0, run_flag);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

// ---------------------------------------------------------------------------
// Gathers straight into BF16 pairs (the split-BF16 fit's operands): each
// element of A is read once and written once as hi = bf16(a), lo =
// bf16(a - hi), with no FP32 copy of C or R in between.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split2(float a, float b, __nv_bfloat162* h, __nv_bfloat162* l) {
  *h = __floats2bfloat162_rn(a, b);
  const float2 f = __bfloat1622float2(*h);
  *l = __floats2bfloat162_rn(a - f.x, b - f.y);
}

// R[rr][j] = A[map[rr]][j] as a pair (zero rows where map < 0).  vec: A rows
// 16-byte aligned (lda % 4 == 0, A aligned) and ldo % 4 == 0 (8-byte aligned
// outputs): four elements per thread, float4 in, two bf16x2 out per part.
__global__ void gather_rows_pair_kernel(const float* A, int64_t lda, int64_t n, const int64_t* map,
                                        __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo,
                                        int vec) {
  const int64_t rr = blockIdx.y;
  const int64_t row = map[rr];
  const float* src = A + (row >= 0 ? row : 0) * lda;
  __nv_bfloat16* dh = hi + rr * ldo;
  __nv_bfloat16* dl = lo ? lo + rr * ldo : nullptr;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  int64_t done = 0;
  if (vec) {
    const int64_t n4 = n / 4;
    for (int64_t q = tid; q < n4; q += nth) {
      const float4 v = row >= 0 ? __ldcs(reinterpret_cast<const float4*>(src) + q)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
      __nv_bfloat162 h[2], l[2];
      split2(v.x, v.y, &h[0], &l[0]);
      split2(v.z, v.w, &h[1], &l[1]);
      reinterpret_cast<uint2*>(dh)[q] = *reinterpret_cast<const uint2*>(h);
      if (dl) reinterpret_cast<uint2*>(dl)[q] = *reinterpret_cast<const uint2*>(l);
    }
    done = 4 * n4;
  }
  for (int64_t j = done + tid; j < n; j += nth) {
    const float a = row >= 0 ? src[j] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(a);
    dh[j] = h;
    if (dl) dl[j] = __float2bfloat16_rn(a - __bfloat162float(h));
  }
}

// C^T[cc][i] = A[i][map[cc]] as a pair, 64 x 64 tiles through shared memory.
// A tile whose 64 gathered columns are consecutive in A and start on a
// 16-byte boundary is read as float4 rows; other tiles (block boundaries
// inside the tile, blocks drawn out of order, ragged sizes) element by
// element.  Output rows past cap are not written; map < 0 gives zeros.
__global__ void __launch_bounds__(256) gather_cols_pair_kernel(const float* A, int64_t lda,
                                                               int64_t m, const int64_t* map,
                                                               int64_t cap, __nv_bfloat16* hi,
                                                               __nv_bfloat16* lo, int64_t ldo,
                                                               int a_vec) {
  __shared__ float t[64][65];
  const int64_t i0 = (int64_t)blockIdx.x * 64, cc0 = (int64_t)blockIdx.y * 64;
  const int tid = threadIdx.x;
  const int64_t c0 = map[cc0];
  int ok = a_vec && c0 >= 0 && (c0 % 4) == 0 && cc0 + 63 < cap;
  if (ok) ok = (map[cc0 + (tid & 63)] == c0 + (tid & 63));
  ok = __syncthreads_and(ok);
  if (ok) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int r = (tid >> 4) + 16 * it, q = tid & 15;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i0 + r < m) v = __ldcs(reinterpret_cast<const float4*>(A + (i0 + r) * lda + c0) + q);
      t[r][4 * q] = v.x;
      t[r][4 * q + 1] = v.y;
      t[r][4 * q + 2] = v.z;
      t[r][4 * q + 3] = v.w;
    }
  } else {
    for (int e = tid; e < 64 * 64; e += 256) {
      const int r = e >> 6, c = e & 63;
      const int64_t cc = cc0 + c, i = i0 + r;
      const int64_t col = cc < cap ? map[cc] : -1;
      t[r][c] = (col >= 0 && i < m) ? A[i * lda + col] : 0.f;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const int c = (tid >> 5) + 8 * it, ip = tid & 31;
    const int64_t cc = cc0 + c, i = i0 + 2 * ip;
    if (cc >= cap || i >= m) continue;
    __nv_bfloat16* dh = hi + cc * ldo + i;
    __nv_bfloat16* dl = lo ? lo + cc * ldo + i : nullptr;
    if (i + 1 < m) {
      __nv_bfloat162 h, l;
      split2(t[2 * ip][c], t[2 * ip + 1][c], &h, &l);
      *reinterpret_cast<__nv_bfloat162*>(dh) = h;
      if (dl) *reinterpret_cast<__nv_bfloat162*>(dl) = l;
    } else {
      const float a = t[2 * ip][c];
      const __nv_bfloat16 h = __float2bfloat16_rn(a);
      dh[0] = h;
      if (dl) dl[0] = __float2bfloat16_rn(a - __bfloat162float(h));
    }
  }
}

bcur_status_t gather_rows_pair(const float* A, int64_t lda, int64_t n, const int64_t* map,
                               int64_t cap, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo,
                               cudaStream_t s) {
  if (cap <= 0 || n <= 0) return BCUR_OK;
  if (cap > 65535) return BCUR_EINVAL;
  const int vec = (lda % 4 == 0) && ((uintptr_t)A % 16 == 0) && (ldo % 4 == 0) &&
                  ((uintptr_t)hi % 8 == 0) && (!lo || (uintptr_t)lo % 8 == 0);
  const int64_t per_row = vec ? n / 4 : n;
  const int64_t gx = std::max<int64_t>(1, std::min<int64_t>(ceil_div(per_row, 256), 16));
  gather_rows_pair_kernel<<<dim3((unsigned)gx, (unsigned)cap), 256, 0, s>>>(A, lda, n, map, hi,
                                                                            lo, ldo, vec);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

bcur_status_t gather_cols_pair(const float* A, int64_t lda, int64_t m, const int64_t* map,
                               int64_t cap, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo,
                               cudaStream_t s) {
  if (cap <= 0 || m <= 0) return BCUR_OK;
  if (ceil_div(cap, 64) > 65535 || ldo % 2 != 0 || (uintptr_t)hi % 4 != 0 ||
      (lo && (uintptr_t)lo % 4 != 0))
    return BCUR_EINVAL;
  const int a_vec = (lda % 4 == 0) && ((uintptr_t)A % 16 == 0);
  dim3 grid((unsigned)ceil_div(m, 64), (unsigned)ceil_div(cap, 64));
  gather_cols_pair_kernel<<<grid, 256, 0, s>>>(A, lda, m, map, cap, hi, lo, ldo, a_vec);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

// ---------------------------------------------------------------------------
// Instantiations
// ---------------------------------------------------------------------------
#define BCUR_INST(T)                                                                              \
  template bcur_status_t reduce_splits_f64<T>(const T*, int, int64_t, int64_t, double*,           \
                                              cudaStream_t);                                      \
  template bcur_status_t chol_small<T>(const double*, int, double, double*, double*, T*, int*,    \
                                       cudaStream_t);                                             \
  template bcur_status_t jacobi_svd_small<T>(const double*, int, T*, T*, double*, T*, int*,       \
                                             cudaStream_t);                                       \
  template bcur_status_t max_diag<T>(const T*, int64_t, int64_t, T*, cudaStream_t, const int*);               \
  template bcur_status_t potrf_diag<T>(T*, int64_t, T*, int64_t, T*, int64_t, int64_t, int,       \
                                       const T*, double, int*, cudaStream_t);                     \
  template bcur_status_t block_scores<T>(const T*, int, int64_t, int64_t, const int64_t*, int,    \
                                         double*, int*, cudaStream_t);                            \
  template bcur_status_t gather_cols_t<T>(const T*, int64_t, int64_t, const int64_t*, int64_t,    \
                                          T*, int64_t, cudaStream_t);                             \
  template bcur_status_t gather_rows<T>(const T*, int64_t, int64_t, const int64_t*, int64_t, T*,  \
                                        int64_t, cudaStream_t);                                   \
  template bcur_status_t copy2d<T>(const T*, int64_t, T*, int64_t, int64_t, int64_t, cudaStream_t);
BCUR_INST(float)
BCUR_INST(double)
template bcur_status_t block_stable_rank<float>(const float*, int, int64_t, const int64_t*, int,
                                                double*, void*, size_t, cudaStream_t);
template bcur_status_t block_stable_rank<double>(const double*, int, int64_t, const int64_t*, int,
                                                 double*, void*, size_t, cudaStream_t);
template bcur_status_t convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template bcur_status_t convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template bcur_status_t convert<double, double>(const double*, double*, int64_t, cudaStream_t);
template bcur_status_t convert<float, float>(const float*, float*, int64_t, cudaStream_t);

}  // namespace bcur
