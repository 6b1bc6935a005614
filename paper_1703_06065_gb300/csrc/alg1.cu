// The paper's Algorithm 1 as printed (Sec. 3.1), on the GPU:
//   1. r rows drawn uniformly with replacement (p_i = 1/m), R = S_R^T A with
//      the scaling 1/sqrt(r p_i) = sqrt(m/r);
//   2. column-block scores l_i(R) = ||V_R^T E_i||_F^2 from an orthonormal basis
//      of the row space of R (Cholesky-QR2 of R; dropped pivots leave the
//      numerical row space), g blocks drawn with replacement from l / sum(l);
//   3. C = A S and W = R S with S's scaling 1/sqrt(g p_j); U = W^+ from the LQ
//      factorisation W = L Q_W (Cholesky-QR2 of W's rows): W^+ = Q_W^T L^{-1};
//   4. the residual ||A - C U R||_F.
// Arithmetic in the storage precision (FP64 or FP32) on CUDA cores; r <= 128.
#include <algorithm>

#include "kernels.h"

namespace bcur {
namespace {

__global__ void fill_f64_kernel(double* x, int64_t n, double v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

__global__ void iota_i64_kernel(int64_t* x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = i;
}

template <typename T>
__global__ void scale_region_kernel(T* x, int64_t rows, int64_t cols, int64_t ld, double s) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    x[i * ld + j] = (T)((double)x[i * ld + j] * s);
  }
}

// Per gathered column cc (draw order) the factor 1/sqrt(g p_t) of the draw it
// came from; 0 past the chosen total.
__global__ void draw_scales_kernel(const int32_t* idx, int g, const int64_t* off, const double* prob,
                                   int64_t cap, double* scale) {
  int64_t base = 0;
  for (int t = 0; t < g; ++t) {
    const int b = idx[t];
    const int64_t size = off[b + 1] - off[b];
    const double s = prob[t] > 0.0 ? 1.0 / sqrt((double)g * prob[t]) : 0.0;
    for (int64_t e = threadIdx.x; e < size; e += blockDim.x)
      if (base + e < cap) scale[base + e] = s;
    base += size;
  }
  for (int64_t e = base + threadIdx.x; e < cap; e += blockDim.x) scale[e] = 0.0;
}

template <typename T>
__global__ void scale_rows_kernel(T* x, int64_t rows, int64_t cols, int64_t ld, const double* s) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    x[i * ld + j] = (T)((double)x[i * ld + j] * s[i]);
  }
}

// W[i][cc] = R[i][map[cc]] * scale[cc] (0 where map < 0): columns of a
// row-major matrix gathered into a row-major result.
template <typename T>
__global__ void gather_cols_rm_kernel(const T* R, int64_t ldr, int64_t rows, const int64_t* map,
                                      const double* scale, int64_t cap, T* W, int64_t ldw) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * cap;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cap, cc = e % cap;
    const int64_t col = map[cc];
    W[i * ldw + cc] = col >= 0 ? (T)((double)R[i * ldr + col] * scale[cc]) : T(0);
  }
}

// Moore-Penrose inverse of a small square matrix from its SVD X = Ut S W^T
// (one-sided Jacobi): X^+ = W S^+ Ut^T, singular values at or below tol
// treated as zero.
template <typename T>
__global__ void pinv_from_svd_kernel(const double* Ut, const double* Wm, const double* sig, int w,
                                     double tol_rel, T* Xp) {
  const double tol = tol_rel * sig[0];
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < w * w; e += blockDim.x * gridDim.x) {
    const int i = e / w, j = e % w;
    double acc = 0.0;
    for (int t = 0; t < w; ++t)
      if (sig[t] > tol) acc += Wm[i * w + t] * Ut[j * w + t] / sig[t];
    Xp[e] = (T)acc;
  }
}

unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), 256), 4096); }

template <typename T> constexpr double eps_of() {
  return sizeof(T) == 8 ? 2.220446049250313e-16 : 1.1920928955078125e-07;
}

struct Alg1Layout {
  size_t ones, iota, row_prob, col_off, rowmap, colmap, counts, scale, Rp, Qp, tmp, gram_part, G64,
      La, Lb, Lprod, Linv64, LinvT, kept, Cp, W, W2, Ub, Pb, partials, SU, SW, Ssig, Sj, total;
  int64_t ldn, ldm, ldc, c_pad, r_pad;
  int ks_n, ks_c;
};

Alg1Layout layout(int64_t m, int64_t n, int G, int64_t c_max, int r, size_t esz) {
  Alg1Layout L{};
  size_t cur = 0;
  auto take = [&](size_t bytes) {
    const size_t at = cur;
    cur += (bytes + 255) / 256 * 256;
    return at;
  };
  L.ldn = round_up(n, 32);
  L.ldm = round_up(m, 32);
  L.c_pad = round_up(std::max<int64_t>(c_max, 1), 32);
  L.ldc = L.c_pad;
  L.r_pad = r;
  L.ks_n = (int)std::max<int64_t>(1, std::min<int64_t>(296, n / 64));
  L.ks_c = (int)std::max<int64_t>(1, std::min<int64_t>(296, L.c_pad / 64));
  const int64_t rr = (int64_t)r * r;
  L.ones = take(m * 8);
  L.iota = take((m + 1) * 8);
  L.row_prob = take(r * 8);
  L.col_off = take((G + 1) * 8);
  L.rowmap = take(r * 8);
  L.colmap = take(L.c_pad * 8);
  L.counts = take(16);
  L.scale = take(L.c_pad * 8);
  L.Rp = take(r * L.ldn * esz);
  L.Qp = take(r * L.ldn * esz);
  L.tmp = take(r * std::max(L.ldn, L.ldc) * esz);
  L.gram_part = take((size_t)std::max(L.ks_n, L.ks_c) * rr * esz);
  L.G64 = take(rr * 8);
  L.La = take(rr * 8);
  L.Lb = take(rr * 8);
  L.Lprod = take(rr * 8);
  L.Linv64 = take(rr * 8);
  L.LinvT = take(rr * esz);
  L.kept = take(16);
  L.Cp = take(L.c_pad * L.ldm * esz);
  L.W = take(r * L.ldc * esz);
  L.W2 = take(r * L.ldc * esz);
  L.Ub = take(L.c_pad * r * esz);
  L.Pb = take(m * r * esz);
  L.partials = take(2 * std::max(gemm_simt_resid_ctas<double>(m, n),
                                 gemm_simt_resid_ctas<float>(m, n)) * 8);
  L.SU = take(rr * 8);
  L.SW = take(rr * 8);
  L.Ssig = take(r * 8);
  L.Sj = take((int64_t)(r + 1) * (r + 1) * 8);
  L.total = cur;
  return L;
}

// Cholesky-QR2 of a panel X (w x h, ld), w <= 128: X <- Q, optionally L (FP64,
// X_in = L Q).  Gram by split-K in the working precision, reduced in FP64.
template <typename T>
bcur_status_t orth_rows(char* ws, const Alg1Layout& L, cudaStream_t s, T* X, T* tmp, int w,
                        int64_t h, int64_t ld, int ksplit, double* Lout) {
  T* gram_part = (T*)(ws + L.gram_part);
  double* Ls[2] = {(double*)(ws + L.La), (double*)(ws + L.Lb)};
  const double tol = sizeof(T) == 8 ? eps_of<T>() * std::max<double>(64.0, 2.0 * (double)h)
                                    : 64.0 * eps_of<T>();
  T* src = X;
  T* dst = tmp;
  for (int pass = 0; pass < 2; ++pass) {
    GemmDesc g;
    g.M = w; g.N = w; g.K = h;
    g.A = src; g.lda = ld; g.B = src; g.ldb = ld; g.transB = 1;
    g.D = gram_part; g.ldd = w;
    g.ksplit = ksplit;
    g.sD = (int64_t)w * w;
    BCUR_TRY(gemm_simt<T>(g, s));
    BCUR_TRY(reduce_splits_f64<T>(gram_part, ksplit, (int64_t)w * w, (int64_t)w * w,
                                  (double*)(ws + L.G64), s));
    BCUR_TRY(chol_small<T>((double*)(ws + L.G64), w, tol, Ls[pass], (double*)(ws + L.Linv64),
                           (T*)(ws + L.LinvT), (int*)(ws + L.kept), s));
    GemmDesc a;
    a.M = w; a.N = h; a.K = w;
    a.A = ws + L.LinvT; a.lda = w; a.triA = 1;
    a.B = src; a.ldb = ld;
    a.D = dst; a.ldd = ld;
    BCUR_TRY(gemm_simt<T>(a, s));
    std::swap(src, dst);
  }
  if (Lout) BCUR_TRY(trmm_small_f64(Ls[0], Ls[1], w, Lout, s));
  return BCUR_OK;
}

template <typename T>
bcur_status_t run_alg1(const T* A, int64_t lda, int64_t m, int64_t n, const int64_t* col_off_host,
                       int G, int r, int g, const double* u_rows, const double* u_cols,
                       int32_t* row_idx, int32_t* col_idx, double* col_scores, double* col_prob,
                       T* Uout, double* err, char* ws, const Alg1Layout& L, cudaStream_t s) {
  int64_t smax = 0;
  for (int i = 0; i < G; ++i) smax = std::max(smax, col_off_host[i + 1] - col_off_host[i]);
  const int64_t c_max = (int64_t)g * smax;
  double* ones = (double*)(ws + L.ones);
  int64_t* iota = (int64_t*)(ws + L.iota);
  int64_t* col_off = (int64_t*)(ws + L.col_off);
  int64_t* rowmap = (int64_t*)(ws + L.rowmap);
  int64_t* colmap = (int64_t*)(ws + L.colmap);
  int64_t* counts = (int64_t*)(ws + L.counts);
  double* scale = (double*)(ws + L.scale);
  double* rprob = (double*)(ws + L.row_prob);
  T* Rp = (T*)(ws + L.Rp);
  T* Qp = (T*)(ws + L.Qp);
  T* tmp = (T*)(ws + L.tmp);
  T* Cp = (T*)(ws + L.Cp);
  T* W = (T*)(ws + L.W);
  T* W2 = (T*)(ws + L.W2);
  T* Ub = (T*)(ws + L.Ub);
  T* Pb = (T*)(ws + L.Pb);
  BCUR_CUDA_TRY(cudaMemsetAsync(ws, 0, L.total, s));
  BCUR_CUDA_TRY(cudaMemcpyAsync(col_off, col_off_host, (G + 1) * sizeof(int64_t),
                                cudaMemcpyHostToDevice, s));
  // 1. rows, uniformly with replacement, and R = sqrt(m/r) A[rows, :]
  fill_f64_kernel<<<grid_for(m), 256, 0, s>>>(ones, m, 1.0);
  BCUR_LAUNCH_CHECK();
  iota_i64_kernel<<<grid_for(m + 1), 256, 0, s>>>(iota, m + 1);
  BCUR_LAUNCH_CHECK();
  BCUR_TRY(sample_blocks(ones, (int)m, u_rows, r, 1, row_idx, rprob, s));
  BCUR_TRY(expand_blocks(row_idx, r, iota, (int)m, r, rowmap, counts, s));
  BCUR_TRY(gather_rows<T>(A, lda, n, rowmap, r, Rp, L.ldn, s));
  scale_region_kernel<T><<<grid_for((int64_t)r * n), 256, 0, s>>>(Rp, r, n, L.ldn,
                                                                   sqrt((double)m / r));
  BCUR_LAUNCH_CHECK();
  // 2. orthonormal basis of row(R), block scores, g blocks with replacement
  BCUR_CUDA_TRY(cudaMemcpyAsync(Qp, Rp, (size_t)r * L.ldn * sizeof(T), cudaMemcpyDeviceToDevice, s));
  BCUR_TRY(orth_rows<T>(ws, L, s, Qp, tmp, r, n, L.ldn, L.ks_n, nullptr));
  BCUR_TRY(block_scores<T>(Qp, r, n, L.ldn, col_off, G, col_scores, nullptr, s));
  BCUR_TRY(sample_blocks(col_scores, G, u_cols, g, 1, col_idx, col_prob, s));
  BCUR_TRY(expand_blocks(col_idx, g, col_off, G, L.c_pad, colmap, counts + 1, s));
  draw_scales_kernel<<<1, 256, 0, s>>>(col_idx, g, col_off, col_prob, L.c_pad, scale);
  BCUR_LAUNCH_CHECK();
  // 3. C = A S (as its panel C^T), W = R S, U = W^+ = Q_W^T L^{-1}
  BCUR_TRY(gather_cols_t<T>(A, lda, m, colmap, L.c_pad, Cp, L.ldm, s));
  scale_rows_kernel<T><<<grid_for(L.c_pad * m), 256, 0, s>>>(Cp, L.c_pad, m, L.ldm, scale);
  BCUR_LAUNCH_CHECK();
  gather_cols_rm_kernel<T><<<grid_for((int64_t)r * L.c_pad), 256, 0, s>>>(Rp, L.ldn, r, colmap,
                                                                          scale, L.c_pad, W, L.ldc);
  BCUR_LAUNCH_CHECK();
  double* Lprod = (double*)(ws + L.Lprod);
  BCUR_TRY(orth_rows<T>(ws, L, s, W, W2, r, L.c_pad, L.ldc, L.ks_c, Lprod));
  // W = L Q_W with Q_W's kept rows orthonormal, so W^+ = Q_W^T L^+ exactly,
  // also when W is rank deficient (rows drawn twice, low-rank A).
  BCUR_TRY(jacobi_svd_small<double>(Lprod, r, (double*)(ws + L.SU), (double*)(ws + L.SW),
                                    (double*)(ws + L.Ssig), (double*)(ws + L.Sj), nullptr, s));
  pinv_from_svd_kernel<T><<<(r * r + 255) / 256, 256, 0, s>>>(
      (double*)(ws + L.SU), (double*)(ws + L.SW), (double*)(ws + L.Ssig), r,
      (double)std::max<int64_t>(r, c_max) * eps_of<T>(), (T*)(ws + L.LinvT));
  BCUR_LAUNCH_CHECK();
  GemmDesc gu;
  gu.M = L.c_pad; gu.N = r; gu.K = r;
  gu.A = W; gu.lda = L.ldc; gu.transA = 1;
  gu.B = ws + L.LinvT; gu.ldb = r;
  gu.D = Ub; gu.ldd = r;
  BCUR_TRY(gemm_simt<T>(gu, s));
  if (Uout) BCUR_TRY(copy2d<T>(Ub, r, Uout, r, c_max, r, s));
  // 4. residual ||A - (C U) R||_F
  GemmDesc gp;
  gp.M = m; gp.N = r; gp.K = L.c_pad;
  gp.A = Cp; gp.lda = L.ldm; gp.transA = 1;
  gp.B = Ub; gp.ldb = r;
  gp.D = Pb; gp.ldd = r;
  BCUR_TRY(gemm_simt<T>(gp, s));
  GemmDesc gr;
  gr.M = m; gr.N = n; gr.K = r;
  gr.A = Pb; gr.lda = r;
  gr.B = Rp; gr.ldb = L.ldn;
  gr.X = A; gr.ldx = lda;
  gr.partials = (double*)(ws + L.partials);
  int64_t np = 0;
  BCUR_TRY(gemm_simt_resid<T>(gr, s, &np));
  return finish_residual((double*)(ws + L.partials), np, err, 0, s);
}

int64_t c_max_of(const int64_t* off, int G, int g) {
  int64_t smax = 0;
  for (int i = 0; i < G; ++i) smax = std::max(smax, off[i + 1] - off[i]);
  return (int64_t)g * smax;
}

}  // namespace
}  // namespace bcur

using namespace bcur;

extern "C" size_t bcur_alg1_workspace(int64_t m, int64_t n, const int64_t* col_off, int32_t G,
                                      int32_t r, int32_t g, int32_t dtype) {
  if (!col_off || m < 1 || n < 1 || G < 1 || r < 1 || g < 1) return 0;
  return layout(m, n, G, c_max_of(col_off, G, g), r, dtype == BCUR_F64 ? 8 : 4).total;
}

extern "C" bcur_status_t bcur_alg1(const void* A, int64_t lda, int64_t m, int64_t n, int32_t dtype,
                                   const int64_t* col_off, int32_t G, int32_t r, int32_t g,
                                   const double* u_rows, const double* u_cols, int32_t* row_idx,
                                   int32_t* col_idx, double* col_scores, double* col_prob,
                                   void* U, double* err, void* workspace, size_t ws_bytes,
                                   void* stream) {
  if (!A || !col_off || !u_rows || !u_cols || !row_idx || !col_idx || !col_scores || !col_prob ||
      !err || !workspace)
    return BCUR_EINVAL;
  if (m < 1 || n < 1 || lda < n || r < 1 || r > 128 || r > m || g < 1 || G < 1 || G > 32768 ||
      m > 32768)
    return BCUR_EINVAL;
  if (col_off[0] != 0 || col_off[G] != n) return BCUR_EINVAL;
  for (int i = 0; i < G; ++i)
    if (col_off[i + 1] <= col_off[i]) return BCUR_EINVAL;
  const size_t esz = dtype == BCUR_F64 ? 8 : 4;
  if (dtype != BCUR_F64 && dtype != BCUR_F32) return BCUR_EINVAL;
  const Alg1Layout L = layout(m, n, G, c_max_of(col_off, G, g), r, esz);
  if (ws_bytes < L.total) return BCUR_ENOMEM;
  if ((uintptr_t)workspace & 255) return BCUR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == BCUR_F64)
    return run_alg1<double>((const double*)A, lda, m, n, col_off, G, r, g, u_rows, u_cols, row_idx,
                            col_idx, col_scores, col_prob, (double*)U, err, (char*)workspace, L, s);
  return run_alg1<float>((const float*)A, lda, m, n, col_off, G, r, g, u_rows, u_cols, row_idx,
                         col_idx, col_scores, col_prob, (float*)U, err, (char*)workspace, L, s);
}
