// Internal launchers shared between the translation units of the library.
#pragma once

#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"

namespace bcur {

// ---------------------------------------------------------------------------
// Dense GEMM on CUDA cores (FP32 / FP64):  D = alpha * A_op B_op + beta * D.
//   A_op(i, kk) = transA ? A[kk*lda + i] : A[i*lda + kk]     (M x K)
//   B_op(kk, j) = transB ? B[j*ldb + kk] : B[kk*ldb + j]     (K x N)
// Triangular operands (stored with explicit zeros) only narrow the K loop:
//   tri = 1: lower (A_op(i,kk) = 0 for kk > i;  B_op(kk,j) = 0 for kk < j)
//   tri = 2: upper (A_op(i,kk) = 0 for kk < i;  B_op(kk,j) = 0 for kk > j)
// batch > 1: independent problems at strides sA, sB, sD.
// ksplit > 1: K is cut into ksplit chunks; chunk z writes D + z*sD (partials).
// out_lower: only elements with i >= j are written (symmetric rank-k update).
// ---------------------------------------------------------------------------
struct GemmDesc {
  int64_t M = 0, N = 0, K = 0;
  const void* A = nullptr; int64_t lda = 0; int transA = 0;
  const void* B = nullptr; int64_t ldb = 0; int transB = 0;
  void* D = nullptr; int64_t ldd = 0;
  double alpha = 1.0, beta = 0.0;
  int64_t sA = 0, sB = 0, sD = 0;
  int batch = 1;
  int ksplit = 1;
  int triA = 0, triB = 0;
  int out_lower = 0;
  // Residual epilogue: accumulate sum (X - alpha*A_op B_op)^2 and sum X^2 per
  // CTA into partials[2 * cta] (FP64), instead of storing D.
  const void* X = nullptr; int64_t ldx = 0; double* partials = nullptr;
  // Optional device scratch the tensor-core path may use for split-K
  // partial slices, and a status word for device-detected errors.
  void* scratch = nullptr; size_t scratch_bytes = 0;
  int* status = nullptr;
  // A and B are stored as BF16 (tensor-core BF16 path only).  With parts = 3
  // the operands are BF16 pairs (A = hi, A_lo = lo; same for B) and the
  // product is A_hi B_hi + A_hi B_lo + A_lo B_hi.  D (FP32) and/or the BF16
  // pair Dh, Dl (same layout and ldd as D) receive the result.
  int ab_bf16 = 0;
  int parts = 1;
  const void* A_lo = nullptr;
  const void* B_lo = nullptr;
  void* Dh = nullptr;
  void* Dl = nullptr;
  // Optional device flag: when it reads 0 at launch the GEMM does nothing
  // (tensor-core path; in a grouped launch per GEMM).
  const int* run_flag = nullptr;
  // Optional device flag for a split product (parts = 3): when it reads 0 at
  // launch the product is taken with one term, A_hi B_hi.
  const int* parts_flag = nullptr;
  // FP8 e4m3 operands (prec BCUR_FP8; A and B K-major, one term), and
  // optional per-row (M) / per-column (N) factors of the result, applied
  // after alpha (tensor-core store only).
  int ab_fp8 = 0;
  const float* scale_m = nullptr;
  const float* scale_n = nullptr;
  // FP8 only: one factor per 128 x 128 block of op(B) seen as N x K (the
  // block holding column j and K index k has factor
  // bscale_b[(j / 128) * bs_n + (k / 128) * bs_k]); each 128-deep K block's
  // product is scaled by it before it is added (store epilogue, FP32 D,
  // M < 128 with N >= 2M so that the product runs transposed).
  const float* bscale_b = nullptr;
  int64_t bs_n = 0, bs_k = 0;
};

template <typename T> bcur_status_t gemm_simt(const GemmDesc& d, cudaStream_t s);
template <typename T> bcur_status_t gemm_simt_resid(const GemmDesc& d, cudaStream_t s,
                                                    int64_t* n_partials);
template <typename T> int64_t gemm_simt_resid_ctas(int64_t M, int64_t N);

// tcgen05 tensor-core GEMM (FP32 storage; TF32 or BF16 arithmetic).  Returns
// BCUR_ENOTSUP for shapes / layouts it does not cover.
bcur_status_t gemm_tc(const GemmDesc& d, int prec, cudaStream_t s);
bcur_status_t gemm_tc_resid(const GemmDesc& d, int prec, cudaStream_t s, int64_t* n_partials);
int64_t gemm_tc_resid_ctas(int64_t M, int64_t N);
bool gemm_tc_available();
// Bound of the tensor-core kernels' main-loop waits on the current device.
bcur_status_t gemm_tc_set_wait_budget(uint64_t ns);

// Grouped tensor-core GEMM: many BF16 GEMMs of different shapes in one
// persistent launch.  The table (tensor maps + parameters per GEMM, tile
// prefix sums) is encoded on the host and copied to `dev` once
// on the `setup` stream, synchronising only that stream; running it is one
// launch.  BN = 0 picks the tile width
// with the least padded work.  resid = 1: every GEMM reduces
// sum (X - A_op B_op)^2 and sum X^2 per (tile, epilogue warp) into
// d.partials[2 * (kResidSlots * tile + warp) + {0, 1}], tiles numbered as
// gemm_tc_units counts them (the launch order does not change the sums).
// Slots of residual partial pairs per tile (one per epilogue warp).
constexpr int kResidSlots = 8;
struct TcGroup {
  int BN = 0, epi = 0, count = 0, total = 0, grid = 0;
  void* table = nullptr;
  const int* starts = nullptr;
  int* status = nullptr;
};
size_t gemm_tc_group_bytes(int count);
bcur_status_t gemm_tc_group_prepare(const GemmDesc* ds, int count, int resid, int BN, void* dev,
                                    size_t bytes, int* status, TcGroup* out, cudaStream_t setup);
bcur_status_t gemm_tc_group_run(const TcGroup& g, cudaStream_t s, int grid = 0);
// Set the residual reference X of every GEMM of a prepared group from a
// device table: GEMM j (in the order given to prepare) reads the pointer at
// base + j * stride + offset.  One small launch.
bcur_status_t gemm_tc_group_patch_x(const TcGroup& g, const void* base, size_t stride,
                                    size_t offset, cudaStream_t s);
int64_t gemm_tc_units(const GemmDesc& d, int resid, int BN);

// Tile-width autotuner of the grouped GEMMs (autotune.cu).  For each GEMM of
// a stage, the width to use: from the tuning table (keyed by the stage name
// and the GEMM's own shape class), measured on a miss when measuring is on
// and `table` has room for a grouped launch of copies of the GEMM, otherwise
// the fixed choice by output width.  Synchronises `stream` when it measures.
struct TuneScratch {
  void* table = nullptr;      // device memory for the measuring launches' tables
  size_t table_bytes = 0;
  int* status = nullptr;
  cudaStream_t stream = nullptr;
  int sms = 148;
};
bcur_status_t tune_widths(const char* stage, const std::vector<GemmDesc>& ds, int resid,
                          const std::vector<int>& cands, const TuneScratch& sc,
                          std::vector<int>* out);
int tune_fixed_bn(const GemmDesc& d, int resid);

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------
// out[e] = sum_{s < nsplit} part[s*stride + e], FP64, fixed order.
template <typename T>
bcur_status_t reduce_splits_f64(const T* part, int nsplit, int64_t stride, int64_t count,
                                double* out, cudaStream_t s);

// Cholesky G = L L^T of a small SPD matrix (w <= 128) in FP64, with the drop
// rule (pivot <= tol_rel * max diag -> direction dropped), plus L^{-1}.
// Writes L and Linv (w x w, ld w, zeros above the diagonal) in FP64 and in T;
// kept[0] = number of kept pivots.
template <typename T>
bcur_status_t chol_small(const double* G, int w, double tol_rel, double* L64, double* Linv64,
                         T* LinvT, int* kept, cudaStream_t s);

// Lc = La * Lb for lower-triangular w x w FP64 matrices (w <= 128).
bcur_status_t trmm_small_f64(const double* La, const double* Lb, int w, double* Lc,
                             cudaStream_t s);

// One-sided Jacobi SVD of a w x w matrix X (given in FP64, ld w), computed in
// T (w <= 128): X = Ut diag(sigma) W^T, sigma descending.  Ut, W: w x w
// row-major in T; sigma: FP64.  jwork: device scratch, w*w T elements.
template <typename T>
bcur_status_t jacobi_svd_small(const double* X, int w, T* Ut, T* W, double* sigma, T* jwork,
                               int* status, cudaStream_t s);

// Blocked pieces of the wide Cholesky-QR.  run (optional device flag): when
// it reads 0 at launch the kernel does nothing.
template <typename T>
bcur_status_t max_diag(const T* G, int64_t w, int64_t ldg, T* out, cudaStream_t s,
                       const int* run = nullptr);
template <typename T>
bcur_status_t potrf_diag(T* G, int64_t ldg, T* L, int64_t ldl, T* Linv, int64_t ldi, int64_t j0,
                         int nb, const T* maxdiag, double tol_rel, int* kept, cudaStream_t s);
// One left-looking 64-column step of the blocked FP32 Cholesky (see small.cu):
// L[j0:, j0:j0+64] and Linv's diagonal block from G and L[:, J0:j0].
bcur_status_t chol_step(const float* G, int64_t w, float* L, float* Linv, int64_t J0, int64_t j0,
                        const float* maxdiag, double tol_rel, int* kept, cudaStream_t s,
                        const int* run = nullptr);

// Block leverage scores from a panel F^T (k x h).
template <typename T>
bcur_status_t block_scores(const T* Ft, int k, int64_t h, int64_t ldf, const int64_t* off,
                           int G, double* scores, int* status, cudaStream_t s);

// mu = (m / k) max_i ||U_k^T e_i||^2 from the panel U_k^T (k x m, ld); out is
// one device double; scratch: 8 bytes of device memory.
template <typename T>
bcur_status_t incoherence(const T* Ut, int k, int64_t m, int64_t ld, double* out, void* scratch,
                          cudaStream_t s);

// Per-block ||F_g||_F^2 / ||F_g||_2^2 (block stable rank terms, Sec. 3.2).
template <typename T>
bcur_status_t block_stable_rank(const T* Ft, int k, int64_t ldf, const int64_t* off, int G,
                                double* ratio, void* ws, size_t ws_bytes, cudaStream_t s);
size_t block_stable_rank_workspace(int k, int G);

bcur_status_t sample_blocks(const double* scores, int G, const double* u, int g, int replacement,
                            int32_t* idx, double* prob, cudaStream_t s);

// Expand block indices into an index map of length cap (entries past the
// chosen total are -1); total written to *count.
bcur_status_t expand_blocks(const int32_t* idx, int g, const int64_t* off, int G, int64_t cap,
                            int64_t* map, int64_t* count, cudaStream_t s);

// Cp[cc][i] = A[i][map[cc]] (0 where map < 0); Cp is cap x ldc_rows (ld ldp).
template <typename T>
bcur_status_t gather_cols_t(const T* A, int64_t lda, int64_t m, const int64_t* map, int64_t cap,
                            T* Cp, int64_t ldp, cudaStream_t s);
// R[rr][j] = A[map[rr]][j] (0 where map < 0).
template <typename T>
bcur_status_t gather_rows(const T* A, int64_t lda, int64_t n, const int64_t* map, int64_t cap,
                          T* R, int64_t ldr, cudaStream_t s);

// Fixed-order FP64 reduction of residual partials: out = {sqrt(e2), sqrt(e2)/sqrt(x2), sqrt(x2)}
// (mode 0) or {e2, x2} (mode 1).  Mode 2: as mode 0 from a one-term BF16
// residual, and *flag = whether that residual is too coarse (see
// residual_needs_refine); mode 3: as mode 0, written only when *flag != 0.
bcur_status_t finish_residual(const double* partials, int64_t n, double* out, int mode,
                              cudaStream_t s, int* flag = nullptr);
// out[0..2] = *flag ? r1[0..2] : r0[0..2] (device pointers).
bcur_status_t select_result(const double* r0, const double* r1, const int* flag, double* out,
                            cudaStream_t s);

template <typename Tin, typename Tout>
bcur_status_t convert(const Tin* in, Tout* out, int64_t count, cudaStream_t s);

// Copy a rows x cols sub-matrix (strided) on the device.
template <typename T>
bcur_status_t copy2d(const T* src, int64_t lds, T* dst, int64_t ldd, int64_t rows, int64_t cols,
                     cudaStream_t s);

bcur_status_t fill_zero(void* p, size_t bytes, cudaStream_t s);
// fill_zero that does nothing when the device flag *run reads 0 at launch
// (run NULL: always).
bcur_status_t fill_zero_if(void* p, size_t bytes, const int* run, cudaStream_t s);
// dst = src (bytes, both 16-byte aligned, bytes a multiple of 16) by the SMs;
// src may be mapped host memory.
bcur_status_t copy_bytes_sm(const void* src, void* dst, size_t bytes, int sms, cudaStream_t s);

// Boosting (boost.cu): the run with the smallest err[i * err_stride] among t
// runs laid out contiguously (first minimum in run order), its index in
// *best and copies of its outputs (U_bytes per run, g_col / g_row indices,
// the 3-double error).  Every output may be null.
bcur_status_t boost_select(int t, const double* err, int64_t err_stride, const void* U,
                           int64_t U_bytes, const int32_t* ci, int gc, const int32_t* ri, int gr,
                           void* U_best, int32_t* ci_best, int32_t* ri_best, double* err_best,
                           int32_t* best, cudaStream_t s);
// out = {sqrt(sum of partials_k's even entries), cur_err[0] / out[0]}.
bcur_status_t rank_k_ratio(const double* cur_err, const double* partials_k, int64_t n,
                           double* out, cudaStream_t s);

template <typename T>
bcur_status_t scale_rows_by(T* X, int64_t rows, int64_t cols, int64_t ld, const double* sc,
                            cudaStream_t s);

// Row-wise FP8 e4m3 quantisation of an FP32 matrix (rows x cols, ldx): with
// v_ij = X_ij * (pre ? pre[j] : 1), scale[i] = max_j |v_ij| / 448 (1 for an
// all-zero row) and Q[i][j] = e4m3(v_ij / scale[i]) (round to nearest,
// saturating), Q bytes with leading dimension ldq.
bcur_status_t quant_rows_e4m3(const float* X, int64_t ldx, int64_t rows, int64_t cols,
                              const float* pre, uint8_t* Q, int64_t ldq, float* scale,
                              cudaStream_t s);
// Blockwise FP8 e4m3 quantisation: for each 128 x 128 block (bi, bj) of X
// (rows x cols, ldx), scale[bi * ceil(cols/128) + bj] = block amax / 448 (1
// for an all-zero block) and Q[i][j] = QT[j][i] = e4m3(X_ij / scale of its
// block) (round to nearest, saturating); Q ld ldq, QT ld ldqt (bytes).
bcur_status_t quant_blocks_e4m3(const float* X, int64_t ldx, int64_t rows, int64_t cols,
                                uint8_t* Q, int64_t ldq, uint8_t* QT, int64_t ldqt, float* scale,
                                cudaStream_t s);
// Byte matrix transpose: T[j][i] = Q[i][j] (Q rows x cols, ldq; T ld ldt).
bcur_status_t transpose_u8(const uint8_t* Q, int64_t ldq, int64_t rows, int64_t cols, uint8_t* T,
                           int64_t ldt, cudaStream_t s);

// Gathers that write the BF16 pair (hi = bf16(a), lo = bf16(a - hi); lo may
// be null) directly: rows R[rr] = A[map[rr]] (R cap x n, ld ldo) and the
// transposed columns C^T[cc] = A[:, map[cc]] (C^T cap x m, ld ldo, even).
// Entries with map < 0 give zeros.
bcur_status_t gather_rows_pair(const float* A, int64_t lda, int64_t n, const int64_t* map,
                               int64_t cap, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo,
                               cudaStream_t s);
bcur_status_t gather_cols_pair(const float* A, int64_t lda, int64_t m, const int64_t* map,
                               int64_t cap, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo,
                               cudaStream_t s);

// Split an FP32 matrix (rows x cols, ldx) into BF16 pairs: hi = bf16(x),
// lo = bf16(x - hi) (round to nearest even both times); outputs have
// leading dimension ldo; lo may be null (hi only).
// write_hi false: only lo is written (hi may then be null); run_flag (device,
// optional): nothing is done when it reads 0 at launch.
bcur_status_t split_bf16(const float* X, int64_t ldx, int64_t rows, int64_t cols,
                         __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo, cudaStream_t s,
                         bool write_hi = true, const int* run_flag = nullptr);

}  // namespace bcur
