/*
 * bcur.h -- Block CUR decomposition hot path on NVIDIA GB300 (sm_103a).
 *
 * Method: Oswal, Jain, Xu, Eriksson, "Block CUR: Decomposing Matrices using
 * Groups of Columns" (arXiv 1703.06065).  Given A (m x n) with predefined
 * contiguous column blocks and row blocks (Sec. 3: G = ceil(n/s) blocks,
 * sizes may vary), the library computes
 *
 *   1. the top-k singular subspaces of A by a randomized range finder with
 *      q steps of subspace iteration on an n x l test matrix, l = k + p
 *      (the paper allows sketching in place of its score estimate, Sec. 3.1);
 *   2. block leverage scores l_g = ||V_{A,k}^T E_g||_F^2 (Def. 2) for column
 *      blocks, and the same quantity on U_{A,k} for row blocks (Sec. 3 applies
 *      the column rules to A^T);
 *   3. g_col column blocks and g_row row blocks drawn by inverse CDF from
 *      p_j = l_j / sum(l) (Alg. 1 step 2; without replacement by default, as in
 *      the experiments of Sec. 4.1);
 *   4. C = A[:, chosen column blocks], R = A[chosen row blocks, :] (Alg. 1);
 *   5. U = C^+ A R^+ through QR factors of C and R^T;
 *   6. ||A - CUR||_F and ||A - CUR||_F / ||A||_F (Sec. 4.2) without forming CUR.
 *
 * Conventions for every entry point:
 *   - Matrices are dense.  "row-major h x w, ld" means element (i, j) at
 *     base[i * ld + j].  A "panel" of a tall matrix X (h x w) is X^T stored
 *     row-major (w x h): each column of X is contiguous.
 *   - Pointers named in the comments as "device" must be CUDA device (or
 *     managed) memory on the current device; "host" pointers are read before
 *     the call returns.  The caller owns every buffer it passes; the library
 *     never frees caller memory.
 *   - All device work is enqueued on the plan's stream (or the `stream`
 *     argument, a cudaStream_t; NULL = legacy default stream) and the calls
 *     return without synchronising, unless stated otherwise.  Inputs must stay
 *     valid and unmodified until the stream has reached the call.
 *   - Host-detectable errors return immediately and enqueue nothing.  Errors
 *     the GPU detects (non-finite data, a wait that ran out) are recorded in a
 *     status word and returned by bcur_sync_status().
 *   - A plan is not thread-safe: use one plan per host thread and stream.
 */
#ifndef BCUR_H_
#define BCUR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BCUR_OK = 0,
  BCUR_EINVAL = 1,      /* invalid argument or descriptor                      */
  BCUR_ENOMEM = 2,      /* workspace missing or too small                      */
  BCUR_ECUDA = 3,       /* a CUDA runtime/driver call failed                   */
  BCUR_ERANK = 4,       /* a factorisation met a zero pivot it could not drop  */
  BCUR_ENONFINITE = 5,  /* NaN or Inf met in the data                          */
  BCUR_ETIMEOUT = 6,    /* a bounded device-side wait gave up                  */
  BCUR_ENOTSUP = 7,     /* combination not supported by the library / device  */
  BCUR_ESTATE = 8       /* call out of order (e.g. bcur_fit before a workspace) */
} bcur_status_t;

/* Storage type of A and arithmetic of a stage.
 *   BCUR_F64    : FP64 storage and FP64 arithmetic everywhere.
 *   BCUR_F32    : FP32 arithmetic on CUDA cores (FP32 storage).
 *   BCUR_TF32   : tcgen05 tensor cores reading FP32 storage as TF32 (bcur_gemm
 *                 only, both operands K-major; plans refuse it).
 *   BCUR_BF16   : tcgen05 tensor cores on BF16 roundings of the FP32 operands,
 *                 FP32 accumulation in tensor memory (about 8 mantissa bits).
 *   BCUR_BF16X3 : tcgen05 tensor cores on BF16 hi/lo pairs, x = hi + lo, with
 *                 A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (about 16 bits).
 *   BCUR_FP8    : sketch only (FP32 storage): tcgen05 kind::f8f6f4 on e4m3
 *                 roughly 4-bit operands, A scaled per row and each skinny
 *                 panel per row (amax / 448), the scales undone exactly in
 *                 the products' epilogue; FP32 accumulation.
 *   BCUR_FP8B   : sketch only (FP32 storage): as BCUR_FP8, with one scale
 *                 per 128 x 128 block of A (block amax / 448) instead of per
 *                 row; each 128-deep K block of a product with A is scaled by
 *                 its block's factor as it is summed (FP32), the panels keep
 *                 their per-row scales.
 *   BCUR_BF16X3A: fit only (FP32 storage), adaptive: the first pass of
 *                 the Cholesky-QR of C and R^T as BCUR_BF16X3; the second
 *                 pass (the Gram of the first pass's factor, near I, and its
 *                 Cholesky factor), the core products (W = A Q_R,
 *                 M = Q_C^T W and the triangular products that turn M into
 *                 U) and the residual ||A - CUR||_F first with one BF16 term
 *                 each, all taken by bcur_fit.  When that residual is too
 *                 coarse for the relative error e it reports, i.e. when one
 *                 term's rounding (2^-8) could move e by more than 2.5e-4
 *                 ((2^-8)^2 / (2 e) > 2.5e-4, e < 0.031), the device redoes
 *                 the second pass (when the factor widths are multiples of
 *                 64), the same products and the residual with three terms.
 *                 e depends on errors in M and in the second pass's factor
 *                 only at second order (their contribution Q_C dM Q_R^T is
 *                 orthogonal to A - Q_C M Q_R^T);
 *                 U at first order, so with one term U carries BF16 rounding
 *                 amplified by the conditioning of C and R.  bcur_fit_terms
 *                 reports the choice; bcur_error returns the fit's residual. */
typedef enum {
  BCUR_F64 = 0,
  BCUR_F32 = 1,
  BCUR_TF32 = 2,
  BCUR_BF16 = 3,
  BCUR_BF16X3 = 4,
  BCUR_FP8 = 5,
  BCUR_BF16X3A = 6,
  BCUR_FP8B = 7
} bcur_prec_t;

typedef struct {
  int64_t m, n;           /* A is m x n                                        */
  int64_t lda;            /* leading dimension of A (elements), lda >= n       */
  int32_t a_dtype;        /* BCUR_F64 or BCUR_F32: storage type of A           */
  int32_t k;              /* target rank, 1 <= k                               */
  int32_t p;              /* oversampling; l = k + p <= min(m, n, 128)         */
  int32_t q;              /* subspace iterations, 0 <= q <= 16                 */
  int32_t G_col;          /* number of column blocks                           */
  const int64_t* col_off; /* host, G_col + 1 increasing offsets, 0 ... n       */
  int32_t G_row;          /* number of row blocks                              */
  const int64_t* row_off; /* host, G_row + 1 increasing offsets, 0 ... m       */
  int32_t g_col, g_row;   /* blocks drawn per side (<= G without replacement) */
  int32_t replacement;    /* 0: without replacement (Sec. 4.1), 1: with (Alg. 1) */
  int32_t sketch_prec;    /* bcur_prec_t of the range-finder GEMMs             */
  int32_t fit_prec;       /* bcur_prec_t of the QR / U / residual GEMMs        */
} bcur_desc_t;

typedef struct bcur_plan_s* bcur_plan_t;

/* ---------------------------------------------------------------------------
 * Plan: validate a descriptor and size the workspace.  Allocates no device
 * memory.  `stream` is a cudaStream_t (may be NULL).  On success *out holds a
 * new plan and *workspace_bytes the device workspace it needs.
 * Errors: BCUR_EINVAL (any descriptor field out of range, offsets not
 * increasing, lda < n, l > min(m, n, 128), g > G without replacement, F64
 * storage with a non-F64 precision), BCUR_ENOTSUP (TF32 stages, or a BF16
 * fit: one BF16 term cannot keep Cholesky-QR of C stable, use BF16X3).
 */
bcur_status_t bcur_plan(const bcur_desc_t* desc, void* stream, bcur_plan_t* out,
                        size_t* workspace_bytes);

/* Attach caller-owned device memory (>= workspace_bytes, 256-byte aligned) as
 * the plan's workspace.  The plan keeps the pointer until destroyed or given
 * another one.  Errors: BCUR_EINVAL (NULL plan/pointer, misaligned),
 * BCUR_ENOMEM (too small). */
bcur_status_t bcur_set_workspace(bcur_plan_t plan, void* workspace, size_t bytes);

/* Stages 1-2: block leverage scores (Def. 2) for column and row blocks.
 *   A          device, row-major m x n (lda), storage type desc.a_dtype.
 *   omega      device, the test matrix Omega (n x l) as a panel: row-major
 *              l x n (ld n), same storage type as A.  Random input chosen by
 *              the caller (a Rademacher matrix in the tests).
 *   col_scores device, G_col doubles;  row_scores device, G_row doubles.
 * The top-k factors stay in the workspace for inspection (bcur_factors).
 * Errors: BCUR_ESTATE (no workspace), BCUR_EINVAL (NULL pointer). */
bcur_status_t bcur_scores(bcur_plan_t plan, const void* A, const void* omega,
                          double* col_scores, double* row_scores);

/* Copy the top-k factors of the last bcur_scores call, as panels: V_k^T
 * (k x n, ld n) and U_k^T (k x m, ld m) in the storage type of A, and the k
 * singular values (double).  Any output may be NULL.  Device pointers. */
bcur_status_t bcur_factors(bcur_plan_t plan, void* Vt, void* Ut, double* sigma);

/* Stage 3: inverse-CDF block sampling (Alg. 1 step 2).  For draw t with
 * uniform u[t] in [0,1) the chosen block is the first remaining j whose FP64
 * running prefix sum of scores (sequential, increasing j, each addition and
 * the product u[t] * total rounded once, no fused multiply-add) exceeds
 * u[t] * total, total = the FP64 sum of the remaining scores; if rounding
 * leaves none, the last remaining block with a positive score; if every
 * remaining score is zero, the first remaining block.  Without replacement
 * a drawn block leaves the pool.
 *   scores  device, G_col (resp. G_row) doubles (e.g. from bcur_scores).
 *   u_col   device, g_col doubles;  u_row device, g_row doubles.
 *   col_idx/row_idx  device int32, g_col / g_row block indices in draw order.
 *   col_prob/row_prob device doubles p_j = l_j / sum(l) per draw (may be NULL).
 */
bcur_status_t bcur_sample(bcur_plan_t plan, const double* col_scores, const double* row_scores,
                          const double* u_col, const double* u_row, int32_t* col_idx,
                          int32_t* row_idx, double* col_prob, double* row_prob);

/* Stages 4-5: gather C and R for the given blocks and fit U = C^+ A R^+.
 *   col_idx/row_idx device int32 block indices (g_col / g_row, in order).
 *   U  device, row-major c x r (ld r), storage type of A; rows follow the
 *      columns of C, columns follow the rows of R.  c = sum of the chosen
 *      column-block sizes, r likewise.  May be NULL.
 *   C  device, optional (NULL): the panel C^T, row-major c x m (ld m).
 *   R  device, optional (NULL): row-major r x n (ld n).
 * Directions of C or R^T that are numerically dependent (a pivot of the
 * Cholesky factor of their Gram matrix below the drop tolerance) are dropped:
 * U is then a least-squares minimiser restricted to the kept directions and
 * bcur_rank() reports the kept counts.  With fit_prec BCUR_BF16X3A and the
 * same A pointer as the last bcur_scores call with a BF16 sketch (contents
 * unchanged in between), the fit reuses the BF16 copy of A that the scores
 * left in the workspace.  Errors: BCUR_ESTATE, BCUR_EINVAL. */
bcur_status_t bcur_fit(bcur_plan_t plan, const void* A, const int32_t* col_idx,
                       const int32_t* row_idx, void* U, void* C, void* R);

/* The BF16 terms the last bcur_fit took for its core products (W = A Q_R,
 * M = Q_C^T W and the triangular products that give U; with BCUR_BF16X3A
 * also the second Cholesky-QR pass): 1 or 3 with
 * fit_prec BCUR_BF16X3A (decided on the device), 3 with BCUR_BF16X3, 0 on
 * CUDA cores.  rel_err_estimate (host, optional) receives the relative error
 * of the one-term residual the adaptive choice was made from (-1 for the
 * other precisions).  Synchronises the plan's stream.
 * Errors: BCUR_EINVAL (NULL plan or terms), BCUR_ESTATE (no fit yet). */
bcur_status_t bcur_fit_terms(bcur_plan_t plan, int32_t* terms, double* rel_err_estimate);

/* Stage 6: residual of the last fit.  out (device, 3 doubles) receives
 * ||A - CUR||_F, ||A - CUR||_F / ||A||_F and ||A||_F.  CUR is never stored:
 * the Frobenius sum is reduced inside the GEMM epilogue in a fixed order, so
 * repeated calls give bit-identical results.  With fit_prec BCUR_BF16X3A the
 * fit has already taken this residual; called with the same A pointer (whose
 * contents must not have changed since bcur_fit), bcur_error copies it. */
bcur_status_t bcur_error(bcur_plan_t plan, const void* A, double* out);

/* Rank-kt truncation of the last fit's U (Sec. 4.1: U_k, the best rank-k
 * approximation of U, gives an exactly rank-k CUR).  The top-kt singular
 * triplets of U (c x r) come from the same randomized range finder as the
 * scores (q steps of subspace iteration, l = k + p columns, test matrix omega
 * given as a panel l x r_max, ld r_max, storage type of A); then
 *   Uk  (device, optional)  U_k, row-major c_max x r_max (ld r_max);
 *   out (device, 3 doubles) ||A - C U_k R||_F, its ratio to ||A||_F, ||A||_F.
 * CUDA-core arithmetic in the storage precision.  1 <= kt <= desc.k; needs
 * l <= min(c, r).  Errors: BCUR_ESTATE (no fit yet), BCUR_EINVAL, BCUR_ENOTSUP
 * (c or r larger than the padded m or n). */
bcur_status_t bcur_truncate(bcur_plan_t plan, const void* A, int32_t kt, const void* omega,
                            void* Uk, double* out);

/* The whole decomposition (stages 1-6) from host buffers: the call a user
 * with data in host memory makes.  A (row-major m x n, lda), omega (the
 * l x n panel, ld n; storage type of A), u_col (g_col) and u_row (g_row)
 * are host pointers; they are copied on the plan's stream into `staging`
 * (caller-owned device memory of at least bcur_host_staging_bytes(plan)
 * bytes, 256-byte aligned), the method runs there as bcur_scores,
 * bcur_sample, bcur_fit and bcur_error do, and the results are copied back
 * into host memory: col_scores (G_col doubles), row_scores (G_row),
 * col_idx (g_col int32), row_idx (g_row int32), U (c_max x r_max in the
 * storage type of A, c_max / r_max the largest possible c and r for the
 * descriptor's g; rows past the drawn c and columns past r are zero) and
 * err (3 doubles, as bcur_error).  Every output but err may be NULL.
 * Asynchronous like every plan call: the host outputs hold the results once
 * the plan's stream has been synchronised (bcur_sync_status), and the host
 * inputs must stay unmodified until then.  Page-locked host memory lets the
 * copies run at full speed (pageable memory is staged by the runtime).
 * Errors: BCUR_ESTATE (no workspace), BCUR_EINVAL (NULL input, misaligned
 * staging), BCUR_ENOMEM (staging too small), and those of the stage calls. */
size_t bcur_host_staging_bytes(bcur_plan_t plan);
bcur_status_t bcur_decompose_host(bcur_plan_t plan, const void* A, const void* omega,
                                  const double* u_col, const double* u_row, void* staging,
                                  size_t staging_bytes, double* col_scores, double* row_scores,
                                  int32_t* col_idx, int32_t* row_idx, void* U, double* err);

/* The rank-k comparison of Sec. 4.1: out (device, 2 doubles) receives
 * ||A - A_k||_F, evaluated as ||A - U_k Sigma_k V_k^T||_F with the top-k
 * factors of the last bcur_scores (the best rank-k error when the range
 * finder captured the top-k subspace, slightly above it otherwise), and the
 * ratio ||A - CUR||_F / ||A - A_k||_F with ||A - CUR||_F from the last
 * bcur_error.  The fused residual on CUDA cores in the storage precision
 * (one more pass over A).  Errors: BCUR_ESTATE (no scores or no error yet),
 * BCUR_EINVAL. */
bcur_status_t bcur_rank_k_error(bcur_plan_t plan, const void* A, double* out);

/* Boosting (Sec. 3.3): the algorithm is repeated t times with independent
 * draws and the decomposition with the smallest ||A - CUR||_F is kept.  With
 * the t runs' outputs laid out contiguously in device memory -- err: t
 * triples at err_stride doubles (>= 3), U: t blocks of U_bytes bytes,
 * col_idx: t x g_col, row_idx: t x g_row -- this picks the run on the
 * device, without a host synchronisation: *best (device int32) = the first
 * run in order with the smallest err[i * err_stride] (NaN loses), and its U,
 * indices and error triple are copied to U_best, col_idx_best, row_idx_best,
 * err_best (device; each may be NULL, as may U).  1 <= t <= 4096.
 * Errors: BCUR_EINVAL. */
bcur_status_t bcur_boost_select(int32_t t, const double* err, int64_t err_stride, const void* U,
                                int64_t U_bytes, const int32_t* col_idx, int32_t g_col,
                                const int32_t* row_idx, int32_t g_row, void* U_best,
                                int32_t* col_idx_best, int32_t* row_idx_best, double* err_best,
                                int32_t* best, void* stream);

/* Sizes of the last fit: c, r, and the number of kept directions of C and
 * R^T.  Host pointers; synchronises the plan's stream. */
bcur_status_t bcur_rank(bcur_plan_t plan, int64_t* c, int64_t* r, int64_t* rank_c,
                        int64_t* rank_r);

/* Synchronise the plan's stream and return (then clear) the first error the
 * device recorded since the last call. */
bcur_status_t bcur_sync_status(bcur_plan_t plan);

void bcur_destroy(bcur_plan_t plan);
const char* bcur_status_string(bcur_status_t status);

/* ---------------------------------------------------------------------------
 * Stage kernels callable without a plan (same arithmetic as the plan calls).
 */

/* Def. 2 for a factor given as a panel F^T (k x h, row-major, ld ldf):
 * scores[g] = sum_{j in [off[g], off[g+1])} sum_{t<k} F[j, t]^2, accumulated
 * in FP64 in a fixed order.  dtype: BCUR_F64 or BCUR_F32.  off: device int64
 * (G + 1, increasing, off[G] <= h); scores: device double (G). */
bcur_status_t bcur_block_scores(const void* Ft, int32_t dtype, int32_t k, int64_t h,
                                int64_t ldf, const int64_t* off, int32_t G, double* scores,
                                void* stream);

/* Block stable rank terms (Sec. 3.2, definition of alpha): for each block g
 * of the factor F whose panel F^T (k x h, ld ldf) is given,
 *   ratio[g] = ||F^T E_g||_F^2 / ||F^T E_g||_2^2   (NaN for an all-zero block),
 * so alpha = min_g ratio[g] and 1 <= ratio[g] <= block size.  The k x k Gram of
 * each block is formed in FP64 and its largest eigenvalue found by one-sided
 * Jacobi.  dtype BCUR_F64 or BCUR_F32, k <= 128; off device int64 (G + 1);
 * ratio device double (G); workspace: device scratch of at least
 * bcur_block_stable_rank_workspace(k, G) bytes (BCUR_ENOMEM otherwise).
 * The incoherence mu = (m/k) max_i ||U_k^T e_i||^2 of the same definition
 * section is bcur_block_scores with blocks of size 1. */
size_t bcur_block_stable_rank_workspace(int32_t k, int32_t G);
bcur_status_t bcur_block_stable_rank(const void* Ft, int32_t dtype, int32_t k, int64_t h,
                                     int64_t ldf, const int64_t* off, int32_t G, double* ratio,
                                     void* workspace, size_t workspace_bytes, void* stream);

/* The incoherence of the same definition section, mu = (m / k) max_i
 * ||U_k^T e_i||^2, from the panel U_k^T (k x m, row-major, ld >= m; dtype
 * F64 or F32; e.g. bcur_factors' Ut): squared row norms in FP64, the
 * maximum taken order-independently.  out: one device double; scratch: 8
 * bytes of device memory (overwritten).  Errors: BCUR_EINVAL. */
bcur_status_t bcur_incoherence(const void* Ut, int32_t dtype, int32_t k, int64_t m, int64_t ld,
                               double* out, void* scratch, void* stream);

/* The paper's Algorithm 1 as printed (Sec. 3.1), one call:
 *   1. r rows of A drawn uniformly with replacement (p_i = 1/m, the inverse-CDF
 *      rule of bcur_sample on equal scores, uniforms u_rows) and
 *      R = S_R^T A = sqrt(m/r) A[rows, :];
 *   2. column-block scores l_i(R) = ||V_R^T E_i||_F^2 with V_R an orthonormal
 *      basis of the numerical row space of R (Cholesky-QR2; pivots below the
 *      drop tolerance leave it), g blocks drawn with replacement from
 *      l / sum(l) (uniforms u_cols);
 *   3. C = A S and W = R S with the scaling I_s / sqrt(g p_j) of Sec. 3.1 and
 *      U = W^+ = Q_W^T L^+ from W = L Q_W (Cholesky-QR2 of W's rows) and the
 *      SVD of the small factor L (singular values at or below
 *      max(r, c) * eps * sigma_1 dropped): the Moore-Penrose inverse, also
 *      when W is rank deficient (a row drawn twice, a low-rank A);
 *   4. err[0..2] = ||A - C U R||_F, its ratio to ||A||_F, and ||A||_F.
 * A device, row-major m x n (lda), dtype BCUR_F64 or BCUR_F32 (arithmetic in
 * that precision on CUDA cores).  col_off host int64 (G + 1).  u_rows (r),
 * u_cols (g), row_idx (r), col_idx (g), col_scores (G), col_prob (g), err (3)
 * device; U device c x r (ld r, c = g * the largest block size) or NULL.
 * Limits: r <= 128, m <= 32768, G <= 32768.  workspace: device scratch of at
 * least bcur_alg1_workspace(...) bytes, 256-byte aligned.
 * Errors: BCUR_EINVAL (argument out of range), BCUR_ENOMEM (workspace). */
size_t bcur_alg1_workspace(int64_t m, int64_t n, const int64_t* col_off, int32_t G, int32_t r,
                           int32_t g, int32_t dtype);
bcur_status_t bcur_alg1(const void* A, int64_t lda, int64_t m, int64_t n, int32_t dtype,
                        const int64_t* col_off, int32_t G, int32_t r, int32_t g,
                        const double* u_rows, const double* u_cols, int32_t* row_idx,
                        int32_t* col_idx, double* col_scores, double* col_prob, void* U,
                        double* err, void* workspace, size_t workspace_bytes, void* stream);

/* Alg. 1 step 2 on one side; the rule is the one stated at bcur_sample.
 * scores device (G), u device (g), idx device int32 (g), prob device (g) or
 * NULL.  G <= 32768.  Errors: BCUR_EINVAL (g > G without replacement). */
bcur_status_t bcur_sample_blocks(const double* scores, int32_t G, const double* u, int32_t g,
                                 int32_t replacement, int32_t* idx, double* prob, void* stream);

/* ||X - P Q||_F^2 reduced in FP64 without forming P Q, where X is row-major
 * m x n (ldx), P row-major m x r (ldp) and Q row-major r x n (ldq).  dtype
 * F64 or F32: X, P, Q of that type, prec F64 (F64 data) or F32 / TF32 (F32
 * data; TF32 falls back to F32 on CUDA cores where TMA cannot serve it).
 * dtype BF16: X FP32, P and Q BF16 (ldp, ldq multiples of 8), prec BF16, on
 * tensor cores.  out: device, 2 doubles {||X - PQ||_F^2, ||X||_F^2}.
 * workspace: device scratch of at least bcur_residual_workspace(m, n, dtype)
 * bytes.  P and Q may be NULL when r = 0.  This is the fused kernel behind
 * bcur_error. */
size_t bcur_residual_workspace(int64_t m, int64_t n, int32_t dtype);
bcur_status_t bcur_residual(const void* X, int64_t ldx, const void* P, int64_t ldp,
                            const void* Q, int64_t ldq, int64_t m, int64_t n, int64_t r,
                            int32_t dtype, int32_t prec, double* out, void* workspace,
                            size_t workspace_bytes, void* stream);

/* bcur_residual for callers that cannot allocate device memory.  The paper
 * has no counterpart: this is a property of the library, not of the method.
 * Who needs it: code whose device memory is entirely owned by another
 * framework's pool (so a fresh cudaMalloc fails or fragments it), request
 * loops that must never call cudaMalloc/cudaFree (cudaFree synchronises the
 * whole device), and plug-ins that are handed only input and output pointers.
 * Same arguments, data types and result as bcur_residual, minus the
 * workspace: dtype F64 (prec F64), F32 (prec F32, TF32 or BF16; where the
 * tensor cores cannot serve the call it runs on the CUDA cores in FP32, as
 * bcur_residual does) or BF16 (X FP32, P and Q BF16, prec BF16, tensor cores
 * only: BCUR_ENOTSUP for operands TMA cannot describe).  The per-CTA partial
 * sums go to a fixed 1 MiB array inside the library's device image (65536
 * partial pairs; every GPU that loads the library holds it until the process
 * exits).
 *   - Sizes whose kernel would need more than 65536 partial pairs (FP32:
 *     more than 65536 tiles of 128 x 128 in X; FP64: tiles of 64 x 64) are
 *     rejected with BCUR_ENOMEM before anything is enqueued.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current, and again if the device's
 *     context has changed since, e.g. after cudaDeviceReset); make that
 *     first call before any stream capture begins.
 *   - No call allocates or frees device memory.
 *   - All calls share the one array and it keeps the last call's contents;
 *     each call writes every slot it later reads, so nothing needs clearing,
 *     but calls that overlap on the GPU (different streams or threads) race
 *     on it and must be serialised by the caller. */
bcur_status_t bcur_residual_noalloc(const void* X, int64_t ldx, const void* P, int64_t ldp,
                                    const void* Q, int64_t ldq, int64_t m, int64_t n, int64_t r,
                                    int32_t dtype, int32_t prec, double* out, void* stream);

/* Plan-free pieces of the fit, for callers that assemble the method from
 * stage calls (the row-sharded form, where each rank holds whole row blocks
 * and the Gram matrices are summed across ranks between the calls).
 *
 * bcur_cholesky_inverse: G = L L^T for a symmetric positive semi-definite
 * w x w matrix (row-major, ld w, lower part read and overwritten by the
 * blocked factorisation's trailing updates), with the drop rule of the fit:
 * a pivot at or below tol_rel times the largest diagonal entry (tol_rel <= 0:
 * 64 units of round-off of dtype) drops its direction (zero row and column
 * of L and L^{-1}).  L and Linv (w x w, zeros above the diagonal) and *kept
 * (device int32, the number of kept pivots) are written.  dtype F64 or F32
 * (CUDA cores, left-looking 64-wide leaves and blocked updates).  w a
 * multiple of 64 (pad with zero rows and columns: they are dropped), at most
 * 65536.  workspace: device scratch of at least 256 bytes, 256-byte aligned.
 *
 * bcur_svd_small: one-sided Jacobi SVD X = Ut diag(sigma) W^T of a w x w FP64
 * matrix (row-major), w <= 128, computed in dtype (F64 or F32); Ut and W
 * row-major w x w in dtype, sigma descending (FP64); work: device scratch of
 * (w + 1)^2 elements of dtype; status (device int32, may be NULL) records
 * BCUR_ETIMEOUT if the sweeps do not converge.
 *
 * bcur_gather_blocks: the chosen blocks of A (row-major m x n, lda, F64 or
 * F32): axis 1 gathers columns into C^T (cap x m, ld ldo >= m), axis 0 rows
 * into R (cap x n, ld ldo >= n); blocks idx (device int32, g entries, in
 * order) of the partition off (device int64, G + 1 offsets); rows of the
 * output past the gathered count are zero; map: device scratch of cap + 1
 * int64 (the gathered count is left in map[cap]).
 * Errors: BCUR_EINVAL, BCUR_ENOMEM. */
bcur_status_t bcur_cholesky_inverse(void* G, int64_t w, int32_t dtype, void* L, void* Linv,
                                    int32_t* kept, double tol_rel, void* workspace,
                                    size_t workspace_bytes, void* stream);
bcur_status_t bcur_svd_small(const double* X, int32_t w, int32_t dtype, void* Ut, void* W,
                             double* sigma, void* work, size_t work_bytes, int32_t* status,
                             void* stream);
bcur_status_t bcur_gather_blocks(const void* A, int64_t lda, int64_t m, int64_t n, int32_t dtype,
                                 int32_t axis, const int64_t* off, int32_t G, const int32_t* idx,
                                 int32_t g, int64_t cap, void* out, int64_t ldo, void* map,
                                 void* stream);

/* Dense GEMM on the library's kernels, exposed for testing the tensor-core
 * path against the CUDA-core path:  D (M x N, row-major, ldd) = A_op B_op,
 * A_op(i, kk) = transA ? A[kk * lda + i] : A[i * lda + kk],
 * B_op(kk, j) = transB ? B[j * ldb + kk] : B[kk * ldb + j].
 * dtype F64/F32: storage of A, B and D, with prec F64 (F64 data), F32 or
 * TF32 (F32 data).  dtype BF16: A and B stored as BF16, D as FP32, prec BF16.
 * dtype FP8: A and B stored as e4m3 bytes, both K-major (transA = 0,
 * transB = 1; otherwise BCUR_ENOTSUP), D as FP32, prec FP8.
 * The tensor-core precisions return BCUR_ENOTSUP for operands TMA cannot
 * describe (base not 16-byte aligned, leading dimension not a multiple of
 * 16 bytes) instead of falling back. */
bcur_status_t bcur_gemm(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                        int32_t transA, const void* B, int64_t ldb, int32_t transB, void* D,
                        int64_t ldd, int32_t dtype, int32_t prec, void* stream);

/* FP8 e4m3 product with one factor per 128 x 128 block of B (the block-scaled
 * path of the FP8B sketch, exposed for testing):
 *   D[i][j] = scale_m[i] * sum_kb bscale[(j / 128) * bs_n + kb * bs_k]
 *                               * sum_{k in K block kb} A[i][k] B[j][k],
 * K blocks of 128.  A (M x K, ld lda bytes) and B (N x K, ld ldb bytes) are
 * e4m3 bytes, both K-major; scale_m (M floats) may be NULL (1); bscale holds
 * the ceil(N/128) x ceil(K/128) block factors with the given strides
 * (elements); D (M x N, FP32, row-major, ldd).  Every 128-deep K block is
 * accumulated in FP32 in its own tensor-memory buffer and added, scaled, in
 * FP32.  Needs M < 128 and N >= 2 M (the product runs transposed, B's blocks
 * along the 128-row tiles), lda and ldb multiples of 16, 16-byte aligned
 * bases.  Errors: BCUR_EINVAL (NULL operand, negative size), BCUR_ENOTSUP
 * (shape or layout outside the above, or no sm_103 tensor cores). */
bcur_status_t bcur_gemm_fp8_blocks(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                                   const void* B, int64_t ldb, const float* scale_m,
                                   const float* bscale, int64_t bs_n, int64_t bs_k, float* D,
                                   int64_t ldd, void* stream);

/* D (M x N, FP32, row-major, ldd) = A B with both operands as BF16 hi/lo
 * pairs (x = hi + lo): A_hi B_hi + A_hi B_lo + A_lo B_hi on the tcgen05
 * tensor cores with FP32 accumulation -- the product the split-BF16 fit uses.
 * Layout conventions as bcur_gemm; A_lo / B_lo share the leading dimension
 * of their hi parts.  All pointers 16-byte aligned, lda, ldb multiples of 8.
 * Errors: BCUR_EINVAL (NULL pointer, negative size), BCUR_ENOTSUP (alignment,
 * or not an sm_103 device). */
bcur_status_t bcur_gemm_split(int64_t M, int64_t N, int64_t K, const void* A_hi, const void* A_lo,
                              int64_t lda, int32_t transA, const void* B_hi, const void* B_lo,
                              int64_t ldb, int32_t transB, float* D, int64_t ldd, void* stream);

/* ---------------------------------------------------------------------------
 * Batched decompositions: many matrices of different m, n, block size and k
 * in one pass of the method, each stage one launch over the whole batch
 * (grouped tcgen05 GEMMs walking every matrix's tiles in one persistent
 * launch, and grouped small kernels).  Same method and precision as a plan
 * with sketch_prec = BCUR_BF16 and fit_prec = BCUR_BF16X3 on FP32 storage:
 * scores from the randomized range finder (Sec. 3.1 allows sketching), block
 * sampling without replacement (Sec. 4.1), U = C^+ A R^+, ||A - CUR||_F.
 * A decomposition's results do not depend on the other members of the
 * batch: every per-matrix sum is formed in a fixed order by the same units of
 * work, whatever else runs beside it.
 */
typedef struct {
  int64_t m, n, lda;   /* A: FP32, row-major m x n, lda >= n, lda % 4 == 0    */
  int32_t k, p;        /* rank and oversampling, l = k + p <= 128; a batch
                          whose items all have l <= 64 uses 64-row panels,
                          otherwise 128-row panels for every item            */
  int32_t block;       /* s: column blocks [j s, min((j+1) s, n)), row blocks
                          likewise over m; G_col = ceil(n/s), G_row = ceil(m/s) */
  int32_t g_col, g_row;/* blocks drawn without replacement; g * s <= 512     */
} bcur_batch_item_t;

/* Per-decomposition device pointers of one run (all device memory):
 *   A          FP32 m x n (lda);  omega: the test matrix as a panel l x n
 *              (ld n, FP32);  u_col (g_col), u_row (g_row): uniforms in [0,1);
 *   col_scores (G_col), row_scores (G_row) doubles;  col_idx (g_col),
 *   row_idx (g_row) int32, in draw order;  U: FP32 (g_col s) x (g_row s),
 *   ld g_row s, rows / columns in gather order, zero past the actual c, r
 *   (may be NULL);  err: 3 doubles {||A - CUR||_F, its ratio to ||A||_F,
 *   ||A||_F}. */
typedef struct {
  const float* A;
  const float* omega;
  const double* u_col;
  const double* u_row;
  double* col_scores;
  double* row_scores;
  int32_t* col_idx;
  int32_t* row_idx;
  float* U;
  double* err;
} bcur_batch_io_t;

typedef struct bcur_batch_s* bcur_batch_t;

/* Tile widths of the grouped GEMMs are picked by the library's autotuner:
 * bcur_batch_set_workspace times, for every GEMM shape class (stage, output
 * width, rows, K, operand layout) not measured before in this process, a
 * grouped launch of copies of one GEMM of that class at each candidate width
 * (64, 128, 256 output columns per tile; 64 or 128 for the skinny sketch
 * products) and keeps the fastest (the widest within 3% of it).  The choice
 * depends only on the GEMM's own shape, so a decomposition's results are the
 * same alone or in any batch.  Environment: BCUR_AUTOTUNE=0 skips the
 * measurements (fixed widths by output width for unseen shapes);
 * BCUR_AUTOTUNE_CACHE=<file> loads earlier choices from that JSON file and
 * writes new ones back.  bcur_autotune_measured() counts the shape classes
 * measured so far in this process. */
int32_t bcur_autotune_measured(void);

/* Validate `count` items and size the workspace; q subspace iterations
 * (0..16) for every item.  Allocates no device memory.  Errors: BCUR_EINVAL
 * (an item out of range: l > 128, g > G, g * s > 512, lda < n or not a
 * multiple of 4, count < 1), BCUR_ENOTSUP (no sm_103 tensor cores). */
bcur_status_t bcur_batch_plan(const bcur_batch_item_t* items, int32_t count, int32_t q,
                              void* stream, bcur_batch_t* out, size_t* workspace_bytes);

/* Attach caller-owned device memory (>= workspace_bytes, 256-byte aligned)
 * and build the launch tables in it (tensor maps of every grouped GEMM,
 * work lists), after the autotuner has chosen the tile widths (above; its
 * measuring launches run on the plan's own setup stream and use only this
 * workspace).  Synchronous.  Errors: BCUR_EINVAL, BCUR_ENOMEM, BCUR_ECUDA. */
bcur_status_t bcur_batch_set_workspace(bcur_batch_t plan, void* workspace, size_t bytes);

/* Fit precision of every item of the batch: BCUR_BF16X3 (the default; every
 * product of the fit as a split BF16 pair) or BCUR_BF16X3A (the adaptive
 * form of bcur_plan's fit_prec: each item's second Cholesky-QR pass Grams,
 * core products W, M and M2 and its residual first with one BF16 term, redone
 * with three (with that pass's Cholesky) for the items whose one-term
 * residual is too coarse for the error it reports, e < 0.031; the
 * two products that give U take the item's term count).  An item's choice
 * depends only on its own data, so its results stay the same alone or in any
 * batch.  Call before bcur_batch_set_workspace.  Errors: BCUR_EINVAL (NULL
 * plan or another precision), BCUR_ESTATE (the workspace is already bound). */
bcur_status_t bcur_batch_set_fit(bcur_batch_t plan, int32_t fit_prec);

/* terms (host, count entries): the BF16 terms each item's core products took
 * in the last run, 1 or 3 (3 for every item of a BCUR_BF16X3 plan).
 * Synchronises the plan's stream.  Errors: BCUR_EINVAL, BCUR_ESTATE (no
 * workspace). */
bcur_status_t bcur_batch_fit_terms(bcur_batch_t plan, int32_t* terms);

/* Run the whole method for every item; io: host array of `count` entries
 * (read before the call returns).  Asynchronous on the plan's stream.  With
 * use_graph != 0 the launch sequence is captured into a CUDA graph on the
 * first call and replayed afterwards (the io table is copied by the graph
 * from the plan's pinned staging buffer).  Errors: BCUR_ESTATE (no
 * workspace), BCUR_EINVAL (NULL pointer in io). */
bcur_status_t bcur_batch_run(bcur_batch_t plan, const bcur_batch_io_t* io, int32_t use_graph);

/* Move the plan to another stream (cudaStream_t; NULL = legacy default) for
 * the following runs, e.g. a plan built on one host thread and run on the
 * stream of whichever lane is free.  Errors: BCUR_EINVAL. */
bcur_status_t bcur_batch_set_stream(bcur_batch_t plan, void* stream);

/* Padded sizes of item i: cmax = g_col s, rmax = g_row s (the U layout), and
 * the number of kernel launches one run makes. */
bcur_status_t bcur_batch_dims(bcur_batch_t plan, int32_t i, int64_t* cmax, int64_t* rmax,
                              int64_t* launches_per_run);

/* Synchronise the plan's stream and return (then clear) the first error the
 * device recorded. */
bcur_status_t bcur_batch_sync_status(bcur_batch_t plan);

/* Profiling of eager runs: with enable != 0 the following runs that are not
 * replayed from a graph record a CUDA event after each launch (or group of
 * launches) of the sequence.  After such a run has completed,
 * bcur_batch_profile_count gives the number of timed steps and
 * bcur_batch_profile_entry the label of step i (a static string naming the
 * kernel kind: "split", "sketch_gemm", "skinny_gram", "skinny_chol",
 * "skinny_apply", "jacobi", "scores", "sample", "gather", "qr_gram",
 * "wide_chol", "qr_apply", "w_gemm", "m_gemm", "u_gemm", "copy_u", "p_gemm",
 * "residual", "finish") and its duration in milliseconds.  Errors:
 * BCUR_EINVAL (no such step), BCUR_ECUDA (run not finished). */
bcur_status_t bcur_batch_profile(bcur_batch_t plan, int32_t enable);
int32_t bcur_batch_profile_count(bcur_batch_t plan);
bcur_status_t bcur_batch_profile_entry(bcur_batch_t plan, int32_t i, const char** label,
                                       double* ms);

void bcur_batch_destroy(bcur_batch_t plan);

/* Number of CUDA kernels this library has launched in this process (all
 * threads, all devices).  Used to report launches per timed step. */
uint64_t bcur_launch_count(void);

/* Bound, in nanoseconds, of every wait inside the tensor-core kernels' main
 * loops (a pipeline stage, an accumulator) on the current device, for the
 * launches that follow; default 2 s, allowed 1 ns ... 60 s.  A wait that
 * runs out records BCUR_ETIMEOUT in the status word of the call (returned
 * by bcur_sync_status / bcur_batch_sync_status); the kernel then waits for
 * the copies and products it has already issued (always with the full 2 s
 * bound), releases its tensor memory and returns, so the context stays
 * usable.  Meant for watchdogs and for tests of that path.  Synchronous.
 * Errors: BCUR_EINVAL (out of range), BCUR_ECUDA. */
bcur_status_t bcur_set_wait_budget_ns(uint64_t ns);

/* Library version, "major.minor.patch". */
const char* bcur_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BCUR_H_ */
