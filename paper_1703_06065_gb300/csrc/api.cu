// C ABI of the Block CUR library: plan, workspace layout and the stage
// orchestration.  Every arithmetic step runs in this library's CUDA kernels;
// the host only validates, lays out memory and enqueues launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "kernels.h"

namespace bcur {

static thread_local char g_last_err[256] = {0};
void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_err, sizeof(g_last_err), "%s: %s (%s:%d)", what, cudaGetErrorString(e), file,
           line);
}

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

template <typename T> struct EpsOf;
template <> struct EpsOf<float> { static constexpr double v = 1.1920928955078125e-07; };
template <> struct EpsOf<double> { static constexpr double v = 2.220446049250313e-16; };

// Bump allocator over the caller's workspace (256-byte aligned slices).
struct Layout {
  size_t cur = 0;
  size_t take(size_t bytes) {
    const size_t at = cur;
    cur += (bytes + 255) / 256 * 256;
    return at;
  }
};

}  // namespace bcur

using namespace bcur;

// Handles are opaque to callers: a tag as the first member lets every entry
// point refuse a handle of the other kind (a batch plan) or a stale one.
constexpr uint32_t kPlanTag = 0x50435542u;  // "BUCP"

struct bcur_plan_s {
  uint32_t tag = kPlanTag;
  bcur_desc_t d;
  std::vector<int64_t> col_off, row_off;
  cudaStream_t stream = nullptr;
  cudaStream_t stream2 = nullptr;      // second lane: the R-side QR runs beside the C side
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_stagger = nullptr;
  int64_t m = 0, n = 0, lda = 0;
  int k = 0, l = 0, q = 0;
  int64_t ldm = 0, ldn = 0;      // padded panel leading dims
  int64_t c_max = 0, r_max = 0;  // largest possible c, r for the chosen g
  int64_t c_pad = 0, r_pad = 0;  // padded to the blocked-Cholesky panel size
  int nb = 64;
  int ksplit_m = 1, ksplit_n = 1;
  size_t esz = 8;
  int sms = 148;
  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0, need = 0;
  struct {
    size_t Pm0, Pm1, Pn0, Pn1, Pn2, gram_part, G64, L64a, L64b, Lprod64, Linv64, LinvT, Ut, W,
        sigma, jwork, Vp, Up, col_off, row_off, status, kept, colmap, rowmap, counts, Cp0, Cp1,
        Rp0, Rp1, GC, L1C, L1Ci, L2C, L2Ci, GR, L1R, L1Ri, L2R, L2Ri, maxdiag, Wb, Mb, U1, U2,
        partials, result, tc_scratch;
    // BF16 tensor-core path
    size_t A16h, A16l, Om16h, Om16l, Qm16h, Qm16l, Zn16h, Zn16l, XC16[4], XR16[4], Lh, Ll, Lih,
        Lil, T1h, T1l, Pnh, Pnl, Wh, Wl, Mh, Ml, U1h, U1l, U2h, U2l, Ph, Pl, refine;
    // adaptive split fit: its refinement flag; the one-term, three-term and
    // chosen residuals it took
    size_t fit_flag, fit_err;
    // FP8 sketch
    size_t A8, A8T, sA, X8m, X8n, sx;
    // per-lane temporaries of the second lane
    size_t Lh2, Ll2, Lih2, Lil2, T1h2, T1l2, Pnh2, Pnl2, maxdiag2, tc_scratch2;
  } o;
  bool bf16_path = false;
  size_t tc_scratch_bytes = 0;
  int64_t n_partials = 0;
  bool have_scores = false, have_fit = false, have_error = false;
  // adaptive split fit: the A its residual was taken of (bcur_error reuses it),
  // and the A whose BF16 hi copy the last scores call left in the workspace
  const void* fit_A = nullptr;
  const void* scores_A16 = nullptr;
  template <typename P> P* at(size_t off) const { return reinterpret_cast<P*>(ws + off); }
};

namespace {

bool plan_ok(const bcur_plan_s* P) { return P && P->tag == kPlanTag; }

bool is_tc_prec(int p) { return p == BCUR_TF32 || p == BCUR_BF16; }
bool is_bf16_prec(int p) { return p == BCUR_BF16 || p == BCUR_BF16X3 || p == BCUR_BF16X3A; }

// The Cholesky updates must keep the working precision's accuracy: a Gram
// matrix with condition number kappa^2 loses kappa^2 * u in them.
template <typename T> constexpr int exact_prec() {
  return std::is_same<T, double>::value ? BCUR_F64 : BCUR_F32;
}

int64_t max_sum_of_g(const std::vector<int64_t>& off, int g, bool replacement) {
  std::vector<int64_t> sz(off.size() - 1);
  for (size_t i = 0; i + 1 < off.size(); ++i) sz[i] = off[i + 1] - off[i];
  std::sort(sz.begin(), sz.end(), std::greater<int64_t>());
  int64_t s = 0;
  if (replacement) return (int64_t)g * (sz.empty() ? 0 : sz[0]);
  for (int i = 0; i < g && i < (int)sz.size(); ++i) s += sz[i];
  return s;
}

bool valid_offsets(const int64_t* off, int G, int64_t total) {
  if (!off || G < 1) return false;
  if (off[0] != 0 || off[G] != total) return false;
  for (int i = 0; i < G; ++i)
    if (off[i + 1] <= off[i]) return false;
  return true;
}

// GEMM dispatch: tensor-core path for TF32 / BF16 precisions on FP32 data,
// CUDA-core FMA path otherwise.
template <typename T>
bcur_status_t gemm(const GemmDesc& d, int prec, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (is_tc_prec(prec)) {
      bcur_status_t st = gemm_tc(d, prec, s);
      if (st != BCUR_ENOTSUP) return st;
    }
  }
  return gemm_simt<T>(d, s);
}

template <typename T>
bcur_status_t gemm_resid(const GemmDesc& d, int prec, cudaStream_t s, int64_t* np) {
  if constexpr (std::is_same<T, float>::value) {
    if (is_tc_prec(prec)) {
      bcur_status_t st = gemm_tc_resid(d, prec, s, np);
      if (st != BCUR_ENOTSUP) return st;
    }
  }
  return gemm_simt_resid<T>(d, s, np);
}

// Plan-aware dispatch: attaches the plan's split-K scratch and status word.
template <typename T>
bcur_status_t pg(bcur_plan_t P, GemmDesc d, int prec);
template <typename T>
bcur_status_t pgr(bcur_plan_t P, GemmDesc d, int prec, int64_t* np);

GemmDesc mk(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, int tA, const void* B,
            int64_t ldb, int tB, void* D, int64_t ldd) {
  GemmDesc g;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.lda = lda; g.transA = tA;
  g.B = B; g.ldb = ldb; g.transB = tB;
  g.D = D; g.ldd = ldd;
  return g;
}

template <typename T>
bcur_status_t pg(bcur_plan_t P, GemmDesc d, int prec) {
  d.scratch = P->at<void>(P->o.tc_scratch);
  d.scratch_bytes = P->tc_scratch_bytes;
  d.status = P->at<int>(P->o.status);
  return gemm<T>(d, prec, P->stream);
}
template <typename T>
bcur_status_t pgr(bcur_plan_t P, GemmDesc d, int prec, int64_t* np) {
  d.status = P->at<int>(P->o.status);
  return gemm_resid<T>(d, prec, P->stream, np);
}

// --- Skinny Cholesky-QR2 on a panel X (w x h, ld), w <= 128 ----------------
// X <- Q (rows orthonormal), L64 out = L with X_in = L Q (FP64, w x w).
template <typename T>
bcur_status_t orth_panel(bcur_plan_t P, T* X, T* tmp, int w, int64_t h, int64_t ld, int ksplit,
                         int prec, double* Lout) {
  cudaStream_t s = P->stream;
  const double tol = 64.0 * EpsOf<T>::v;
  T* src = X;
  T* dst = tmp;
  double* Ls[2] = {P->at<double>(P->o.L64a), P->at<double>(P->o.L64b)};
  for (int pass = 0; pass < 2; ++pass) {
    GemmDesc g = mk(w, w, h, src, ld, 0, src, ld, 1, P->at<T>(P->o.gram_part), w);
    g.ksplit = ksplit;
    g.sD = (int64_t)w * w;
    BCUR_TRY(pg<T>(P, g, prec));
    BCUR_TRY(reduce_splits_f64<T>(P->at<T>(P->o.gram_part), ksplit, (int64_t)w * w,
                                  (int64_t)w * w, P->at<double>(P->o.G64), s));
    BCUR_TRY(chol_small<T>(P->at<double>(P->o.G64), w, tol, Ls[pass], P->at<double>(P->o.Linv64),
                           P->at<T>(P->o.LinvT), P->at<int>(P->o.kept), s));
    GemmDesc a = mk(w, h, w, P->at<T>(P->o.LinvT), w, 0, src, ld, 0, dst, ld);
    a.triA = 1;
    BCUR_TRY(pg<T>(P, a, prec));
    std::swap(src, dst);
  }
  // after two passes the result is back in X
  if (Lout) BCUR_TRY(trmm_small_f64(Ls[0], Ls[1], w, Lout, s));
  return BCUR_OK;
}

// --- Wide Cholesky-QR2 on a panel X (w x h, ld), w a multiple of nb -------
// X = L1 L2 Q;  writes Q into `Q`, and L1, L1^{-1}, L2, L2^{-1} (w x w).
// Drop tolerance for the pivots of a Gram matrix X X^T with inner dimension
// h, relative to its largest diagonal entry.  In FP64 the rounding of the
// Gram itself reaches h * u * max diag, so pivots below 2 h u are noise.  In
// FP32 that worst case would also drop real directions of well-conditioned
// inputs (h = 32768 gives 7.8e-3), so FP32 keeps the fixed 64 u.
template <typename T>
double drop_tol(int64_t h) {
  return std::is_same<T, double>::value ? EpsOf<T>::v * std::max<double>(64.0, 2.0 * (double)h)
                                        : 64.0 * EpsOf<T>::v;
}

template <typename T>
bcur_status_t chol_inv_blocked(bcur_plan_t P, T* G, T* L, T* Li, int64_t w, int prec, int* kept,
                               double tol) {
  cudaStream_t s = P->stream;
  const int nb = P->nb;
  T* md = P->at<T>(P->o.maxdiag);
  BCUR_TRY(fill_zero(L, (size_t)w * w * sizeof(T), s));
  BCUR_TRY(fill_zero(Li, (size_t)w * w * sizeof(T), s));
  BCUR_TRY(fill_zero(kept, sizeof(int), s));
  BCUR_TRY(max_diag<T>(G, w, w, md, s));
  for (int64_t j0 = 0; j0 < w; j0 += nb) {
    BCUR_TRY(potrf_diag<T>(G, w, L, w, Li, w, j0, nb, md, tol, kept, s));
    const int64_t j1 = j0 + nb;
    if (j1 >= w) break;
    GemmDesc pn = mk(w - j1, nb, nb, G + j1 * w + j0, w, 0, Li + j0 * w + j0, w, 1,
                     L + j1 * w + j0, w);
    pn.triB = 2;
    BCUR_TRY(pg<T>(P, pn, exact_prec<T>()));
    GemmDesc tr = mk(w - j1, w - j1, nb, L + j1 * w + j0, w, 0, L + j1 * w + j0, w, 1,
                     G + j1 * w + j1, w);
    tr.alpha = -1.0;
    tr.beta = 1.0;
    tr.out_lower = 1;
    BCUR_TRY(pg<T>(P, tr, exact_prec<T>()));
  }
  // Inverse of the whole lower factor by doubling: with X11, X22 the inverses
  // of the diagonal halves, X21 = -X22 L21 X11.  G serves as the temporary.
  for (int64_t h = nb; h < w; h *= 2) {
    const int64_t npairs_full = w / (2 * h);
    if (npairs_full > 0) {
      GemmDesc t1 = mk(h, h, h, L + h * w, w, 0, Li, w, 0, G, h);
      t1.triB = 1;
      t1.batch = (int)npairs_full;
      t1.sA = 2 * h * (w + 1);
      t1.sB = 2 * h * (w + 1);
      t1.sD = h * h;
      BCUR_TRY(pg<T>(P, t1, prec));
      GemmDesc t2 = mk(h, h, h, Li + h * w + h, w, 0, G, h, 0, Li + h * w, w);
      t2.triA = 1;
      t2.alpha = -1.0;
      t2.batch = (int)npairs_full;
      t2.sA = 2 * h * (w + 1);
      t2.sB = h * h;
      t2.sD = 2 * h * (w + 1);
      BCUR_TRY(pg<T>(P, t2, prec));
    }
    const int64_t b1 = npairs_full * 2 * h, b2 = b1 + h;
    if (b2 < w) {  // ragged last pair
      const int64_t h2 = w - b2;
      GemmDesc t1 = mk(h2, h, h, L + b2 * w + b1, w, 0, Li + b1 * w + b1, w, 0, G, h);
      t1.triB = 1;
      BCUR_TRY(pg<T>(P, t1, prec));
      GemmDesc t2 = mk(h2, h, h2, Li + b2 * w + b2, w, 0, G, h, 0, Li + b2 * w + b1, w);
      t2.triA = 1;
      t2.alpha = -1.0;
      BCUR_TRY(pg<T>(P, t2, prec));
    }
  }
  return BCUR_OK;
}

template <typename T>
bcur_status_t wide_cqr2(bcur_plan_t P, T* X, T* tmp, int64_t w, int64_t h, int64_t ld, T* G,
                        T* L1, T* L1i, T* L2, T* L2i, int prec, int* kept) {
  cudaStream_t s = P->stream;
  T* src = X;
  T* dst = tmp;
  T* Ls[2] = {L1, L2};
  T* Lis[2] = {L1i, L2i};
  for (int pass = 0; pass < 2; ++pass) {
    GemmDesc g = mk(w, w, h, src, ld, 0, src, ld, 1, G, w);
    g.out_lower = 1;
    BCUR_TRY(pg<T>(P, g, prec));
    BCUR_TRY(chol_inv_blocked<T>(P, G, Ls[pass], Lis[pass], w, prec, kept + pass, drop_tol<T>(h)));
    GemmDesc a = mk(w, h, w, Lis[pass], w, 0, src, ld, 0, dst, ld);
    a.triA = 1;
    BCUR_TRY(pg<T>(P, a, prec));
    std::swap(src, dst);
  }
  return BCUR_OK;  // Q is back in X
}

// --- Stage 1-2 -------------------------------------------------------------
template <typename T>
bcur_status_t scores_tail(bcur_plan_t P, double* cs, double* rs);

template <typename T>
bcur_status_t run_scores(bcur_plan_t P, const T* A, const T* omega, double* cs, double* rs) {
  cudaStream_t s = P->stream;
  const int l = P->l, k = P->k;
  const int sp = P->d.sketch_prec;
  const int64_t m = P->m, n = P->n, lda = P->lda, ldm = P->ldm, ldn = P->ldn;
  T* Pm0 = P->at<T>(P->o.Pm0);
  T* Pm1 = P->at<T>(P->o.Pm1);
  T* Pn0 = P->at<T>(P->o.Pn0);
  T* Pn1 = P->at<T>(P->o.Pn1);
  // Y^T = Omega^T A^T  (Y = A Omega)
  BCUR_TRY(pg<T>(P, mk(l, m, n, omega, n, 0, A, lda, 1, Pm0, ldm), sp));
  BCUR_TRY(orth_panel<T>(P, Pm0, Pm1, l, m, ldm, P->ksplit_m, sp, nullptr));
  for (int it = 0; it < P->q; ++it) {
    // Z^T = Q^T A  (Z = A^T Q)
    BCUR_TRY(pg<T>(P, mk(l, n, m, Pm0, ldm, 0, A, lda, 0, Pn0, ldn), sp));
    BCUR_TRY(orth_panel<T>(P, Pn0, Pn1, l, n, ldn, P->ksplit_n, sp, nullptr));
    // Y^T = Z^T A^T
    BCUR_TRY(pg<T>(P, mk(l, m, n, Pn0, ldn, 0, A, lda, 1, Pm0, ldm), sp));
    BCUR_TRY(orth_panel<T>(P, Pm0, Pm1, l, m, ldm, P->ksplit_m, sp, nullptr));
  }
  // B = Q^T A (l x n) = L_B Q_B, then SVD of L_B.
  BCUR_TRY(pg<T>(P, mk(l, n, m, Pm0, ldm, 0, A, lda, 0, Pn0, ldn), sp));
  return scores_tail<T>(P, cs, rs);
}

// Shared end of stage 1-2: with B^T (l x n panel) in Pn0 and Q^T in Pm0,
// B = L_B Q_B, the SVD of L_B gives V_k = Q_B W_k and U_k = Q U~_k, then the
// block scores.
template <typename T>
bcur_status_t scores_tail(bcur_plan_t P, double* cs, double* rs) {
  cudaStream_t s = P->stream;
  const int l = P->l, k = P->k;
  const int64_t m = P->m, n = P->n, ldm = P->ldm, ldn = P->ldn;
  T* Pm0 = P->at<T>(P->o.Pm0);
  T* Pn0 = P->at<T>(P->o.Pn0);
  T* Pn1 = P->at<T>(P->o.Pn1);
  double* LB = P->at<double>(P->o.Lprod64);
  BCUR_TRY(orth_panel<T>(P, Pn0, Pn1, l, n, ldn, P->ksplit_n, exact_prec<T>(), LB));
  T* Ut = P->at<T>(P->o.Ut);
  T* W = P->at<T>(P->o.W);
  BCUR_TRY(jacobi_svd_small<T>(LB, l, Ut, W, P->at<double>(P->o.sigma), P->at<T>(P->o.jwork),
                               P->at<int>(P->o.status), s));
  // V_k^T = W_k^T Q_B^T ,  U_k^T = Ut_k^T Q^T
  T* Vp = P->at<T>(P->o.Vp);
  T* Up = P->at<T>(P->o.Up);
  BCUR_TRY(gemm_simt<T>(mk(k, n, l, W, l, 1, Pn0, ldn, 0, Vp, ldn), s));
  BCUR_TRY(gemm_simt<T>(mk(k, m, l, Ut, l, 1, Pm0, ldm, 0, Up, ldm), s));
  BCUR_TRY(block_scores<T>(Vp, k, n, ldn, P->at<int64_t>(P->o.col_off), P->d.G_col, cs,
                           P->at<int>(P->o.status), s));
  BCUR_TRY(block_scores<T>(Up, k, m, ldm, P->at<int64_t>(P->o.row_off), P->d.G_row, rs,
                           P->at<int>(P->o.status), s));
  return BCUR_OK;
}

// --- Stages 4-5 ------------------------------------------------------------
template <typename T>
bcur_status_t run_fit(bcur_plan_t P, const T* A, const int32_t* ci, const int32_t* ri, T* Uout,
                      T* Cout, T* Rout) {
  cudaStream_t s = P->stream;
  const int fp = P->d.fit_prec;
  const int64_t m = P->m, n = P->n, lda = P->lda, ldm = P->ldm, ldn = P->ldn;
  const int64_t cw = P->c_pad, rw = P->r_pad;
  int64_t* counts = P->at<int64_t>(P->o.counts);
  BCUR_TRY(expand_blocks(ci, P->d.g_col, P->at<int64_t>(P->o.col_off), P->d.G_col, cw,
                         P->at<int64_t>(P->o.colmap), counts, s));
  BCUR_TRY(expand_blocks(ri, P->d.g_row, P->at<int64_t>(P->o.row_off), P->d.G_row, rw,
                         P->at<int64_t>(P->o.rowmap), counts + 1, s));
  T* Cp = P->at<T>(P->o.Cp0);
  T* Rp = P->at<T>(P->o.Rp0);
  BCUR_TRY(gather_cols_t<T>(A, lda, m, P->at<int64_t>(P->o.colmap), cw, Cp, ldm, s));
  BCUR_TRY(gather_rows<T>(A, lda, n, P->at<int64_t>(P->o.rowmap), rw, Rp, ldn, s));
  if (Cout) BCUR_TRY(copy2d<T>(Cp, ldm, Cout, m, P->c_max, m, s));
  if (Rout) BCUR_TRY(copy2d<T>(Rp, ldn, Rout, n, P->r_max, n, s));
  // QR of C (through its panel C^T) and of R^T (through R itself).
  BCUR_TRY(wide_cqr2<T>(P, Cp, P->at<T>(P->o.Cp1), cw, m, ldm, P->at<T>(P->o.GC),
                        P->at<T>(P->o.L1C), P->at<T>(P->o.L1Ci), P->at<T>(P->o.L2C),
                        P->at<T>(P->o.L2Ci), fp, P->at<int>(P->o.kept) + 4));
  BCUR_TRY(wide_cqr2<T>(P, Rp, P->at<T>(P->o.Rp1), rw, n, ldn, P->at<T>(P->o.GR),
                        P->at<T>(P->o.L1R), P->at<T>(P->o.L1Ri), P->at<T>(P->o.L2R),
                        P->at<T>(P->o.L2Ri), fp, P->at<int>(P->o.kept) + 6));
  // W = A Q_R (m x r),  M = Q_C^T W (c x r)
  T* Wb = P->at<T>(P->o.Wb);
  T* Mb = P->at<T>(P->o.Mb);
  BCUR_TRY(pg<T>(P, mk(m, rw, n, A, lda, 0, Rp, ldn, 1, Wb, rw), fp));
  BCUR_TRY(pg<T>(P, mk(cw, rw, m, Cp, ldm, 0, Wb, rw, 0, Mb, rw), fp));
  // U = L1C^{-T} L2C^{-T} M L2R^{-1} L1R^{-1}
  T* U1 = P->at<T>(P->o.U1);
  T* U2 = P->at<T>(P->o.U2);
  {
    GemmDesc g1 = mk(cw, rw, rw, Mb, rw, 0, P->at<T>(P->o.L2Ri), rw, 0, U1, rw);
    g1.triB = 1;
    BCUR_TRY(pg<T>(P, g1, fp));
    GemmDesc g2 = mk(cw, rw, rw, U1, rw, 0, P->at<T>(P->o.L1Ri), rw, 0, U2, rw);
    g2.triB = 1;
    BCUR_TRY(pg<T>(P, g2, fp));
    GemmDesc g3 = mk(cw, rw, cw, P->at<T>(P->o.L2Ci), cw, 1, U2, rw, 0, U1, rw);
    g3.triA = 2;
    BCUR_TRY(pg<T>(P, g3, fp));
    GemmDesc g4 = mk(cw, rw, cw, P->at<T>(P->o.L1Ci), cw, 1, U1, rw, 0, U2, rw);
    g4.triA = 2;
    BCUR_TRY(pg<T>(P, g4, fp));
  }
  if (Uout) BCUR_TRY(copy2d<T>(U2, rw, Uout, P->r_max, P->c_max, P->r_max, s));
  return BCUR_OK;
}

// --- Stage 6 ---------------------------------------------------------------
template <typename T>
bcur_status_t run_error(bcur_plan_t P, const T* A, double* out) {
  cudaStream_t s = P->stream;
  const int fp = P->d.fit_prec;
  const int64_t m = P->m, n = P->n, ldm = P->ldm, ldn = P->ldn;
  const int64_t cw = P->c_pad, rw = P->r_pad;
  T* Wb = P->at<T>(P->o.Wb);
  // P = Q_C M  (m x r)
  BCUR_TRY(pg<T>(P, mk(m, rw, cw, P->at<T>(P->o.Cp0), ldm, 1, P->at<T>(P->o.Mb), rw, 0, Wb, rw),
                  fp));
  GemmDesc r = mk(m, n, rw, Wb, rw, 0, P->at<T>(P->o.Rp0), ldn, 0, nullptr, 0);
  r.X = A;
  r.ldx = P->lda;
  r.partials = P->at<double>(P->o.partials);
  int64_t np = 0;
  BCUR_TRY(pgr<T>(P, r, fp, &np));
  BCUR_TRY(finish_residual(P->at<double>(P->o.partials), np, out, 0, s));
  return BCUR_OK;
}


// ===========================================================================
// BF16 tensor-core pipeline (FP32 storage).  Operands of every large GEMM are
// BF16 roundings (BCUR_BF16) or BF16 hi/lo pairs (BCUR_BF16X3) produced by
// split kernels or written directly by the producing GEMM's epilogue; the
// skinny l x l algebra, the Cholesky diagonal blocks and panels stay FP32 /
// FP64 on CUDA cores.
// ===========================================================================
using bf16 = __nv_bfloat16;
struct S16 {
  bf16* h;
  bf16* l;
  S16 off(int64_t e) const { return {h + e, l ? l + e : nullptr}; }
};

int parts_of(int prec) { return (prec == BCUR_BF16X3 || prec == BCUR_BF16X3A) ? 3 : 1; }

S16 s16(bcur_plan_t P, size_t oh, size_t ol, bool with_lo) {
  return {P->at<bf16>(oh), with_lo ? P->at<bf16>(ol) : nullptr};
}

bcur_status_t split(bcur_plan_t P, const float* X, int64_t ldx, int64_t rows, int64_t cols,
                    S16 out, int64_t ldo) {
  return split_bf16(X, ldx, rows, cols, out.h, out.l, ldo, P->stream);
}

GemmDesc mk16(int64_t M, int64_t N, int64_t K, S16 A, int64_t lda, int tA, S16 B, int64_t ldb,
              int tB, int64_t ldd) {
  GemmDesc g = mk(M, N, K, A.h, lda, tA, B.h, ldb, tB, nullptr, ldd);
  g.A_lo = A.l;
  g.B_lo = B.l;
  g.ab_bf16 = 1;
  return g;
}

// An execution lane: a stream plus the temporaries that must not be shared
// between concurrently running factorisations.
struct Lane {
  cudaStream_t s;
  size_t Pnh, Pnl, Lh, Ll, Lih, Lil, T1h, T1l, maxdiag, scratch;
};

Lane lane_of(bcur_plan_t P, int i) {
  const auto& o = P->o;
  if (i == 0)
    return {P->stream, o.Pnh, o.Pnl, o.Lh, o.Ll, o.Lih, o.Lil, o.T1h, o.T1l, o.maxdiag, o.tc_scratch};
  return {P->stream2, o.Pnh2, o.Pnl2, o.Lh2, o.Ll2, o.Lih2, o.Lil2, o.T1h2, o.T1l2, o.maxdiag2,
          o.tc_scratch2};
}

// Tensor-core GEMM on BF16 operands; never falls back (ENOTSUP is an error).
bcur_status_t g16_on(bcur_plan_t P, const Lane& ln, GemmDesc d, int parts) {
  d.parts = parts;
  if (parts != 3) { d.A_lo = nullptr; d.B_lo = nullptr; }
  d.scratch = P->at<void>(ln.scratch);
  d.scratch_bytes = P->tc_scratch_bytes;
  d.status = P->at<int>(P->o.status);
  return gemm_tc(d, BCUR_BF16, ln.s);
}

bcur_status_t g16(bcur_plan_t P, GemmDesc d, int parts) { return g16_on(P, lane_of(P, 0), d, parts); }

// Blocked Cholesky G = L L^T (w x w, FP32, lower part) and L^{-1}.  Two
// levels: outer panels whose trailing update is one large tensor-core GEMM
// (K = the panel width), and inside each outer panel steps of nb = 64
// columns.  With w a multiple of 64 a step is one launch, left-looking inside
// the outer panel (chol_step: exact FP32 products, outer panels of
// kOuterStep columns); otherwise the right-looking order with kOuter-wide
// panels (FP32 diagonal factorisation and panel solve on CUDA cores, the
// update of the rest of the outer panel on tensor cores).  The inverse is
// assembled by doubling (X21 = -X22 L21 X11) on tensor cores.  Tensor-core
// products use `parts` BF16 terms.  run (optional device flag, the 64-column
// step path only): every launch does nothing when *run reads 0.
constexpr int64_t kOuter = 1024;
constexpr int64_t kOuterStep = 512;

bool chol_steps_apply(bcur_plan_t P, int64_t w) { return P->nb == 64 && w % 64 == 0; }

bcur_status_t chol_inv_blocked16(bcur_plan_t P, const Lane& ln, float* G, float* L, float* Li,
                                 int64_t w, int parts, int* kept, double tol,
                                 const int* run = nullptr) {
  cudaStream_t s = ln.s;
  const int nb = P->nb;
  const bool lo = parts == 3;
  float* md = P->at<float>(ln.maxdiag);
  S16 Pn = s16(P, ln.Pnh, ln.Pnl, lo);
  S16 L16 = s16(P, ln.Lh, ln.Ll, lo);
  S16 Li16 = s16(P, ln.Lih, ln.Lil, lo);
  S16 T1 = s16(P, ln.T1h, ln.T1l, lo);
  auto split = [&](bcur_plan_t, const float* X, int64_t ldx, int64_t rows, int64_t cols, S16 out,
                   int64_t ldo) {
    return split_bf16(X, ldx, rows, cols, out.h, out.l, ldo, s, true, run);
  };
  auto g16 = [&](bcur_plan_t, GemmDesc d, int pr) {
    d.run_flag = run;
    return g16_on(P, ln, d, pr);
  };
  const bool step = chol_steps_apply(P, w);
  if (run && !step) return BCUR_EINVAL;  // the gated form needs the step path
  BCUR_TRY(fill_zero_if(L, (size_t)w * w * sizeof(float), run, s));
  BCUR_TRY(fill_zero_if(Li, (size_t)w * w * sizeof(float), run, s));
  BCUR_TRY(fill_zero_if(kept, sizeof(int), run, s));
  BCUR_TRY(max_diag<float>(G, w, w, md, s, run));
  const int64_t outer = step ? kOuterStep : kOuter;
  for (int64_t J0 = 0; J0 < w; J0 += outer) {
    const int64_t J1 = std::min(w, J0 + outer);
    for (int64_t j0 = J0; step && j0 < J1; j0 += nb)
      BCUR_TRY(chol_step(G, w, L, Li, J0, j0, md, tol, kept, s, run));
    for (int64_t j0 = J0; !step && j0 < J1; j0 += nb) {
      BCUR_TRY(potrf_diag<float>(G, w, L, w, Li, w, j0, nb, md, tol, kept, s));
      const int64_t j1 = j0 + nb;
      if (j1 >= w) break;
      // panel below the leaf, full height: L[j1:, j0:j1] = G[j1:, j0:j1] L_jj^{-T}
      GemmDesc pn = mk(w - j1, nb, nb, G + j1 * w + j0, w, 0, Li + j0 * w + j0, w, 1,
                       L + j1 * w + j0, w);
      pn.triB = 2;
      BCUR_TRY(gemm_simt<float>(pn, s));
      if (j1 < J1) {  // update the rest of this outer panel, all rows below
        BCUR_TRY(split(P, L + j1 * w + j0, w, w - j1, nb, Pn, nb));
        GemmDesc tr = mk16(w - j1, J1 - j1, nb, Pn, nb, 0, Pn, nb, 1, w);
        tr.D = G + j1 * w + j1;
        tr.alpha = -1.0;
        tr.beta = 1.0;
        tr.out_lower = 1;
        BCUR_TRY(g16(P, tr, parts));
      }
    }
    if (J1 < w) {  // outer trailing update with K = the outer panel width
      const int64_t kw = J1 - J0;
      BCUR_TRY(split(P, L + J1 * w + J0, w, w - J1, kw, Pn, kw));
      GemmDesc tr = mk16(w - J1, w - J1, kw, Pn, kw, 0, Pn, kw, 1, w);
      tr.D = G + J1 * w + J1;
      tr.alpha = -1.0;
      tr.beta = 1.0;
      tr.out_lower = 1;
      BCUR_TRY(g16(P, tr, parts));
    }
  }
  BCUR_TRY(split(P, L, w, w, w, L16, w));
  BCUR_TRY(split(P, Li, w, w, w, Li16, w));  // diagonal blocks; the doubling keeps it current
  for (int64_t h = nb; h < w; h *= 2) {
    const int64_t npairs_full = w / (2 * h);
    if (npairs_full > 0) {
      GemmDesc t1 = mk16(h, h, h, L16.off(h * w), w, 0, Li16, w, 0, h);
      t1.Dh = T1.h;
      t1.Dl = T1.l;
      t1.triB = 1;
      t1.batch = (int)npairs_full;
      t1.sA = 2 * h * (w + 1);
      t1.sB = 2 * h * (w + 1);
      t1.sD = h * h;
      BCUR_TRY(g16(P, t1, parts));
      GemmDesc t2 = mk16(h, h, h, Li16.off(h * w + h), w, 0, T1, h, 0, w);
      t2.D = Li + h * w;
      t2.Dh = Li16.h + h * w;
      t2.Dl = Li16.l ? Li16.l + h * w : nullptr;
      t2.triA = 1;
      t2.alpha = -1.0;
      t2.batch = (int)npairs_full;
      t2.sA = 2 * h * (w + 1);
      t2.sB = h * h;
      t2.sD = 2 * h * (w + 1);
      BCUR_TRY(g16(P, t2, parts));
    }
    const int64_t b1 = npairs_full * 2 * h, b2 = b1 + h;
    if (b2 < w) {
      const int64_t h2 = w - b2;
      GemmDesc t1 = mk16(h2, h, h, L16.off(b2 * w + b1), w, 0, Li16.off(b1 * w + b1), w, 0, h);
      t1.Dh = T1.h;
      t1.Dl = T1.l;
      t1.triB = 1;
      BCUR_TRY(g16(P, t1, parts));
      GemmDesc t2 = mk16(h2, h, h2, Li16.off(b2 * w + b2), w, 0, T1, h, 0, w);
      t2.D = Li + b2 * w + b1;
      t2.Dh = Li16.h + b2 * w + b1;
      t2.Dl = Li16.l ? Li16.l + b2 * w + b1 : nullptr;
      t2.triA = 1;
      t2.alpha = -1.0;
      BCUR_TRY(g16(P, t2, parts));
    }
  }
  return BCUR_OK;
}

// Wide Cholesky-QR2 of a BF16-pair panel X (w x h): X = L1 L2 Q.  The pairs
// pr[0] (input, then result) and pr[1] (intermediate) ping-pong.  With
// second_apply false the second pass stops at L2: pr[1] keeps Q1 = L1^{-1} X
// (Q = L2^{-1} Q1 is then applied to the small products instead).  parts2:
// the terms of the second pass's Gram and factorisation (0: parts).
bcur_status_t wide_cqr2_16(bcur_plan_t P, const Lane& ln, S16 pr[2], int64_t w, int64_t h,
                           int64_t ld, float* G, float* L1, float* L1i, float* L2, float* L2i,
                           int parts, int* kept, cudaEvent_t after_gram = nullptr,
                           bool second_apply = true, int parts2 = 0) {
  if (parts2 > 0 && parts2 != parts && second_apply) return BCUR_EINVAL;
  const bool lo = parts == 3;
  S16 Li16 = s16(P, ln.Lih, ln.Lil, lo);
  auto g16 = [&](bcur_plan_t, GemmDesc d, int pr2) { return g16_on(P, ln, d, pr2); };
  float* Ls[2] = {L1, L2};
  float* Lis[2] = {L1i, L2i};
  for (int pass = 0; pass < 2; ++pass) {
    S16 src = pr[pass], dst = pr[1 - pass];
    const int pt = (pass == 1 && parts2 > 0) ? parts2 : parts;
    GemmDesc g = mk16(w, w, h, src, ld, 0, src, ld, 1, w);
    g.D = G;
    g.out_lower = 1;
    BCUR_TRY(g16(P, g, pt));
    if (pass == 0 && after_gram) BCUR_CUDA_TRY(cudaEventRecord(after_gram, ln.s));
    BCUR_TRY(chol_inv_blocked16(P, ln, G, Ls[pass], Lis[pass], w, pt, kept + pass,
                                drop_tol<float>(h)));
    if (pass == 1 && !second_apply) break;
    GemmDesc a = mk16(w, h, w, Li16, w, 0, src, ld, 0, ld);  // Li16 holds L^{-1} already
    a.Dh = dst.h;
    a.Dl = dst.l;
    a.triA = 1;
    BCUR_TRY(g16(P, a, parts));
  }
  return BCUR_OK;
}

// The second Cholesky-QR pass of wide_cqr2_16 again with three terms (the
// Gram Q1^T Q1 of the pair q1 and its factorisation into L2, L2i), every
// launch gated by the device flag run: the refinement of the adaptive fit,
// which took this pass with one term first.  Same launches as the split fit's
// second pass, so a refined result is the split fit's bit for bit.
bcur_status_t redo_second_pass(bcur_plan_t P, S16 q1, int64_t w, int64_t h, int64_t ld, float* G,
                               float* L2, float* L2i, int* kept, const int* run) {
  const Lane ln = lane_of(P, 0);
  GemmDesc g = mk16(w, w, h, q1, ld, 0, q1, ld, 1, w);
  g.D = G;
  g.out_lower = 1;
  g.run_flag = run;
  BCUR_TRY(g16_on(P, ln, g, 3));
  return chol_inv_blocked16(P, ln, G, L2, L2i, w, 3, kept, drop_tol<float>(h), run);
}

// Stages 1-2 with the products by A on tensor cores.
bcur_status_t run_scores16(bcur_plan_t P, const float* A, const float* omega, double* cs,
                           double* rs) {
  const int l = P->l;
  const int parts = parts_of(P->d.sketch_prec);
  const bool lo = parts == 3;
  const int64_t m = P->m, n = P->n, lda = P->lda, ldm = P->ldm, ldn = P->ldn;
  float* Pm0 = P->at<float>(P->o.Pm0);
  float* Pm1 = P->at<float>(P->o.Pm1);
  float* Pn0 = P->at<float>(P->o.Pn0);
  float* Pn1 = P->at<float>(P->o.Pn1);
  S16 A16 = s16(P, P->o.A16h, P->o.A16l, lo);
  S16 Om = s16(P, P->o.Om16h, P->o.Om16l, lo);
  S16 Q16 = s16(P, P->o.Qm16h, P->o.Qm16l, lo);
  S16 Z16 = s16(P, P->o.Zn16h, P->o.Zn16l, lo);
  BCUR_TRY(split(P, A, lda, m, n, A16, ldn));
  BCUR_TRY(split(P, omega, n, l, n, Om, ldn));
  auto prodAt = [&](S16 X, float* Y) {  // Y^T (l x m) = X^T A^T, X^T panel l x n
    GemmDesc g = mk16(l, m, n, X, ldn, 0, A16, ldn, 1, ldm);
    g.D = Y;
    return g16(P, g, parts);
  };
  auto prodA = [&](S16 X, float* Z) {   // Z^T (l x n) = X^T A, X^T panel l x m
    GemmDesc g = mk16(l, n, m, X, ldm, 0, A16, ldn, 0, ldn);
    g.D = Z;
    return g16(P, g, parts);
  };
  const int ep = BCUR_F32;
  BCUR_TRY(prodAt(Om, Pm0));
  BCUR_TRY(orth_panel<float>(P, Pm0, Pm1, l, m, ldm, P->ksplit_m, ep, nullptr));
  for (int it = 0; it < P->q; ++it) {
    BCUR_TRY(split(P, Pm0, ldm, l, m, Q16, ldm));
    BCUR_TRY(prodA(Q16, Pn0));
    BCUR_TRY(orth_panel<float>(P, Pn0, Pn1, l, n, ldn, P->ksplit_n, ep, nullptr));
    BCUR_TRY(split(P, Pn0, ldn, l, n, Z16, ldn));
    BCUR_TRY(prodAt(Z16, Pm0));
    BCUR_TRY(orth_panel<float>(P, Pm0, Pm1, l, m, ldm, P->ksplit_m, ep, nullptr));
  }
  BCUR_TRY(split(P, Pm0, ldm, l, m, Q16, ldm));
  BCUR_TRY(prodA(Q16, Pn0));
  return scores_tail<float>(P, cs, rs);
}

// Stages 1-2 with the products by A on FP8 e4m3 tensor cores.  A is
// quantised once and kept twice (A8 and its transpose, so both products read
// K-major operands); each skinny panel is quantised per row before its
// product.  BCUR_FP8: one scale per row of A (A = diag(s_A) A8), folded into
// the panel when the product sums over the rows of A, so that every scale
// comes out of the products exactly and is applied in the GEMM epilogue.
// BCUR_FP8B: one scale per 128 x 128 block of A; a block's scale varies along
// K, so each 128-deep K block of a product is scaled as it is added (the
// GEMM's block-scaled path).  The panels stay FP32 and are re-orthonormalised
// after every product as in the BF16 form.
bcur_status_t run_scores8(bcur_plan_t P, const float* A, const float* omega, double* cs,
                          double* rs) {
  const bool blk = P->d.sketch_prec == BCUR_FP8B;
  cudaStream_t s = P->stream;
  const int l = P->l;
  const int64_t m = P->m, n = P->n, lda = P->lda, ldm = P->ldm, ldn = P->ldn;
  const int64_t ldm8 = round_up(m, 16), ldn8 = round_up(n, 16);
  float* Pm0 = P->at<float>(P->o.Pm0);
  float* Pm1 = P->at<float>(P->o.Pm1);
  float* Pn0 = P->at<float>(P->o.Pn0);
  float* Pn1 = P->at<float>(P->o.Pn1);
  uint8_t* A8 = P->at<uint8_t>(P->o.A8);
  uint8_t* A8T = P->at<uint8_t>(P->o.A8T);
  float* sA = P->at<float>(P->o.sA);
  uint8_t* X8m = P->at<uint8_t>(P->o.X8m);
  uint8_t* X8n = P->at<uint8_t>(P->o.X8n);
  float* sx = P->at<float>(P->o.sx);
  const int64_t gn = (n + 127) / 128;  // column blocks of A (block scales, row-major)
  if (blk) {
    BCUR_TRY(quant_blocks_e4m3(A, lda, m, n, A8, ldn8, A8T, ldm8, sA, s));
  } else {
    BCUR_TRY(quant_rows_e4m3(A, lda, m, n, nullptr, A8, ldn8, sA, s));
    BCUR_TRY(transpose_u8(A8, ldn8, m, n, A8T, ldm8, s));
  }
  // Y^T (l x m) = X^T A^T from the panel X^T (l x n):  D = X8 A8^T, rows
  // scaled by sx, columns by sA (per row), or each K block by its block's
  // scale (op(B) = A8^T seen as N x K is A8: block (row block, column block))
  auto prodAt = [&](const float* X, int64_t ldx, float* Y) {
    BCUR_TRY(quant_rows_e4m3(X, ldx, l, n, nullptr, X8n, ldn8, sx, s));
    GemmDesc g = mk(l, m, n, X8n, ldn8, 0, A8, ldn8, 1, Y, ldm);
    g.ab_fp8 = 1;
    g.scale_m = sx;
    if (blk) {
      g.bscale_b = sA;
      g.bs_n = gn;
      g.bs_k = 1;
    } else {
      g.scale_n = sA;
    }
    g.status = P->at<int>(P->o.status);
    return gemm_tc(g, BCUR_FP8, s);
  };
  // Z^T (l x n) = X^T A from the panel X^T (l x m):  X^T diag(s_A) is
  // quantised (per-row scales) or X^T itself (block scales: op(B) seen as
  // N x K is A8T, whose block (j, k) is A's block (k, j)), D = X8 A8T^T, rows
  // scaled by sx
  auto prodA = [&](const float* X, float* Z) {
    BCUR_TRY(quant_rows_e4m3(X, ldm, l, m, blk ? nullptr : sA, X8m, ldm8, sx, s));
    GemmDesc g = mk(l, n, m, X8m, ldm8, 0, A8T, ldm8, 1, Z, ldn);
    g.ab_fp8 = 1;
    g.scale_m = sx;
    if (blk) {
      g.bscale_b = sA;
      g.bs_n = 1;
      g.bs_k = gn;
    }
    g.status = P->at<int>(P->o.status);
    return gemm_tc(g, BCUR_FP8, s);
  };
  const int ep = BCUR_F32;
  BCUR_TRY(prodAt(omega, n, Pm0));  // the caller's Omega panel has leading dimension n
  BCUR_TRY(orth_panel<float>(P, Pm0, Pm1, l, m, ldm, P->ksplit_m, ep, nullptr));
  for (int it = 0; it < P->q; ++it) {
    BCUR_TRY(prodA(Pm0, Pn0));
    BCUR_TRY(orth_panel<float>(P, Pn0, Pn1, l, n, ldn, P->ksplit_n, ep, nullptr));
    BCUR_TRY(prodAt(Pn0, ldn, Pm0));
    BCUR_TRY(orth_panel<float>(P, Pm0, Pm1, l, m, ldm, P->ksplit_m, ep, nullptr));
  }
  BCUR_TRY(prodA(Pm0, Pn0));
  return scores_tail<float>(P, cs, rs);
}

// Stages 4-5 on tensor cores.
bcur_status_t resid16(bcur_plan_t P, const float* A, bool split3, int* flag, const int* run,
                      double* out, int mode);

bcur_status_t run_fit16(bcur_plan_t P, const float* A, const int32_t* ci, const int32_t* ri,
                        float* Uout, float* Cout, float* Rout) {
  cudaStream_t s = P->stream;
  const int parts = parts_of(P->d.fit_prec);
  const bool lo = parts == 3;
  const int64_t m = P->m, n = P->n, lda = P->lda, ldm = P->ldm, ldn = P->ldn;
  const int64_t cw = P->c_pad, rw = P->r_pad;
  int64_t* counts = P->at<int64_t>(P->o.counts);
  BCUR_TRY(expand_blocks(ci, P->d.g_col, P->at<int64_t>(P->o.col_off), P->d.G_col, cw,
                         P->at<int64_t>(P->o.colmap), counts, s));
  BCUR_TRY(expand_blocks(ri, P->d.g_row, P->at<int64_t>(P->o.row_off), P->d.G_row, rw,
                         P->at<int64_t>(P->o.rowmap), counts + 1, s));
  const int64_t* colmap = P->at<int64_t>(P->o.colmap);
  const int64_t* rowmap = P->at<int64_t>(P->o.rowmap);
  // C^T and R are gathered straight into their BF16 pairs (one read of the
  // chosen columns / rows of A, one write of the pair); the FP32 copies the
  // caller may ask for are gathered into its buffers.
  if (Cout) BCUR_TRY(gather_cols_t<float>(A, lda, m, colmap, P->c_max, Cout, m, s));
  if (Rout) BCUR_TRY(gather_rows<float>(A, lda, n, rowmap, P->r_max, Rout, n, s));
  S16 XC[2] = {s16(P, P->o.XC16[0], P->o.XC16[1], lo), s16(P, P->o.XC16[2], P->o.XC16[3], lo)};
  S16 XR[2] = {s16(P, P->o.XR16[0], P->o.XR16[1], lo), s16(P, P->o.XR16[2], P->o.XR16[3], lo)};
  BCUR_TRY(gather_cols_pair(A, lda, m, colmap, cw, XC[0].h, XC[0].l, ldm, s));
  BCUR_TRY(gather_rows_pair(A, lda, n, rowmap, rw, XR[0].h, XR[0].l, ldn, s));
  int* kept = P->at<int>(P->o.kept);
  // The QR factors of C and R^T are independent: the R side runs on the
  // second lane (fork / join through events, so this also works in a graph).
  // The R side starts when the C side's first Gram is done, so that each
  // side's latency-bound Cholesky steps run beside the other side's GEMMs
  // instead of beside each other.
  const Lane l0 = lane_of(P, 0), l1 = lane_of(P, 1);
  // The adaptive form takes the second pass's Gram Q1^T Q1 (near I) and its
  // factorisation with one BF16 term first: like M, it enters e only at
  // second order and U at first order at one term's level; the refinement
  // redoes that pass with three terms (redo_second_pass).
  const bool adapt = P->d.fit_prec == BCUR_BF16X3A;
  const bool pass2_one = adapt && chol_steps_apply(P, cw) && chol_steps_apply(P, rw);
  const int parts2 = pass2_one ? 1 : parts;
  BCUR_CUDA_TRY(cudaEventRecord(P->ev_fork, s));
  BCUR_CUDA_TRY(cudaStreamWaitEvent(P->stream2, P->ev_fork, 0));
  BCUR_TRY(wide_cqr2_16(P, l0, XC, cw, m, ldm, P->at<float>(P->o.GC), P->at<float>(P->o.L1C),
                        P->at<float>(P->o.L1Ci), P->at<float>(P->o.L2C), P->at<float>(P->o.L2Ci),
                        parts, kept + 4, P->ev_stagger, false, parts2));
  BCUR_CUDA_TRY(cudaStreamWaitEvent(P->stream2, P->ev_stagger, 0));
  BCUR_TRY(wide_cqr2_16(P, l1, XR, rw, n, ldn, P->at<float>(P->o.GR), P->at<float>(P->o.L1R),
                        P->at<float>(P->o.L1Ri), P->at<float>(P->o.L2R), P->at<float>(P->o.L2Ri),
                        parts, kept + 6, nullptr, false, parts2));
  BCUR_CUDA_TRY(cudaEventRecord(P->ev_join, P->stream2));
  BCUR_CUDA_TRY(cudaStreamWaitEvent(s, P->ev_join, 0));
  // The second Cholesky-QR pass stops at L2: with Q1 = X L1^{-T} (the pairs
  // XC[1], XR[1]) and Q = Q1 L2^{-T}, every product by Q becomes a product by
  // Q1 and a small triangular one.  W1 = A Q1_R (m x r); M1 = Q1_C^T W1
  // (c x r);
  //   M2 = L2C^{-T} L2C^{-1} M1 L2R^{-T} L2R^{-1}, so Q_C M Q_R^T = Q1_C M2 Q1_R^T
  //        (M = Q_C^T A Q_R; the residual uses M2 with Q1);
  //   U  = L1C^{-T} L2C^{-T} M L2R^{-1} L1R^{-1} = L1C^{-T} M2 L1R^{-1}.
  // Adaptive form (BCUR_BF16X3A): the products up to M2 and the residual
  // ||A - Q1_C M2 Q1_R^T||_F first with one BF16 term; when that residual is
  // too coarse for the error it reports (residual_needs_refine, decided on
  // the device) the same launches are redone with three terms (gated by the
  // flag, always enqueued so the sequence stays capturable), after the second
  // QR pass when it took one term, and the two products after M2 take the
  // flag's term count.  The residual is kept for bcur_error.
  S16 A16 = s16(P, P->o.A16h, P->o.A16l, lo);
  S16 W16 = s16(P, P->o.Wh, P->o.Wl, lo);
  S16 M16 = s16(P, P->o.Mh, P->o.Ml, lo);
  S16 Li16 = s16(P, P->o.Lih, P->o.Lil, lo);
  S16 U1 = s16(P, P->o.U1h, P->o.U1l, lo);
  S16 U2 = s16(P, P->o.U2h, P->o.U2l, lo);
  float* Uf = P->at<float>(P->o.U2);
  int* flag = P->at<int>(P->o.fit_flag);
  double* ferr = P->at<double>(P->o.fit_err);
  // The adaptive form needs A's lo half only if it refines (split then, gated
  // by the flag), and its hi half is the BF16 sketch's own copy when the
  // scores were taken of this A.
  if (!adapt) BCUR_TRY(split(P, A, lda, m, n, A16, ldn));
  else if (A != P->scores_A16) BCUR_TRY(split_bf16(A, lda, m, n, A16.h, nullptr, ldn, s));
  auto tri = [&](GemmDesc d, S16 out, float* outf, int pr, const int* run, const int* terms) {
    d.Dh = out.h;
    d.Dl = out.l;
    d.D = outf;
    d.run_flag = run;
    d.parts_flag = terms;
    return g16(P, d, pr);
  };
  // W1, M1 and M2 with pr terms (launches skipped unless *run when run is set)
  auto to_m2 = [&](int pr, const int* run) -> bcur_status_t {
    BCUR_TRY(tri(mk16(m, rw, n, A16, ldn, 0, XR[1], ldn, 1, rw), W16, nullptr, pr, run, nullptr));
    BCUR_TRY(tri(mk16(cw, rw, m, XC[1], ldm, 0, W16, rw, 0, rw), M16, nullptr, pr, run, nullptr));
    BCUR_TRY(split(P, P->at<float>(P->o.L2Ri), rw, rw, rw, Li16, rw));
    GemmDesc t1 = mk16(cw, rw, rw, M16, rw, 0, Li16, rw, 1, rw);  // M1 L2R^{-T}
    t1.triB = 2;
    BCUR_TRY(tri(t1, U1, nullptr, pr, run, nullptr));
    GemmDesc t2 = mk16(cw, rw, rw, U1, rw, 0, Li16, rw, 0, rw);   // ... L2R^{-1}
    t2.triB = 1;
    BCUR_TRY(tri(t2, U2, nullptr, pr, run, nullptr));
    BCUR_TRY(split(P, P->at<float>(P->o.L2Ci), cw, cw, cw, Li16, cw));
    GemmDesc t3 = mk16(cw, rw, cw, Li16, cw, 0, U2, rw, 0, rw);   // L2C^{-1} ...
    t3.triA = 1;
    BCUR_TRY(tri(t3, U1, nullptr, pr, run, nullptr));
    GemmDesc t4 = mk16(cw, rw, cw, Li16, cw, 1, U1, rw, 0, rw);   // M2 = L2C^{-T} ...
    t4.triA = 2;
    return tri(t4, M16, P->at<float>(P->o.Mb), pr, run, nullptr);
  };
  if (adapt) {
    BCUR_TRY(to_m2(1, nullptr));
    BCUR_TRY(resid16(P, A, false, flag, nullptr, ferr, 2));
    BCUR_TRY(split_bf16(A, lda, m, n, nullptr, A16.l, ldn, s, false, flag));
    if (pass2_one) {
      BCUR_TRY(redo_second_pass(P, XC[1], cw, m, ldm, P->at<float>(P->o.GC),
                                P->at<float>(P->o.L2C), P->at<float>(P->o.L2Ci), kept + 5, flag));
      BCUR_TRY(redo_second_pass(P, XR[1], rw, n, ldn, P->at<float>(P->o.GR),
                                P->at<float>(P->o.L2R), P->at<float>(P->o.L2Ri), kept + 7, flag));
    }
    BCUR_TRY(to_m2(3, flag));
    BCUR_TRY(resid16(P, A, true, flag, flag, ferr + 3, 3));
    BCUR_TRY(select_result(ferr, ferr + 3, flag, ferr + 6, s));
  } else {
    BCUR_TRY(to_m2(parts, nullptr));
  }
  const int* dyn = adapt ? flag : nullptr;
  BCUR_TRY(split(P, P->at<float>(P->o.L1Ri), rw, rw, rw, Li16, rw));
  GemmDesc t5 = mk16(cw, rw, rw, M16, rw, 0, Li16, rw, 0, rw);    // M2 L1R^{-1}
  t5.triB = 1;
  BCUR_TRY(tri(t5, U2, nullptr, parts, nullptr, dyn));
  BCUR_TRY(split(P, P->at<float>(P->o.L1Ci), cw, cw, cw, Li16, cw));
  GemmDesc t6 = mk16(cw, rw, cw, Li16, cw, 1, U2, rw, 0, rw);     // U = L1C^{-T} ...
  t6.triA = 2;
  BCUR_TRY(tri(t6, S16{}, Uf, parts, nullptr, dyn));
  if (Uout) BCUR_TRY(copy2d<float>(Uf, rw, Uout, P->r_max, P->c_max, P->r_max, s));
  return BCUR_OK;
}

// One pass of the tensor-core residual: P = Q1_C M2 (m x r) and
// sum (A - P Q1_R^T)^2 in the GEMM epilogue, with one BF16 term (split3
// false) or BF16 pairs; launches skipped unless *run when run is set; the
// partial sums reduced into out (finish_residual mode, refinement flag).
bcur_status_t resid16(bcur_plan_t P, const float* A, bool split3, int* flag, const int* run,
                      double* out, int mode) {
  const int64_t m = P->m, n = P->n, ldm = P->ldm, ldn = P->ldn;
  const int64_t cw = P->c_pad, rw = P->r_pad;
  S16 QC = s16(P, P->o.XC16[2], P->o.XC16[3], split3);  // Q1_C, Q1_R (with M2, see run_fit16)
  S16 QR = s16(P, P->o.XR16[2], P->o.XR16[3], split3);
  S16 M16 = s16(P, P->o.Mh, P->o.Ml, split3);
  S16 Pp = s16(P, P->o.Ph, P->o.Pl, split3);
  GemmDesc g = mk16(m, rw, cw, QC, ldm, 1, M16, rw, 0, rw);
  g.Dh = Pp.h;
  g.Dl = Pp.l;
  g.run_flag = run;
  BCUR_TRY(g16(P, g, split3 ? 3 : 1));
  GemmDesc r = mk16(m, n, rw, Pp, rw, 0, QR, ldn, 0, 0);
  r.X = A;
  r.ldx = P->lda;
  r.partials = P->at<double>(P->o.partials);
  r.parts = split3 ? 3 : 1;
  r.status = P->at<int>(P->o.status);
  r.run_flag = run;
  int64_t np = 0;
  BCUR_TRY(gemm_tc_resid(r, BCUR_BF16, P->stream, &np));
  return finish_residual(P->at<double>(P->o.partials), np, out, mode, P->stream, flag);
}

// Stage 6 on tensor cores: P = Q_C^T M, then sum (A - P Q_R)^2 in the GEMM
// epilogue.  First with one BF16 term; when the fit runs in BF16 pairs and
// the one-term result is too coarse for the relative error it reports
// (residual_needs_refine, decided on the device), P and the residual are
// recomputed with BF16 pairs.  The second pair of launches is always
// enqueued (the sequence stays capturable) and does nothing unless the flag
// is set.  The adaptive fit has taken this residual already: for the same A
// it is copied.
bcur_status_t run_error16(bcur_plan_t P, const float* A, double* out) {
  if (P->d.fit_prec == BCUR_BF16X3A && A == P->fit_A) {
    BCUR_CUDA_TRY(cudaMemcpyAsync(out, P->at<double>(P->o.fit_err) + 6, 3 * sizeof(double),
                                  cudaMemcpyDeviceToDevice, P->stream));
    return BCUR_OK;
  }
  const int parts = parts_of(P->d.fit_prec);
  int* flag = P->at<int>(P->o.refine);
  BCUR_TRY(resid16(P, A, false, flag, nullptr, out, parts == 3 ? 2 : 0));
  if (parts == 3) BCUR_TRY(resid16(P, A, true, flag, flag, out, 3));
  return BCUR_OK;
}


// --- Rank-k truncation of U (Sec. 4.1) -------------------------------------
// Randomized top-kt SVD of U (c x r, in the workspace) with the plan's
// skinny temporaries, then U_k = Ut_k^T diag(sigma) V_k and
// ||A - C U_k R||_F through P_k = C Ut_k^T (m x kt) and Q_k = diag(sigma) V_k R
// (kt x n) in the fused residual.  CUDA cores, storage precision.
template <typename T>
bcur_status_t run_truncate(bcur_plan_t P, const T* A, int kt, const T* omega, T* Ukout,
                           double* out) {
  cudaStream_t s = P->stream;
  const int l = P->l;
  const int64_t m = P->m, n = P->n, lda = P->lda, ldm = P->ldm, ldn = P->ldn;
  const int64_t cw = P->c_pad, rw = P->r_pad, c = P->c_max, r = P->r_max;
  const int ex = exact_prec<T>();
  T* U = P->at<T>(P->o.U2);  // c_pad x r_pad, ld r_pad
  T* Ym = P->at<T>(P->o.Pm0);
  T* Ym1 = P->at<T>(P->o.Pm1);
  T* Zn = P->at<T>(P->o.Pn0);
  T* Zn1 = P->at<T>(P->o.Pn1);
  const int ks_c = (int)std::max<int64_t>(1, std::min<int64_t>(2 * P->sms, cw / 64));
  const int ks_r = (int)std::max<int64_t>(1, std::min<int64_t>(2 * P->sms, rw / 64));
  // range finder on U: Y^T = Omega^T U^T, q steps of subspace iteration
  BCUR_TRY(gemm_simt<T>(mk(l, cw, r, omega, r, 0, U, rw, 1, Ym, ldm), s));
  BCUR_TRY(orth_panel<T>(P, Ym, Ym1, l, cw, ldm, ks_c, ex, nullptr));
  for (int it = 0; it < P->q; ++it) {
    BCUR_TRY(gemm_simt<T>(mk(l, rw, cw, Ym, ldm, 0, U, rw, 0, Zn, ldn), s));
    BCUR_TRY(orth_panel<T>(P, Zn, Zn1, l, rw, ldn, ks_r, ex, nullptr));
    BCUR_TRY(gemm_simt<T>(mk(l, cw, rw, Zn, ldn, 0, U, rw, 1, Ym, ldm), s));
    BCUR_TRY(orth_panel<T>(P, Ym, Ym1, l, cw, ldm, ks_c, ex, nullptr));
  }
  BCUR_TRY(gemm_simt<T>(mk(l, rw, cw, Ym, ldm, 0, U, rw, 0, Zn, ldn), s));
  double* LB = P->at<double>(P->o.Lprod64);
  BCUR_TRY(orth_panel<T>(P, Zn, Zn1, l, rw, ldn, ks_r, ex, LB));
  T* Ut = P->at<T>(P->o.Ut);
  T* W = P->at<T>(P->o.W);
  double* sig = P->at<double>(P->o.sigma) + l;  // second half of the sigma slot
  BCUR_TRY(jacobi_svd_small<T>(LB, l, Ut, W, sig, P->at<T>(P->o.jwork), P->at<int>(P->o.status),
                               s));
  // Left factor X = Ut_k^T Q^T (kt x c) and right factor Y = diag(sigma) W_k^T Q_B^T (kt x r).
  T* Xp = P->at<T>(P->o.Pm1);
  T* Yp = P->at<T>(P->o.Pn1);
  BCUR_TRY(gemm_simt<T>(mk(kt, cw, l, Ut, l, 1, Ym, ldm, 0, Xp, ldm), s));
  BCUR_TRY(gemm_simt<T>(mk(kt, rw, l, W, l, 1, Zn, ldn, 0, Yp, ldn), s));
  BCUR_TRY(scale_rows_by(Yp, kt, rw, ldn, sig, s));
  if (Ukout) {  // U_k = X^T Y
    T* Ub = P->at<T>(P->o.U1);
    BCUR_TRY(gemm_simt<T>(mk(cw, rw, kt, Xp, ldm, 1, Yp, ldn, 0, Ub, rw), s));
    BCUR_TRY(copy2d<T>(Ub, rw, Ukout, r, c, r, s));
  }
  // C and R gathered again (the fit may have overwritten them with Q factors)
  T* Cp = P->at<T>(P->o.Cp1);
  T* Rp = P->at<T>(P->o.Rp1);
  BCUR_TRY(gather_cols_t<T>(A, lda, m, P->at<int64_t>(P->o.colmap), cw, Cp, ldm, s));
  BCUR_TRY(gather_rows<T>(A, lda, n, P->at<int64_t>(P->o.rowmap), rw, Rp, ldn, s));
  // P_k = C X^T (m x kt) = Cp^T X^T;  Q_k = Y R (kt x n)
  T* Pk = P->at<T>(P->o.Wb);
  T* Qk = P->at<T>(P->o.Pn2);
  BCUR_TRY(gemm_simt<T>(mk(m, kt, cw, Cp, ldm, 1, Xp, ldm, 1, Pk, kt), s));
  BCUR_TRY(gemm_simt<T>(mk(kt, n, rw, Yp, ldn, 0, Rp, ldn, 0, Qk, ldn), s));
  GemmDesc rd = mk(m, n, kt, Pk, kt, 0, Qk, ldn, 0, nullptr, 0);
  rd.X = A;
  rd.ldx = lda;
  rd.partials = P->at<double>(P->o.partials);
  int64_t np = 0;
  BCUR_TRY(gemm_simt_resid<T>(rd, s, &np));
  return finish_residual(P->at<double>(P->o.partials), np, out, 0, s);
}

// ||A - U_k Sigma_k V_k^T||_F from the factors of the last bcur_scores (the
// fused residual with P = U_k, Q = Sigma_k V_k^T; CUDA cores, storage
// precision) and its ratio to the last ||A - CUR||_F.
template <typename T>
bcur_status_t run_rank_k(bcur_plan_t P, const T* A, double* out) {
  cudaStream_t s = P->stream;
  const int k = P->k;
  const int64_t m = P->m, n = P->n, ldm = P->ldm, ldn = P->ldn;
  T* Q = P->at<T>(P->o.Pn2);
  BCUR_TRY(copy2d<T>(P->at<T>(P->o.Vp), ldn, Q, ldn, k, n, s));
  BCUR_TRY(scale_rows_by<T>(Q, k, n, ldn, P->at<double>(P->o.sigma), s));
  GemmDesc r = mk(m, n, k, P->at<T>(P->o.Up), ldm, 1, Q, ldn, 0, nullptr, 0);
  r.X = A;
  r.ldx = P->lda;
  r.partials = P->at<double>(P->o.partials);
  int64_t np = 0;
  BCUR_TRY(gemm_simt_resid<T>(r, s, &np));
  return rank_k_ratio(P->at<double>(P->o.result), P->at<double>(P->o.partials), np, out, s);
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* bcur_version(void) { return "0.1.0"; }

uint64_t bcur_launch_count(void) { return (uint64_t)g_launches.load(); }

bcur_status_t bcur_set_wait_budget_ns(uint64_t ns) {
  if (ns == 0 || ns > 60000000000ull) return BCUR_EINVAL;
  return gemm_tc_set_wait_budget(ns);
}

bcur_status_t bcur_gemm_split(int64_t M, int64_t N, int64_t K, const void* A_hi, const void* A_lo,
                              int64_t lda, int32_t transA, const void* B_hi, const void* B_lo,
                              int64_t ldb, int32_t transB, float* D, int64_t ldd, void* stream) {
  if (!A_hi || !A_lo || !B_hi || !B_lo || !D || M < 0 || N < 0 || K < 0) return BCUR_EINVAL;
  GemmDesc g = mk(M, N, K, A_hi, lda, transA != 0, B_hi, ldb, transB != 0, D, ldd);
  g.ab_bf16 = 1;
  g.parts = 3;
  g.A_lo = A_lo;
  g.B_lo = B_lo;
  return gemm_tc(g, BCUR_BF16, (cudaStream_t)stream);
}

const char* bcur_status_string(bcur_status_t st) {
  switch (st) {
    case BCUR_OK: return "ok";
    case BCUR_EINVAL: return "invalid argument";
    case BCUR_ENOMEM: return "workspace missing or too small";
    case BCUR_ECUDA: return g_last_err[0] ? g_last_err : "CUDA error";
    case BCUR_ERANK: return "rank breakdown";
    case BCUR_ENONFINITE: return "non-finite value in the data";
    case BCUR_ETIMEOUT: return "device wait timed out";
    case BCUR_ENOTSUP: return "not supported";
    case BCUR_ESTATE: return "call out of order";
  }
  return "unknown status";
}

bcur_status_t bcur_plan(const bcur_desc_t* d, void* stream, bcur_plan_t* out,
                        size_t* workspace_bytes) {
  if (!d || !out) return BCUR_EINVAL;
  *out = nullptr;
  if (d->m < 1 || d->n < 1 || d->lda < d->n) return BCUR_EINVAL;
  if (d->a_dtype != BCUR_F64 && d->a_dtype != BCUR_F32) return BCUR_EINVAL;
  if (d->k < 1 || d->p < 0 || d->q < 0 || d->q > 16) return BCUR_EINVAL;
  const int64_t l = (int64_t)d->k + d->p;
  if (l > 128 || l > d->m || l > d->n) return BCUR_EINVAL;
  if (d->G_col < 1 || d->G_row < 1 || d->G_col > 32768 || d->G_row > 32768) return BCUR_EINVAL;
  if (!valid_offsets(d->col_off, d->G_col, d->n) || !valid_offsets(d->row_off, d->G_row, d->m))
    return BCUR_EINVAL;
  if (d->g_col < 1 || d->g_row < 1) return BCUR_EINVAL;
  if (!d->replacement && (d->g_col > d->G_col || d->g_row > d->G_row)) return BCUR_EINVAL;
  const bool fp8 = d->sketch_prec == BCUR_FP8 || d->sketch_prec == BCUR_FP8B;
  if (fp8 && d->a_dtype != BCUR_F32) return BCUR_EINVAL;
  // FP8 is a sketch precision only
  if (d->fit_prec == BCUR_FP8 || d->fit_prec == BCUR_FP8B) return BCUR_EINVAL;
  if (d->sketch_prec == BCUR_BF16X3A) return BCUR_EINVAL;  // the adaptive form is a fit's
  for (int p : {d->sketch_prec, d->fit_prec}) {
    if (p == BCUR_FP8 || p == BCUR_FP8B) continue;
    if (p < BCUR_F64 || p > BCUR_BF16X3A) return BCUR_EINVAL;
    if (d->a_dtype == BCUR_F64 && p != BCUR_F64) return BCUR_EINVAL;
    if (d->a_dtype == BCUR_F32 && p == BCUR_F64) return BCUR_EINVAL;
    if (p == BCUR_TF32) return BCUR_ENOTSUP;
  }
  // A single BF16 term cannot keep Cholesky-QR of C and R^T stable (kappa^2
  // times 2^-9 exceeds 1 for kappa ~ 50): the fit needs F32 or split BF16.
  if (d->fit_prec == BCUR_BF16) return BCUR_ENOTSUP;
  bcur_plan_t P = new (std::nothrow) bcur_plan_s();
  if (!P) return BCUR_ENOMEM;
  P->d = *d;
  P->col_off.assign(d->col_off, d->col_off + d->G_col + 1);
  P->row_off.assign(d->row_off, d->row_off + d->G_row + 1);
  P->d.col_off = P->col_off.data();
  P->d.row_off = P->row_off.data();
  P->stream = (cudaStream_t)stream;
  P->m = d->m; P->n = d->n; P->lda = d->lda;
  P->k = d->k; P->l = (int)l; P->q = d->q;
  P->esz = d->a_dtype == BCUR_F64 ? 8 : 4;
  P->nb = 64;
  P->ldm = round_up(P->m, 32);
  P->ldn = round_up(P->n, 32);
  P->c_max = max_sum_of_g(P->col_off, d->g_col, d->replacement != 0);
  P->r_max = max_sum_of_g(P->row_off, d->g_row, d->replacement != 0);
  P->c_pad = round_up(P->c_max, P->nb);
  P->r_pad = round_up(P->r_max, P->nb);
  if (P->c_pad > 65535 || P->r_pad > 65535) { delete P; return BCUR_EINVAL; }
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
    P->sms = sms;
  else
    cudaGetLastError();
  P->ksplit_m = (int)std::max<int64_t>(1, std::min<int64_t>(2 * P->sms, P->m / 64));
  P->ksplit_n = (int)std::max<int64_t>(1, std::min<int64_t>(2 * P->sms, P->n / 64));

  Layout L;
  const size_t e = P->esz;
  const int64_t ll = l * l;
  auto& o = P->o;
  o.Pm0 = L.take(l * P->ldm * e);
  o.Pm1 = L.take(l * P->ldm * e);
  o.Pn0 = L.take(l * P->ldn * e);
  o.Pn1 = L.take(l * P->ldn * e);
  o.Pn2 = L.take(l * P->ldn * e);
  o.gram_part = L.take((size_t)std::max(P->ksplit_m, P->ksplit_n) * ll * e);
  o.G64 = L.take(ll * 8);
  o.L64a = L.take(ll * 8);
  o.L64b = L.take(ll * 8);
  o.Lprod64 = L.take(ll * 8);
  o.Linv64 = L.take(ll * 8);
  o.LinvT = L.take(ll * e);
  o.Ut = L.take(ll * e);
  o.W = L.take(ll * e);
  o.sigma = L.take(2 * l * 8);
  o.jwork = L.take((l + 1) * (l + 1) * e);
  o.Vp = L.take((int64_t)P->k * P->ldn * e);
  o.Up = L.take((int64_t)P->k * P->ldm * e);
  o.col_off = L.take((P->d.G_col + 1) * 8);
  o.row_off = L.take((P->d.G_row + 1) * 8);
  o.status = L.take(16);
  o.kept = L.take(64);
  const int64_t cw = P->c_pad, rw = P->r_pad;
  o.colmap = L.take(cw * 8);
  o.rowmap = L.take(rw * 8);
  o.counts = L.take(16);
  o.Cp0 = L.take(cw * P->ldm * e);
  o.Cp1 = L.take(cw * P->ldm * e);
  o.Rp0 = L.take(rw * P->ldn * e);
  o.Rp1 = L.take(rw * P->ldn * e);
  o.GC = L.take(cw * cw * e);
  o.L1C = L.take(cw * cw * e);
  o.L1Ci = L.take(cw * cw * e);
  o.L2C = L.take(cw * cw * e);
  o.L2Ci = L.take(cw * cw * e);
  o.GR = L.take(rw * rw * e);
  o.L1R = L.take(rw * rw * e);
  o.L1Ri = L.take(rw * rw * e);
  o.L2R = L.take(rw * rw * e);
  o.L2Ri = L.take(rw * rw * e);
  o.maxdiag = L.take(16);
  o.Wb = L.take(P->m * rw * e);
  o.Mb = L.take(cw * rw * e);
  o.U1 = L.take(cw * rw * e);
  o.U2 = L.take(cw * rw * e);
  P->n_partials = std::max(gemm_simt_resid_ctas<double>(P->m, P->n),
                           std::max(gemm_simt_resid_ctas<float>(P->m, P->n),
                                    gemm_tc_resid_ctas(P->m, P->n)));
  o.partials = L.take(2 * P->n_partials * 8);
  o.result = L.take(64);
  P->bf16_path = is_bf16_prec(d->sketch_prec) || is_bf16_prec(d->fit_prec);
  P->tc_scratch_bytes = P->bf16_path ? (64u << 20) : 0;
  o.tc_scratch = L.take(P->tc_scratch_bytes);
  if (P->bf16_path) {
    const size_t h2 = 2;  // bytes per BF16
    const int64_t wm = std::max(cw, rw);
    const bool s3 = d->sketch_prec == BCUR_BF16X3, f3 = parts_of(d->fit_prec) == 3;
    const bool any3 = s3 || f3;
    o.A16h = L.take(P->m * P->ldn * h2);
    o.A16l = L.take(any3 ? P->m * P->ldn * h2 : 0);
    o.Om16h = L.take(l * P->ldn * h2);
    o.Om16l = L.take(l * P->ldn * h2);
    o.Qm16h = L.take(l * P->ldm * h2);
    o.Qm16l = L.take(l * P->ldm * h2);
    o.Zn16h = L.take(l * P->ldn * h2);
    o.Zn16l = L.take(l * P->ldn * h2);
    if (is_bf16_prec(d->fit_prec)) {
      for (int i = 0; i < 4; ++i) o.XC16[i] = L.take(cw * P->ldm * h2);
      for (int i = 0; i < 4; ++i) o.XR16[i] = L.take(rw * P->ldn * h2);
      o.Lh = L.take(wm * wm * h2);
      o.Ll = L.take(wm * wm * h2);
      o.Lih = L.take(wm * wm * h2);
      o.Lil = L.take(wm * wm * h2);
      o.T1h = L.take(wm * wm * h2);
      o.T1l = L.take(wm * wm * h2);
      o.Pnh = L.take(wm * std::min<int64_t>(wm, 1024) * h2);
      o.Pnl = L.take(wm * std::min<int64_t>(wm, 1024) * h2);
      o.Wh = L.take(P->m * rw * h2);
      o.Wl = L.take(P->m * rw * h2);
      o.Mh = L.take(cw * rw * h2);
      o.Ml = L.take(cw * rw * h2);
      o.U1h = L.take(cw * rw * h2);
      o.U1l = L.take(cw * rw * h2);
      o.U2h = L.take(cw * rw * h2);
      o.U2l = L.take(cw * rw * h2);
      o.Ph = L.take(P->m * rw * h2);
      o.Pl = L.take(P->m * rw * h2);
      o.refine = L.take(sizeof(int));
      o.fit_flag = L.take(sizeof(int));
      o.fit_err = L.take(9 * sizeof(double));
      o.Lh2 = L.take(wm * wm * h2);
      o.Ll2 = L.take(wm * wm * h2);
      o.Lih2 = L.take(wm * wm * h2);
      o.Lil2 = L.take(wm * wm * h2);
      o.T1h2 = L.take(wm * wm * h2);
      o.T1l2 = L.take(wm * wm * h2);
      o.Pnh2 = L.take(wm * std::min<int64_t>(wm, 1024) * h2);
      o.Pnl2 = L.take(wm * std::min<int64_t>(wm, 1024) * h2);
      o.maxdiag2 = L.take(16);
      o.tc_scratch2 = L.take(P->tc_scratch_bytes);
    }
  }
  if (fp8) {
    const int64_t ldm8 = round_up(P->m, 16), ldn8 = round_up(P->n, 16);
    o.A8 = L.take(P->m * ldn8);
    o.A8T = L.take(P->n * ldm8);
    // row scales (FP8) or 128 x 128 block scales (FP8B)
    o.sA = L.take(4 * std::max<int64_t>(P->m, ((P->m + 127) / 128) * ((P->n + 127) / 128)));
    o.X8m = L.take(l * ldm8);
    o.X8n = L.take(l * ldn8);
    o.sx = L.take(l * 4);
  }
  P->need = L.cur;
  if (workspace_bytes) *workspace_bytes = P->need;
  *out = P;
  return BCUR_OK;
}

bcur_status_t bcur_set_workspace(bcur_plan_t P, void* ws, size_t bytes) {
  if (!plan_ok(P) || !ws || ((uintptr_t)ws & 255)) return BCUR_EINVAL;
  if (bytes < P->need) return BCUR_ENOMEM;
  if (!P->stream2) {
    BCUR_CUDA_TRY(cudaStreamCreateWithFlags(&P->stream2, cudaStreamNonBlocking));
    BCUR_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
    BCUR_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
    BCUR_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_stagger, cudaEventDisableTiming));
  }
  P->ws = (char*)ws;
  P->ws_bytes = bytes;
  cudaStream_t s = P->stream;
  BCUR_CUDA_TRY(cudaMemcpyAsync(P->at<int64_t>(P->o.col_off), P->col_off.data(),
                                P->col_off.size() * 8, cudaMemcpyHostToDevice, s));
  BCUR_CUDA_TRY(cudaMemcpyAsync(P->at<int64_t>(P->o.row_off), P->row_off.data(),
                                P->row_off.size() * 8, cudaMemcpyHostToDevice, s));
  BCUR_CUDA_TRY(cudaMemsetAsync(P->at<int>(P->o.status), 0, 16, s));
  // Panels are read with padded leading dimensions: clear the padding once.
  BCUR_CUDA_TRY(cudaMemsetAsync(P->ws, 0, P->need, s));
  BCUR_CUDA_TRY(cudaMemcpyAsync(P->at<int64_t>(P->o.col_off), P->col_off.data(),
                                P->col_off.size() * 8, cudaMemcpyHostToDevice, s));
  BCUR_CUDA_TRY(cudaMemcpyAsync(P->at<int64_t>(P->o.row_off), P->row_off.data(),
                                P->row_off.size() * 8, cudaMemcpyHostToDevice, s));
  BCUR_CUDA_TRY(cudaStreamSynchronize(s));
  P->have_scores = P->have_fit = false;
  P->fit_A = nullptr;
  P->scores_A16 = nullptr;
  return BCUR_OK;
}

bcur_status_t bcur_scores(bcur_plan_t P, const void* A, const void* omega, double* cs,
                          double* rs) {
  if (!plan_ok(P)) return BCUR_EINVAL;
  if (!P->ws) return BCUR_ESTATE;
  if (!A || !omega || !cs || !rs) return BCUR_EINVAL;
  bcur_status_t st;
  if (P->d.a_dtype == BCUR_F64)
    st = run_scores<double>(P, (const double*)A, (const double*)omega, cs, rs);
  else if (is_bf16_prec(P->d.sketch_prec))
    st = run_scores16(P, (const float*)A, (const float*)omega, cs, rs);
  else if (P->d.sketch_prec == BCUR_FP8 || P->d.sketch_prec == BCUR_FP8B)
    st = run_scores8(P, (const float*)A, (const float*)omega, cs, rs);
  else
    st = run_scores<float>(P, (const float*)A, (const float*)omega, cs, rs);
  if (st == BCUR_OK) P->have_scores = true;
  P->scores_A16 = (st == BCUR_OK && P->d.a_dtype == BCUR_F32 && is_bf16_prec(P->d.sketch_prec))
                      ? A : nullptr;
  return st;
}

bcur_status_t bcur_factors(bcur_plan_t P, void* Vt, void* Ut, double* sigma) {
  if (!plan_ok(P)) return BCUR_EINVAL;
  if (!P->ws || !P->have_scores) return BCUR_ESTATE;
  cudaStream_t s = P->stream;
  if (P->d.a_dtype == BCUR_F64) {
    if (Vt) BCUR_TRY(copy2d<double>(P->at<double>(P->o.Vp), P->ldn, (double*)Vt, P->n, P->k, P->n, s));
    if (Ut) BCUR_TRY(copy2d<double>(P->at<double>(P->o.Up), P->ldm, (double*)Ut, P->m, P->k, P->m, s));
  } else {
    if (Vt) BCUR_TRY(copy2d<float>(P->at<float>(P->o.Vp), P->ldn, (float*)Vt, P->n, P->k, P->n, s));
    if (Ut) BCUR_TRY(copy2d<float>(P->at<float>(P->o.Up), P->ldm, (float*)Ut, P->m, P->k, P->m, s));
  }
  if (sigma)
    BCUR_CUDA_TRY(cudaMemcpyAsync(sigma, P->at<double>(P->o.sigma), P->k * sizeof(double),
                                  cudaMemcpyDeviceToDevice, s));
  return BCUR_OK;
}

bcur_status_t bcur_sample(bcur_plan_t P, const double* cs, const double* rs, const double* uc,
                          const double* ur, int32_t* ci, int32_t* ri, double* cp, double* rp) {
  if (!plan_ok(P)) return BCUR_EINVAL;
  if (!cs || !rs || !uc || !ur || !ci || !ri) return BCUR_EINVAL;
  BCUR_TRY(sample_blocks(cs, P->d.G_col, uc, P->d.g_col, P->d.replacement, ci, cp, P->stream));
  BCUR_TRY(sample_blocks(rs, P->d.G_row, ur, P->d.g_row, P->d.replacement, ri, rp, P->stream));
  return BCUR_OK;
}

bcur_status_t bcur_fit(bcur_plan_t P, const void* A, const int32_t* ci, const int32_t* ri, void* U,
                       void* C, void* R) {
  if (!plan_ok(P)) return BCUR_EINVAL;
  if (!P->ws) return BCUR_ESTATE;
  if (!A || !ci || !ri) return BCUR_EINVAL;
  bcur_status_t st;
  if (P->d.a_dtype == BCUR_F64)
    st = run_fit<double>(P, (const double*)A, ci, ri, (double*)U, (double*)C, (double*)R);
  else if (is_bf16_prec(P->d.fit_prec))
    st = run_fit16(P, (const float*)A, ci, ri, (float*)U, (float*)C, (float*)R);
  else
    st = run_fit<float>(P, (const float*)A, ci, ri, (float*)U, (float*)C, (float*)R);
  P->have_fit = (st == BCUR_OK);
  P->have_error = false;
  P->fit_A = (st == BCUR_OK && P->d.fit_prec == BCUR_BF16X3A) ? A : nullptr;
  return st;
}

bcur_status_t bcur_fit_terms(bcur_plan_t P, int32_t* terms, double* est) {
  if (!plan_ok(P) || !terms) return BCUR_EINVAL;
  if (!P->ws || !P->have_fit) return BCUR_ESTATE;
  if (est) *est = -1.0;
  if (P->d.a_dtype == BCUR_F64 || !is_bf16_prec(P->d.fit_prec)) {
    *terms = 0;
    return BCUR_OK;
  }
  if (P->d.fit_prec != BCUR_BF16X3A) {
    *terms = parts_of(P->d.fit_prec);
    return BCUR_OK;
  }
  int flag = 0;
  double e1[3] = {-1.0, -1.0, -1.0};
  BCUR_CUDA_TRY(cudaMemcpyAsync(&flag, P->at<int>(P->o.fit_flag), sizeof(int),
                                cudaMemcpyDeviceToHost, P->stream));
  BCUR_CUDA_TRY(cudaMemcpyAsync(e1, P->at<double>(P->o.fit_err), sizeof(e1),
                                cudaMemcpyDeviceToHost, P->stream));
  BCUR_CUDA_TRY(cudaStreamSynchronize(P->stream));
  *terms = flag ? 3 : 1;
  if (est) *est = e1[1];
  return BCUR_OK;
}

bcur_status_t bcur_error(bcur_plan_t P, const void* A, double* out) {
  if (!plan_ok(P)) return BCUR_EINVAL;
  if (!P->ws || !P->have_fit) return BCUR_ESTATE;
  if (!A || !out) return BCUR_EINVAL;
  bcur_status_t st;
  if (P->d.a_dtype == BCUR_F64) st = run_error<double>(P, (const double*)A, out);
  else if (is_bf16_prec(P->d.fit_prec)) st = run_error16(P, (const float*)A, out);
  else st = run_error<float>(P, (const float*)A, out);
  BCUR_TRY(st);
  // kept for bcur_rank_k_error's ratio
  BCUR_CUDA_TRY(cudaMemcpyAsync(P->at<double>(P->o.result), out, 3 * sizeof(double),
                                cudaMemcpyDeviceToDevice, P->stream));
  P->have_error = true;
  return BCUR_OK;
}

bcur_status_t bcur_rank_k_error(bcur_plan_t P, const void* A, double* out) {
  if (!plan_ok(P)) return BCUR_EINVAL;
  if (!P->ws || !P->have_scores || !P->have_error) return BCUR_ESTATE;
  if (!A || !out) return BCUR_EINVAL;
  return P->d.a_dtype == BCUR_F64 ? run_rank_k<double>(P, (const double*)A, out)
                                  : run_rank_k<float>(P, (const float*)A, out);
}

// --- Plan-free factorisation pieces (used by the row-sharded form) --------
bcur_status_t bcur_cholesky_inverse(void* G, int64_t w, int32_t dtype, void* L, void* Linv,
                                    int32_t* kept, double tol_rel, void* workspace,
                                    size_t workspace_bytes, void* stream) {
  if (!G || !L || !Linv || !kept || !workspace) return BCUR_EINVAL;
  if (w < 64 || w % 64 != 0 || w > 65536) return BCUR_EINVAL;
  if (dtype != BCUR_F64 && dtype != BCUR_F32) return BCUR_EINVAL;
  if (workspace_bytes < 256 || ((uintptr_t)workspace & 255)) return BCUR_EINVAL;
  // A minimal plan: the stream, the leaf size and two slots of the caller's
  // scratch (the largest diagonal entry, a status word).
  bcur_plan_s P;
  P.stream = (cudaStream_t)stream;
  P.nb = 64;
  P.ws = (char*)workspace;
  P.ws_bytes = workspace_bytes;
  P.o.maxdiag = 0;
  P.o.status = 128;
  P.o.tc_scratch = 0;
  P.tc_scratch_bytes = 0;
  if (dtype == BCUR_F64) {
    const double tol = tol_rel > 0.0 ? tol_rel : 64.0 * EpsOf<double>::v;
    return chol_inv_blocked<double>(&P, (double*)G, (double*)L, (double*)Linv, w, BCUR_F64,
                                    (int*)kept, tol);
  }
  const double tol = tol_rel > 0.0 ? tol_rel : 64.0 * EpsOf<float>::v;
  return chol_inv_blocked<float>(&P, (float*)G, (float*)L, (float*)Linv, w, BCUR_F32, (int*)kept,
                                 tol);
}

bcur_status_t bcur_svd_small(const double* X, int32_t w, int32_t dtype, void* Ut, void* W,
                             double* sigma, void* work, size_t work_bytes, int32_t* status,
                             void* stream) {
  if (!X || !Ut || !W || !sigma || !work || w < 1 || w > 128) return BCUR_EINVAL;
  if (dtype != BCUR_F64 && dtype != BCUR_F32) return BCUR_EINVAL;
  const size_t esz = dtype == BCUR_F64 ? 8 : 4;
  if (work_bytes < (size_t)(w + 1) * (w + 1) * esz) return BCUR_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == BCUR_F64)
    return jacobi_svd_small<double>(X, w, (double*)Ut, (double*)W, sigma, (double*)work,
                                    (int*)status, s);
  return jacobi_svd_small<float>(X, w, (float*)Ut, (float*)W, sigma, (float*)work, (int*)status, s);
}

bcur_status_t bcur_gather_blocks(const void* A, int64_t lda, int64_t m, int64_t n, int32_t dtype,
                                 int32_t axis, const int64_t* off, int32_t G, const int32_t* idx,
                                 int32_t g, int64_t cap, void* out, int64_t ldo, void* map,
                                 void* stream) {
  if (!A || !off || !idx || !out || !map || m < 1 || n < 1 || lda < n || G < 1 || g < 0)
    return BCUR_EINVAL;
  if (dtype != BCUR_F64 && dtype != BCUR_F32) return BCUR_EINVAL;
  if (axis != 0 && axis != 1) return BCUR_EINVAL;
  if (cap < 1 || ldo < (axis == 1 ? m : n)) return BCUR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t* mp = static_cast<int64_t*>(map);
  int64_t* count = mp + cap;
  BCUR_TRY(expand_blocks(idx, g, off, G, cap, mp, count, s));
  if (axis == 1) {  // columns: out = C^T (cap x m, ld ldo)
    return dtype == BCUR_F64
               ? gather_cols_t<double>((const double*)A, lda, m, mp, cap, (double*)out, ldo, s)
               : gather_cols_t<float>((const float*)A, lda, m, mp, cap, (float*)out, ldo, s);
  }
  return dtype == BCUR_F64
             ? gather_rows<double>((const double*)A, lda, n, mp, cap, (double*)out, ldo, s)
             : gather_rows<float>((const float*)A, lda, n, mp, cap, (float*)out, ldo, s);
}

bcur_status_t bcur_boost_select(int32_t t, const double* err, int64_t err_stride, const void* U,
                                int64_t U_bytes, const int32_t* col_idx, int32_t g_col,
                                const int32_t* row_idx, int32_t g_row, void* U_best,
                                int32_t* col_idx_best, int32_t* row_idx_best, double* err_best,
                                int32_t* best, void* stream) {
  return boost_select(t, err, err_stride, U, U_bytes, col_idx, g_col, row_idx, g_row, U_best,
                      col_idx_best, row_idx_best, err_best, best, (cudaStream_t)stream);
}

bcur_status_t bcur_truncate(bcur_plan_t P, const void* A, int32_t kt, const void* omega,
                            void* Uk, double* out) {
  if (!plan_ok(P)) return BCUR_EINVAL;
  if (!P->ws || !P->have_fit) return BCUR_ESTATE;
  if (!A || !omega || !out || kt < 1 || kt > P->k) return BCUR_EINVAL;
  if (P->c_pad > P->ldm || P->r_pad > P->ldn || P->l > std::min(P->c_max, P->r_max))
    return BCUR_ENOTSUP;
  if (P->d.a_dtype == BCUR_F64)
    return run_truncate<double>(P, (const double*)A, kt, (const double*)omega, (double*)Uk, out);
  return run_truncate<float>(P, (const float*)A, kt, (const float*)omega, (float*)Uk, out);
}

// --- Whole decomposition from host buffers --------------------------------
// Staging layout (device, caller-owned): A, Omega panel, the two uniform
// vectors, scores, indices, U and the error triple, each slice 256-byte
// aligned.
struct HostStage {
  size_t A, om, uc, ur, cs, rs, ci, ri, U, err, total;
};
static HostStage host_stage_layout(const bcur_plan_s* P) {
  Layout L;
  HostStage h;
  const size_t e = P->esz;
  h.A = L.take((size_t)P->m * P->lda * e);
  h.om = L.take((size_t)P->l * P->n * e);
  h.uc = L.take((size_t)P->d.g_col * 8);
  h.ur = L.take((size_t)P->d.g_row * 8);
  h.cs = L.take((size_t)P->d.G_col * 8);
  h.rs = L.take((size_t)P->d.G_row * 8);
  h.ci = L.take((size_t)P->d.g_col * 4);
  h.ri = L.take((size_t)P->d.g_row * 4);
  h.U = L.take((size_t)P->c_max * P->r_max * e);
  h.err = L.take(3 * 8);
  h.total = L.cur;
  return h;
}

size_t bcur_host_staging_bytes(bcur_plan_t P) { return plan_ok(P) ? host_stage_layout(P).total : 0; }

bcur_status_t bcur_decompose_host(bcur_plan_t P, const void* A, const void* omega,
                                  const double* u_col, const double* u_row, void* staging,
                                  size_t staging_bytes, double* col_scores, double* row_scores,
                                  int32_t* col_idx, int32_t* row_idx, void* U, double* err) {
  if (!plan_ok(P)) return BCUR_EINVAL;
  if (!P->ws) return BCUR_ESTATE;
  if (!A || !omega || !u_col || !u_row || !staging || !err) return BCUR_EINVAL;
  if ((uintptr_t)staging & 255) return BCUR_EINVAL;
  const HostStage h = host_stage_layout(P);
  if (staging_bytes < h.total) return BCUR_ENOMEM;
  char* base = static_cast<char*>(staging);
  cudaStream_t s = P->stream;
  const size_t e = P->esz;
  auto h2d = [&](size_t off, const void* src, size_t bytes) {
    return cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, s);
  };
  auto d2h = [&](void* dst, size_t off, size_t bytes) {
    return cudaMemcpyAsync(dst, base + off, bytes, cudaMemcpyDeviceToHost, s);
  };
  // A, the one large input: read by the SMs over the host link when the
  // page-locked buffer is mapped into the device's address space (measured
  // faster than the copy engines on GB300), otherwise copied.
  // BCUR_H2D=copy forces the copy engines.
  {
    const size_t abytes = (size_t)P->m * P->lda * e;
    void* mapped = nullptr;
    const char* mode = getenv("BCUR_H2D");
    const bool want_sm = !(mode && strcmp(mode, "copy") == 0);
    bool done = false;
    if (want_sm && abytes % 16 == 0 &&
        cudaHostGetDevicePointer(&mapped, const_cast<void*>(A), 0) == cudaSuccess && mapped &&
        ((uintptr_t)mapped & 15) == 0) {
      BCUR_TRY(copy_bytes_sm(mapped, base + h.A, abytes, P->sms, s));
      done = true;
    } else {
      cudaGetLastError();  // a buffer that is not mapped is not an error here
    }
    if (!done) BCUR_CUDA_TRY(h2d(h.A, A, abytes));
  }
  BCUR_CUDA_TRY(h2d(h.om, omega, (size_t)P->l * P->n * e));
  BCUR_CUDA_TRY(h2d(h.uc, u_col, (size_t)P->d.g_col * 8));
  BCUR_CUDA_TRY(h2d(h.ur, u_row, (size_t)P->d.g_row * 8));
  const void* Ad = base + h.A;
  double* cs = reinterpret_cast<double*>(base + h.cs);
  double* rs = reinterpret_cast<double*>(base + h.rs);
  int32_t* ci = reinterpret_cast<int32_t*>(base + h.ci);
  int32_t* ri = reinterpret_cast<int32_t*>(base + h.ri);
  double* ed = reinterpret_cast<double*>(base + h.err);
  BCUR_TRY(bcur_scores(P, Ad, base + h.om, cs, rs));
  BCUR_TRY(bcur_sample(P, cs, rs, reinterpret_cast<const double*>(base + h.uc),
                       reinterpret_cast<const double*>(base + h.ur), ci, ri, nullptr, nullptr));
  BCUR_TRY(bcur_fit(P, Ad, ci, ri, U ? base + h.U : nullptr, nullptr, nullptr));
  BCUR_TRY(bcur_error(P, Ad, ed));
  if (col_scores) BCUR_CUDA_TRY(d2h(col_scores, h.cs, (size_t)P->d.G_col * 8));
  if (row_scores) BCUR_CUDA_TRY(d2h(row_scores, h.rs, (size_t)P->d.G_row * 8));
  if (col_idx) BCUR_CUDA_TRY(d2h(col_idx, h.ci, (size_t)P->d.g_col * 4));
  if (row_idx) BCUR_CUDA_TRY(d2h(row_idx, h.ri, (size_t)P->d.g_row * 4));
  if (U) BCUR_CUDA_TRY(d2h(U, h.U, (size_t)P->c_max * P->r_max * e));
  BCUR_CUDA_TRY(d2h(err, h.err, 3 * 8));
  return BCUR_OK;
}

bcur_status_t bcur_rank(bcur_plan_t P, int64_t* c, int64_t* r, int64_t* rank_c, int64_t* rank_r) {
  if (!plan_ok(P)) return BCUR_EINVAL;
  if (!P->ws || !P->have_fit) return BCUR_ESTATE;
  int64_t counts[2] = {0, 0};
  int kept[8] = {0};
  BCUR_CUDA_TRY(cudaMemcpyAsync(counts, P->at<int64_t>(P->o.counts), sizeof(counts),
                                cudaMemcpyDeviceToHost, P->stream));
  BCUR_CUDA_TRY(cudaMemcpyAsync(kept, P->at<int>(P->o.kept), sizeof(kept),
                                cudaMemcpyDeviceToHost, P->stream));
  BCUR_CUDA_TRY(cudaStreamSynchronize(P->stream));
  if (c) *c = counts[0];
  if (r) *r = counts[1];
  if (rank_c) *rank_c = kept[4];
  if (rank_r) *rank_r = kept[6];
  return BCUR_OK;
}

bcur_status_t bcur_sync_status(bcur_plan_t P) {
  if (!plan_ok(P)) return BCUR_EINVAL;
  BCUR_CUDA_TRY(cudaStreamSynchronize(P->stream));
  if (!P->ws) return BCUR_OK;
  int st = 0;
  BCUR_CUDA_TRY(cudaMemcpyAsync(&st, P->at<int>(P->o.status), sizeof(int), cudaMemcpyDeviceToHost,
                                P->stream));
  BCUR_CUDA_TRY(cudaStreamSynchronize(P->stream));
  if (st) {
    BCUR_CUDA_TRY(cudaMemsetAsync(P->at<int>(P->o.status), 0, sizeof(int), P->stream));
    BCUR_CUDA_TRY(cudaStreamSynchronize(P->stream));
  }
  return (bcur_status_t)st;
}

void bcur_destroy(bcur_plan_t P) {
  if (!plan_ok(P)) return;
  if (P->stream2) {
    cudaStreamSynchronize(P->stream2);
    cudaStreamDestroy(P->stream2);
  }
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  if (P->ev_stagger) cudaEventDestroy(P->ev_stagger);
  P->tag = 0;
  delete P;
}

bcur_status_t bcur_block_scores(const void* Ft, int32_t dtype, int32_t k, int64_t h, int64_t ldf,
                                const int64_t* off, int32_t G, double* scores, void* stream) {
  if (!Ft || !off || !scores || k < 1 || h < 1 || ldf < h || G < 1) return BCUR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == BCUR_F64)
    return block_scores<double>((const double*)Ft, k, h, ldf, off, G, scores, nullptr, s);
  if (dtype == BCUR_F32)
    return block_scores<float>((const float*)Ft, k, h, ldf, off, G, scores, nullptr, s);
  return BCUR_EINVAL;
}

size_t bcur_block_stable_rank_workspace(int32_t k, int32_t G) {
  return block_stable_rank_workspace(k, G);
}

bcur_status_t bcur_block_stable_rank(const void* Ft, int32_t dtype, int32_t k, int64_t h,
                                     int64_t ldf, const int64_t* off, int32_t G, double* ratio,
                                     void* workspace, size_t workspace_bytes, void* stream) {
  if (!Ft || !off || !ratio || k < 1 || k > 128 || h < 1 || ldf < h || G < 1) return BCUR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == BCUR_F64)
    return block_stable_rank<double>((const double*)Ft, k, ldf, off, G, ratio, workspace,
                                     workspace_bytes, s);
  if (dtype == BCUR_F32)
    return block_stable_rank<float>((const float*)Ft, k, ldf, off, G, ratio, workspace,
                                    workspace_bytes, s);
  return BCUR_EINVAL;
}

bcur_status_t bcur_incoherence(const void* Ut, int32_t dtype, int32_t k, int64_t m, int64_t ld,
                               double* out, void* scratch, void* stream) {
  if (!Ut || !out || !scratch) return BCUR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == BCUR_F64) return incoherence<double>((const double*)Ut, k, m, ld, out, scratch, s);
  if (dtype == BCUR_F32) return incoherence<float>((const float*)Ut, k, m, ld, out, scratch, s);
  return BCUR_EINVAL;
}

bcur_status_t bcur_sample_blocks(const double* scores, int32_t G, const double* u, int32_t g,
                                 int32_t replacement, int32_t* idx, double* prob, void* stream) {
  if (!scores || !u || !idx) return BCUR_EINVAL;
  return sample_blocks(scores, G, u, g, replacement, idx, prob, (cudaStream_t)stream);
}

size_t bcur_residual_workspace(int64_t m, int64_t n, int32_t dtype) {
  (void)dtype;
  const int64_t np = std::max(gemm_simt_resid_ctas<double>(m, n),
                              std::max(gemm_simt_resid_ctas<float>(m, n), gemm_tc_resid_ctas(m, n)));
  return (size_t)(2 * np * 8);
}

bcur_status_t bcur_residual(const void* X, int64_t ldx, const void* Pm, int64_t ldp, const void* Q,
                            int64_t ldq, int64_t m, int64_t n, int64_t r, int32_t dtype,
                            int32_t prec, double* out, void* workspace, size_t ws_bytes,
                            void* stream) {
  if (!X || !out || !workspace || m < 1 || n < 1 || r < 0) return BCUR_EINVAL;
  if (r > 0 && (!Pm || !Q)) return BCUR_EINVAL;
  if (ldx < n || ldp < r || ldq < n) return BCUR_EINVAL;
  if (ws_bytes < bcur_residual_workspace(m, n, dtype)) return BCUR_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  GemmDesc g = mk(m, n, r, Pm, ldp, 0, Q, ldq, 0, nullptr, 0);
  g.X = X;
  g.ldx = ldx;
  g.partials = (double*)workspace;
  int64_t np = 0;
  if (dtype == BCUR_BF16) {  // X FP32, P and Q BF16: tensor cores only
    if (prec != BCUR_BF16) return BCUR_EINVAL;
    g.ab_bf16 = 1;
    BCUR_TRY(gemm_tc_resid(g, prec, s, &np));
  } else if (dtype == BCUR_F64) {
    if (prec != BCUR_F64) return BCUR_EINVAL;
    BCUR_TRY(gemm_resid<double>(g, prec, s, &np));
  } else if (dtype == BCUR_F32) {
    if (prec == BCUR_F64) return BCUR_EINVAL;
    BCUR_TRY(gemm_resid<float>(g, prec, s, &np));
  } else {
    return BCUR_EINVAL;
  }
  return finish_residual((const double*)workspace, np, out, 1, s);
}

bcur_status_t bcur_gemm_fp8_blocks(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                                   const void* B, int64_t ldb, const float* scale_m,
                                   const float* bscale, int64_t bs_n, int64_t bs_k, float* D,
                                   int64_t ldd, void* stream) {
  if (!A || !B || !bscale || !D || M < 0 || N < 0 || K < 0) return BCUR_EINVAL;
  if (M == 0 || N == 0) return BCUR_OK;
  if (K == 0 || !(M < 128 && N >= 2 * M)) return BCUR_ENOTSUP;
  GemmDesc g = mk(M, N, K, A, lda, 0, B, ldb, 1, D, ldd);
  g.ab_fp8 = 1;
  g.scale_m = scale_m;
  g.bscale_b = bscale;
  g.bs_n = bs_n;
  g.bs_k = bs_k;
  return gemm_tc(g, BCUR_FP8, (cudaStream_t)stream);
}

bcur_status_t bcur_gemm(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                        int32_t transA, const void* B, int64_t ldb, int32_t transB, void* D,
                        int64_t ldd, int32_t dtype, int32_t prec, void* stream) {
  if (!A || !B || !D || M < 0 || N < 0 || K < 0) return BCUR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  GemmDesc g = mk(M, N, K, A, lda, transA != 0, B, ldb, transB != 0, D, ldd);
  if (dtype == BCUR_F64) {
    if (prec != BCUR_F64) return BCUR_EINVAL;
    return gemm_simt<double>(g, s);
  }
  if (dtype == BCUR_BF16) {  // BF16 A and B, FP32 D: tensor cores only
    if (prec != BCUR_BF16) return BCUR_EINVAL;
    g.ab_bf16 = 1;
    return gemm_tc(g, prec, s);
  }
  if (dtype == BCUR_FP8) {  // e4m3 A and B (K-major), FP32 D: tensor cores only
    if (prec != BCUR_FP8) return BCUR_EINVAL;
    g.ab_fp8 = 1;
    return gemm_tc(g, prec, s);
  }
  if (dtype != BCUR_F32 || prec == BCUR_F64 || prec == BCUR_BF16) return BCUR_EINVAL;
  if (is_tc_prec(prec)) return gemm_tc(g, prec, s);  // no silent fallback here
  return gemm_simt<float>(g, s);
}

}  // extern "C"
