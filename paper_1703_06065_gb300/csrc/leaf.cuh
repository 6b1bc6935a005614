// Device-side building blocks shared by the single-problem kernels and the
// batched (grouped) kernels: the same arithmetic in the same order, so that
// a decomposition gives the same numbers whichever launch it runs in.
#pragma once

#include "common.cuh"

namespace bcur {

// ---------------------------------------------------------------------------
// Precision of the fused residual.  With P = Q_C^T M and Q_R rounded to BF16
// (unit round-off u = 2^-8) the reconstruction error dCUR adds about
// (2/3) u^2 ||CUR||_F^2 to ||A - CUR||_F^2 (the cross term with A - CUR is
// orthogonal to it up to rounding), so the relative error e moves by about
// u^2 (1 - e^2) / (3 e).  A one-term residual is kept while the bound
// u^2 / (2 e) stays below 2.5e-4 (a quarter of the 1e-3 accuracy target);
// otherwise the residual is recomputed with BF16 pairs (three terms, about
// 2^-16 relative).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool residual_needs_refine(double rel_err) {
  const double u = 0.00390625;  // 2^-8
  return !(rel_err > 0.0) || (u * u / (2.0 * rel_err) > 2.5e-4);
}

// ---------------------------------------------------------------------------
// Small FP64 Cholesky with the drop rule, and its inverse (w <= 128).
// S: shared memory of w * (w + 1) doubles.  G (w x w, ld ld >= w): only the
// lower part is read.  A pivot d with d <= tol_rel * max_i G_ii (or d <= 0)
// drops its direction: the column of L and the row of L^{-1} are zero.
// Writes L64 and Linv64 (FP64) and LinvT (T), all ld x ld with zeros above
// the diagonal and outside the leading w x w block (a zero-padded G gives the
// same result as factoring it whole: the padding pivots are dropped);
// *kept = number of kept pivots.  Every thread of the block must call it.
// Right-looking, two barriers per column (scale the column by 1/L_jj; update
// the trailing lower part on a 16 x (threads / 16) grid).  Each pivot's
// square root and reciprocal are taken once, by the thread that finishes the
// diagonal entry (FP64 sqrt and divide are long sequences on this GPU's FP64
// pipe), and published by the barrier that ends the column.  L^{-1} by
// forward substitution, one column per thread, multiplying by the stored
// reciprocals, kept in the strictly upper part of S (X[r][c] at S[c][r + 1],
// which the factorisation never touches).
// ---------------------------------------------------------------------------
template <typename T>
__device__ void chol_small_body(const double* G, int w, int ldio, double tol_rel, double* L64,
                                double* Linv64, T* LinvT, int* kept, double* S) {
  const int ld = w + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ty = tid >> 4, tx = tid & 15, nty = nt >> 4;
  for (int e = tid; e < w * w; e += nt) {
    const int i = e / w, j = e % w;
    S[i * ld + j] = (j <= i) ? G[i * ldio + j] : 0.0;
  }
  __shared__ double s_tol;
  __shared__ int s_kept;
  __shared__ double s_p[128], s_inv[128];  // L_jj and 1 / L_jj (0 when dropped)
  auto pivot = [&](int j, double tol) {
    const double d = S[j * ld + j];
    const bool keep = d > tol && d > 0.0;
    const double p = keep ? sqrt(d) : 0.0;
    s_p[j] = p;
    s_inv[j] = keep ? 1.0 / p : 0.0;
  };
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < w; ++i) mx = fmax(mx, S[i * ld + i]);
    s_tol = tol_rel * mx;
    s_kept = 0;
    pivot(0, tol_rel * mx);
  }
  __syncthreads();
  for (int j = 0; j < w; ++j) {
    const double inv = s_inv[j];
    for (int i = j + 1 + tid; i < w; i += nt) S[i * ld + j] *= inv;
    __syncthreads();
    if (tid == 0) {
      S[j * ld + j] = s_p[j];
      if (s_p[j] > 0.0) s_kept++;
    }
    for (int a = j + 1 + ty; a < w; a += nty) {
      const double la = S[a * ld + j];
      for (int b = j + 1 + tx; b <= a; b += 16) {
        S[a * ld + b] = fma(-la, S[b * ld + j], S[a * ld + b]);
        if (a == j + 1 && b == j + 1) pivot(j + 1, s_tol);  // the next diagonal entry is final
      }
    }
    __syncthreads();
  }
  for (int c = tid; c < w; c += nt) {
    double* xc = S + c * ld + 1;  // xc[k] = X[k][c], k >= c
    for (int r = c; r < w; ++r) {
      const double* lr = S + r * ld;
      double a0 = (r == c) ? 1.0 : 0.0, a1 = 0.0;
      int k = c;
      for (; k + 1 < r; k += 2) {
        a0 = fma(-lr[k], xc[k], a0);
        a1 = fma(-lr[k + 1], xc[k + 1], a1);
      }
      if (k < r) a0 = fma(-lr[k], xc[k], a0);
      xc[r] = (a0 + a1) * s_inv[r];
    }
  }
  __syncthreads();
  for (int e = tid; e < ldio * ldio; e += nt) {
    const int i = e / ldio, j = e % ldio;
    const bool in = i < w && j <= i;
    L64[e] = in ? S[i * ld + j] : 0.0;
    const double x = in ? S[j * ld + i + 1] : 0.0;
    Linv64[e] = x;
    LinvT[e] = (T)x;
  }
  if (tid == 0 && kept) *kept = s_kept;
}

// ---------------------------------------------------------------------------
// Factor one NB x NB diagonal block of a Gram matrix (lower part of G, ld
// ldg, already updated by the trailing updates) as L L^T with the drop rule
// (pivot <= tol -> direction dropped) and form L^{-1}.  Results stay in
// shared memory: S (NB x LD) holds L, X (NB x LD) holds L^{-1}, LD = NB +
// 256 / NB, zeros above the diagonal.  Left-looking and column-parallel: for
// column j every row i >= j forms its dot product with row j of the finished
// columns (split over 256/NB consecutive threads and combined with shuffles),
// then the pivot owner scales the column; the inverse is built row by row the
// same way.  Threads 0..255 work; further threads only take part in the
// barriers.  Returns the number of kept pivots (valid in every thread).
// ---------------------------------------------------------------------------
template <typename T, int NB>
__device__ int potrf_leaf(const T* G, int64_t ldg, T* S, T* X, T tol) {
  constexpr int TPR = 256 / NB;  // threads per row (2 or 4), consecutive lanes
  constexpr int LD = NB + TPR;   // LD = TPR (mod 32): the row-split loads are conflict-free
  constexpr unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x;
  const bool act = tid < 256;
  const int i = tid / TPR, h = tid % TPR;
  if (act) {
    for (int c = h; c < NB; c += TPR) {
      S[i * LD + c] = (c <= i) ? G[(int64_t)i * ldg + c] : T(0);
      X[i * LD + c] = T(0);
    }
  }
  __shared__ T s_inv;
  __shared__ int s_kept;
  if (tid == 0) s_kept = 0;
  __syncthreads();
  for (int j = 0; j < NB; ++j) {
    T v = T(0);
    if (act) {
      // four independent partial sums keep the shared-memory loads in flight
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      int k = h;
      for (; k + 3 * TPR < j; k += 4 * TPR) {
        a0 += S[i * LD + k] * S[j * LD + k];
        a1 += S[i * LD + k + TPR] * S[j * LD + k + TPR];
        a2 += S[i * LD + k + 2 * TPR] * S[j * LD + k + 2 * TPR];
        a3 += S[i * LD + k + 3 * TPR] * S[j * LD + k + 3 * TPR];
      }
      for (; k < j; k += TPR) a0 += S[i * LD + k] * S[j * LD + k];
      T acc = (a0 + a1) + (a2 + a3);
#pragma unroll
      for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
      v = S[i * LD + j] - acc;
      if (i == j && h == 0) {
        const T p = (v > tol && v > T(0)) ? sqrt(v) : T(0);
        S[j * LD + j] = p;
        s_inv = (p > T(0)) ? T(1) / p : T(0);
        if (p > T(0)) s_kept++;
      }
    }
    __syncthreads();
    if (act && i > j && h == 0) S[i * LD + j] = v * s_inv;
    __syncthreads();
  }
  // X = L^{-1}, row r from the rows above it:
  //   X[r][c] = (delta_rc - sum_{c <= k < r} L[r][k] X[k][c]) / L[r][r]
  for (int r = 0; r < NB; ++r) {
    if (act) {
      const int c = i;  // column handled by this thread group
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      if (c <= r) {
        int k = c + h;
        for (; k + 3 * TPR < r; k += 4 * TPR) {
          a0 += S[r * LD + k] * X[k * LD + c];
          a1 += S[r * LD + k + TPR] * X[(k + TPR) * LD + c];
          a2 += S[r * LD + k + 2 * TPR] * X[(k + 2 * TPR) * LD + c];
          a3 += S[r * LD + k + 3 * TPR] * X[(k + 3 * TPR) * LD + c];
        }
        for (; k < r; k += TPR) a0 += S[r * LD + k] * X[k * LD + c];
      }
      T acc = (a0 + a1) + (a2 + a3);
#pragma unroll
      for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
      if (c <= r && h == 0) {
        const T lrr = S[r * LD + r];
        X[r * LD + c] = (lrr > T(0)) ? (((c == r) ? T(1) : T(0)) - acc) / lrr : T(0);
      }
    }
    __syncthreads();
  }
  return s_kept;
}

// ---------------------------------------------------------------------------
// One warp: Cholesky with the drop rule of a 32 x 32 FP32 block held in
// shared memory (lower part of A, ld lda; factored in place, zeros written
// above the diagonal).  Lane i owns row i in registers as a window that
// slides one column per step: at step j, a[t] holds entry (i, j + t), so the
// register indices stay compile-time constants while the step loop stays
// rolled (unrolling the steps would make it bound on instruction fetch).
// Step j: pivot d from lane j by shuffle; drop rule d <= tol or d <= 0;
// r = 1/sqrt(d) (rsqrtf), L_jj = d r, l_ij = a_ij r.  Column j is also
// written to cb row j, shifted (cb[j][t] = L[j + t][j], zero past the
// block), so that the update a[t] -= l_i l_{j+t} reads it with eight
// broadcast float4 loads, and r to cb's reciprocal row.  Entries above the
// diagonal are updated too (their lanes carry l = 0 from then on, so they
// never feed back; A gets zeros there).  A dropped pivot zeroes its column.
// cb: 32 x 36 + 32 floats of shared scratch.  Returns the number of kept
// pivots (same in every lane).
// ---------------------------------------------------------------------------
__device__ inline int warp_chol32_fact(float* A, int lda, float tol, float* cb) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int CL = 36;
  float* rp = cb + 32 * CL;  // 1 / L_jj (0 when dropped)
  const int lane = threadIdx.x & 31;
  float a[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) a[t] = (t <= lane) ? A[lane * lda + t] : 0.f;
  __syncwarp();
  int kept = 0;
#pragma unroll 1
  for (int j = 0; j < 32; ++j) {
    const float d = __shfl_sync(FULL, a[0], j);
    const bool keep = d > tol && d > 0.f;
    const float r = keep ? rsqrtf(d) : 0.f;
    kept += keep ? 1 : 0;
    const float l = (lane > j) ? a[0] * r : ((lane == j) ? d * r : 0.f);
    A[lane * lda + j] = l;
    cb[j * CL + ((lane - j) & 31)] = (lane >= j) ? l : 0.f;
    if (lane == 0) rp[j] = r;
    __syncwarp();
    float wv[32];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(&cb[j * CL + 4 * q]);
      wv[4 * q] = v.x;
      wv[4 * q + 1] = v.y;
      wv[4 * q + 2] = v.z;
      wv[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int t = 1; t < 32; ++t) a[t] = fmaf(-l, wv[t], a[t]);
#pragma unroll
    for (int t = 0; t < 31; ++t) a[t] = a[t + 1];
    a[31] = 0.f;
  }
  __syncwarp();
  return kept;
}

// One warp: forward substitution with the factor left in cb by
// warp_chol32_fact.  Lane c solves L y = b (b: its 32 right-hand-side values
// in registers) with the same sliding window: y_k = b_k r_k, then
// b_{k+t} -= L[k+t][k] y_k from cb row k; y_k goes to out[k * so + c * sl].
// With b = e_c this is column c of L^{-1} (a dropped pivot gives a zero row).
__device__ inline void warp_fwd32(const float* cb, float (&b)[32], float* out, int so, int sl) {
  constexpr int CL = 36;
  const float* rp = cb + 32 * CL;
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int k = 0; k < 32; ++k) {
    const float xk = b[0] * rp[k];
    out[k * so + lane * sl] = xk;
    float wv[32];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(&cb[k * CL + 4 * q]);
      wv[4 * q] = v.x;
      wv[4 * q + 1] = v.y;
      wv[4 * q + 2] = v.z;
      wv[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int t = 1; t < 32; ++t) b[t] = fmaf(-wv[t], xk, b[t]);
#pragma unroll
    for (int t = 0; t < 31; ++t) b[t] = b[t + 1];
    b[31] = 0.f;
  }
  __syncwarp();
}

// The 64 x 64 leaf in FP32 from two warp-level 32 x 32 factorisations:
//   L11 = chol(G11);  X11 = L11^{-1} and L21 = G21 L11^{-T} by forward
//   substitution, side by side in warps 0 and 1;  L22 = chol(G22 - L21 L21^T)
//   in warp 0 while the other warps form T = L21 X11;  X22 = L22^{-1};
//   X21 = -X22 T.
// leaf64_core starts from the block already in shared memory (S: lower part,
// zeros above the diagonal, LD = 68; X: zeros) after a block barrier; it
// leaves S = L and X = L^{-1} (threads 0..255 work, all must call it).  A
// dropped pivot of L11 zeroes its column of L21, so the update of G22 is
// unaffected by it, as in the unblocked order.
__device__ inline int leaf64_core(float* S, float* X, float tol) {
  constexpr int LD = 68, H = 32;
  const int tid = threadIdx.x;
  const bool act = tid < 256;
  const int warp = tid >> 5, lane = tid & 31;
  __shared__ int s_kept;
  __shared__ __align__(16) float s_cb[32 * 36 + 32];
  int k1 = 0;
  if (warp == 0) k1 = warp_chol32_fact(S, LD, tol, s_cb);
  __syncthreads();
  if (warp == 0) {  // X11 = L11^{-1}, column `lane`
    float b[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) b[t] = (t == lane) ? 1.f : 0.f;
    warp_fwd32(s_cb, b, X, LD, 1);
  } else if (warp == 1) {  // row `lane` of L21 = G21 L11^{-T}, in place
    float b[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) b[t] = S[(H + lane) * LD + t];
    __syncwarp();
    warp_fwd32(s_cb, b, S + H * LD, 1, LD);
  }
  __syncthreads();
  const int i = (tid >> 3) & 31, c4 = (tid & 7) * 4;
  // G22 -= L21 L21^T (lower part)
  if (act) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = c4 + q;
      if (j > i) continue;
      float s2 = 0.f;
      for (int t = 0; t < H; ++t) s2 = fmaf(S[(H + i) * LD + t], S[(H + j) * LD + t], s2);
      S[(H + i) * LD + H + j] -= s2;
    }
  }
  __syncthreads();
  int k2 = 0;
  if (warp == 0) {
    k2 = warp_chol32_fact(S + H * LD + H, LD, tol, s_cb);
    float b[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) b[t] = (t == lane) ? 1.f : 0.f;
    warp_fwd32(s_cb, b, X + H * LD + H, LD, 1);
  } else if (act) {
    // T = L21 X11 (X11 lower: t >= c), in X21's place; warp 0 touches only
    // the (2, 2) blocks meanwhile
    for (int e = tid - 32; e < H * H; e += 224) {
      const int r = e >> 5, c = e & 31;
      float t2 = 0.f;
      for (int t = c; t < H; ++t) t2 = fmaf(S[(H + r) * LD + t], X[t * LD + c], t2);
      X[(H + r) * LD + c] = t2;
    }
  }
  if (tid == 0) s_kept = k1 + k2;
  __syncthreads();
  // X21 = -X22 T (X22 lower: t <= i)
  float acc[4];
  if (act) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c4 + q;
      float t2 = 0.f;
      for (int t = 0; t <= i; ++t) t2 = fmaf(X[(H + i) * LD + H + t], X[(H + t) * LD + c], t2);
      acc[q] = -t2;
    }
  }
  __syncthreads();
  if (act)
#pragma unroll
    for (int q = 0; q < 4; ++q) X[(H + i) * LD + c4 + q] = acc[q];
  __syncthreads();
  return s_kept;
}

// Same contract as the generic potrf_leaf (S = L, X = L^{-1}, LD = 68).  The
// block is loaded with all of a thread's reads in flight at once.
template <>
__device__ inline int potrf_leaf<float, 64>(const float* G, int64_t ldg, float* S, float* X,
                                            float tol) {
  constexpr int NB = 64, LD = 68;
  const int tid = threadIdx.x;
  if (tid < 256) {
    float g[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = tid + 256 * q, i = e / NB, c = e % NB;
      g[q] = (c <= i) ? G[(int64_t)i * ldg + c] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = tid + 256 * q, i = e / NB, c = e % NB;
      S[i * LD + c] = g[q];
      X[i * LD + c] = 0.f;
    }
  }
  __syncthreads();
  return leaf64_core(S, X, tol);
}

// ---------------------------------------------------------------------------
// Inverse-CDF block sampling, one thread.  The arithmetic is the sequential
// FP64 order of the oracle: every add / multiply is an explicit
// round-to-nearest intrinsic (no contraction into FMA).  For draw t with
// uniform u[t]: T = sum of the remaining scores, x = u[t] * T, pick the first
// remaining j whose running prefix sum exceeds x; if rounding leaves none,
// the last remaining block with a positive score, else the first remaining
// block.  remaining: G bytes of scratch.  prob may be null.
// ---------------------------------------------------------------------------
__device__ inline void sample_seq(const double* scores, int G, const double* u, int g,
                                  int replacement, int32_t* idx, double* prob,
                                  unsigned char* remaining) {
  for (int j = 0; j < G; ++j) remaining[j] = 1;
  double total0 = 0.0;
  for (int j = 0; j < G; ++j) total0 = __dadd_rn(total0, scores[j]);
  for (int t = 0; t < g; ++t) {
    double T = 0.0;
    for (int j = 0; j < G; ++j)
      if (remaining[j]) T = __dadd_rn(T, scores[j]);
    const double x = __dmul_rn(u[t], T);
    int pick = -1;
    double S = 0.0;
    for (int j = 0; j < G; ++j) {
      if (!remaining[j]) continue;
      S = __dadd_rn(S, scores[j]);
      if (S > x) { pick = j; break; }
    }
    if (pick < 0) {
      for (int j = G - 1; j >= 0; --j)
        if (remaining[j] && scores[j] > 0.0) { pick = j; break; }
      if (pick < 0)
        for (int j = 0; j < G; ++j)
          if (remaining[j]) { pick = j; break; }
    }
    idx[t] = pick;
    if (prob) prob[t] = total0 > 0.0 ? __ddiv_rn(scores[pick], total0) : 0.0;
    if (!replacement) remaining[pick] = 0;
  }
}

}  // namespace bcur
