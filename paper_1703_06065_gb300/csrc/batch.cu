// Grouped small kernels of the batched Block CUR path (sm_103a).  Each
// launch covers every decomposition of the batch: a CTA finds its
// decomposition through a prefix-sum work list (or blockIdx.x when the work
// is one CTA per decomposition) and reads the decomposition's sizes and
// buffers from the device table of Items.  Every per-decomposition sum is
// formed by the same CTA in the same order whatever else is in the batch, so
// a decomposition's results do not depend on its neighbours.
#include "batch.h"
#include "leaf.cuh"

namespace bcur {
namespace batch {

namespace {

__device__ __forceinline__ float* panel(const Item& I, int sel) {
  switch (sel) {
    case PM0: return I.Pm0;
    case PM1: return I.Pm1;
    case PN0: return I.Pn0;
    default: return I.Pn1;
  }
}
__device__ __forceinline__ int64_t panel_h(const Item& I, int sel) { return sel < PN0 ? I.m : I.n; }
__device__ __forceinline__ int64_t panel_ld(const Item& I, int sel) {
  return sel < PN0 ? I.ldm : I.ldn;
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum: strided per thread (caller), xor tree per warp,
// warps in order.  Result valid in thread 0.
__device__ double block_sum(double v, double* red) {
  v = wsum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// ---------------------------------------------------------------------------
// A -> BF16 hi/lo pair (8 rows per CTA) and Omega^T -> BF16 panel (zero rows
// past l), one launch.  mode 0: hi and lo; mode 1: hi only (the adaptive fit
// needs lo only for the items it refines); mode 2: lo only, for the items
// whose refinement flag is set (the Omega part is not launched).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) split_kernel(const Item* items, const bcur_batch_io_t* io,
                                                    Work rows8, int total8, int lp, int mode) {
  const int x = blockIdx.x;
  if (x < total8) {
    const int b = find_item(rows8, x);
    const Item& I = items[b];
    if (mode == 2 && *I.refine == 0) return;  // uniform over the CTA
    const bool wh = mode != 2, wl = mode != 1;
    const int64_t r0 = (int64_t)(x - rows8.prefix[b]) * 8;
    const float* A = io[b].A;
    const bool v4 = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (I.lda % 4 == 0) &&
                    (I.n % 4 == 0);
    for (int rr = 0; rr < 8; ++rr) {
      const int64_t r = r0 + rr;
      if (r >= I.m) break;
      const float* xr = A + r * I.lda;
      bf16* hr = I.Ah + r * I.ldn;
      bf16* lr = I.Al + r * I.ldn;
      if (v4) {
        for (int64_t c = threadIdx.x; c < I.n / 4; c += blockDim.x) {
          const float4 v = reinterpret_cast<const float4*>(xr)[c];
          const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y);
          const __nv_bfloat162 h23 = __floats2bfloat162_rn(v.z, v.w);
          if (wh) {
            reinterpret_cast<__nv_bfloat162*>(hr)[2 * c] = h01;
            reinterpret_cast<__nv_bfloat162*>(hr)[2 * c + 1] = h23;
          }
          if (wl) {
            const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
            reinterpret_cast<__nv_bfloat162*>(lr)[2 * c] =
                __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
            reinterpret_cast<__nv_bfloat162*>(lr)[2 * c + 1] =
                __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
          }
        }
      } else {
        for (int64_t c = threadIdx.x; c < I.n; c += blockDim.x) {
          const float v = xr[c];
          const bf16 h = __float2bfloat16_rn(v);
          if (wh) hr[c] = h;
          if (wl) lr[c] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
      }
    }
  } else {
    const int y = x - total8;
    const int b = y / (lp / 8);
    const Item& I = items[b];
    const int t0 = (y % (lp / 8)) * 8;
    for (int tt = 0; tt < 8; ++tt) {
      const int t = t0 + tt;
      bf16* o = I.Om + (int64_t)t * I.ldn;
      const float* om = io[b].omega + (int64_t)t * I.n;
      for (int64_t j = threadIdx.x; j < I.n; j += blockDim.x)
        o[j] = __float2bfloat16_rn(t < I.l ? om[j] : 0.f);
    }
  }
}

// ---------------------------------------------------------------------------
// Skinny Cholesky-QR of an LP x h panel X (rows l..LP-1 zero):
//   gram:  per chunk of CH columns, the FP32 partial Gram X_c X_c^T;
//   chol:  FP64 sum of the partials in chunk order, Cholesky with the drop
//          rule (64 u of FP32, relative to the largest diagonal entry) and
//          L^{-1};
//   apply: X' = L^{-1} X (FP32), optionally also as BF16 for the next
//          product with A.
// ---------------------------------------------------------------------------
// The Gram is symmetric and only its lower part is read.  Its rows past the
// item's l are zero, so only the lower R x R tiles of the leading
// nb = ceil(l / R) tile rows are formed: T = nb (nb + 1) / 2 tiles.  The 256
// threads are split into G = 256 / T groups of T: thread (g, t) forms tile t
// over the slice columns c = g, g + G, ..., and the groups' partial tiles are
// added in group order at the end (so the sum order depends only on l, never
// on the rest of the batch).  Work and loads scale with l^2, not with the
// panel height LP.  The next 64-column slice is fetched into registers while
// the current one is multiplied.
__device__ __forceinline__ void tri_tile(int t, int& ti, int& tj) {
  ti = 0;
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  tj = t - ti * (ti + 1) / 2;
}

template <int LP>
__global__ void __launch_bounds__(256, LP == 64 ? 2 : 1) sgram_kernel(const Item* items,
                                                                      Work chunks, int sel) {
  constexpr int R = LP / 16;          // R x R outputs per tile
  constexpr int NL = LP * 64 / 256;   // slice elements loaded per thread
  constexpr int TLD = LP + 4;         // XsT[c][r]: column c of the slice, rows r
  constexpr int SMEM = (64 * TLD > 136 * R * R) ? 64 * TLD : 136 * R * R;
  const int b = find_item(chunks, blockIdx.x);
  const Item& I = items[b];
  const int ch = blockIdx.x - chunks.prefix[b];
  const float* X = panel(I, sel);
  const int64_t h = panel_h(I, sel), ld = panel_ld(I, sel);
  const int l = I.l;
  __shared__ __align__(16) float XsT[SMEM];
  const int tid = threadIdx.x;
  const int nb = (l + R - 1) / R;
  const int T = nb * (nb + 1) / 2;
  const int G = 256 / T;
  const int g = tid / T, t = tid - g * T;
  const bool active = g < G;
  int ti = 0, tj = 0;
  if (active) tri_tile(t, ti, tj);
  float acc[R][R];
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[a][c] = 0.f;
  const int64_t c_begin = (int64_t)ch * CH;
  const int64_t c_end = c_begin + CH < h ? c_begin + CH : h;
  float rx[NL];
  auto fetch = [&](int64_t c0) {
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = tid + 256 * q, r = e / 64, c = e % 64;
      rx[q] = (r < l && c0 + c < c_end) ? X[r * ld + c0 + c] : 0.f;
    }
  };
  fetch(c_begin);
  for (int64_t c0 = c_begin; c0 < c_end; c0 += 64) {
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = tid + 256 * q, r = e / 64, c = e % 64;
      XsT[c * TLD + r] = rx[q];
    }
    __syncthreads();
    if (c0 + 64 < c_end) fetch(c0 + 64);
    if (active) {
#pragma unroll 2
      for (int c = g; c < 64; c += G) {
        float a[R], bb[R];
#pragma unroll
        for (int q = 0; q < R; q += 4) {
          const float4 a4 = *reinterpret_cast<const float4*>(&XsT[c * TLD + R * ti + q]);
          const float4 b4 = *reinterpret_cast<const float4*>(&XsT[c * TLD + R * tj + q]);
          a[q] = a4.x; a[q + 1] = a4.y; a[q + 2] = a4.z; a[q + 3] = a4.w;
          bb[q] = b4.x; bb[q + 1] = b4.y; bb[q + 2] = b4.z; bb[q + 3] = b4.w;
        }
#pragma unroll
        for (int q = 0; q < R; ++q)
#pragma unroll
          for (int p = 0; p < R; ++p) acc[q][p] = fmaf(a[q], bb[p], acc[q][p]);
      }
    }
    __syncthreads();
  }
  // groups 1 .. G-1 hand their partial tiles to group 0, in group order
  for (int gg = 1; gg < G; ++gg) {
    if (active && g == gg)
#pragma unroll
      for (int q = 0; q < R; ++q)
#pragma unroll
        for (int p = 0; p < R; ++p) XsT[(t * R + q) * R + p] = acc[q][p];
    __syncthreads();
    if (active && g == 0)
#pragma unroll
      for (int q = 0; q < R; ++q)
#pragma unroll
        for (int p = 0; p < R; ++p) acc[q][p] += XsT[(t * R + q) * R + p];
    __syncthreads();
  }
  if (active && g == 0) {
    float* out = I.gpart + (int64_t)ch * LP * LP;
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
      for (int p = 0; p < R; ++p) out[(R * ti + q) * LP + R * tj + p] = acc[q][p];
  }
}

template <int LP>
__global__ void __launch_bounds__(256) schol_kernel(const Item* items, int sel, int pass,
                                                    int want_lb) {
  extern __shared__ double S[];  // l x (l + 1)
  const Item& I = items[blockIdx.x];
  const int nch = sel < PN0 ? I.chunks_m : I.chunks_n;
  const int l = I.l;  // panel rows l..LP-1 are zero: only the leading l x l block is factored
  for (int e = threadIdx.x; e < LP * LP; e += blockDim.x) {
    const int i = e / LP, j = e % LP;
    double g = 0.0;
    if (i < l && j <= i)
      for (int c = 0; c < nch; ++c) g += (double)I.gpart[(int64_t)c * LP * LP + e];
    I.G64[e] = g;
  }
  __syncthreads();
  double* L = pass ? I.L64b : I.L64a;
  chol_small_body<float>(I.G64, l, LP, 64.0 * 1.1920928955078125e-07, L, I.Linv64, I.LinvT,
                         nullptr, S);
  if (want_lb && pass == 1) {
    __syncthreads();
    // L_B = L_a L_b: X = L_a Q' and Q' = L_b Q give X = L_a L_b Q
    for (int e = threadIdx.x; e < LP * LP; e += blockDim.x) {
      const int i = e / LP, j = e % LP;
      double acc = 0.0;
      if (i < l && j <= i)
        for (int k = j; k <= i; ++k) acc += I.L64a[i * LP + k] * I.L64b[k * LP + j];
      I.Lb[e] = acc;
    }
  }
}

// apply: a CTA takes AP columns in slices of 64; thread (ti, tj) forms rows
// RR ti.. (RR = LP / 16) and columns 4 tj.. of the slice as a small GEMM from
// shared memory (L^{-1} transposed, the slice row-major), summing t = 0..r in
// increasing order and stopping at the last nonzero column of its rows.  The
// next slice is fetched into registers while the current one is multiplied.
template <int LP>
__global__ void __launch_bounds__(256, LP == 64 ? 3 : 2) sapply_kernel(const Item* items, Work chunks, int src,
                                                     int dst, int write_bf16) {
  constexpr int RR = LP / 16;         // rows per thread
  constexpr int LLD = LP + 4;         // LsT[t][r] = L^{-1}[r][t]
  constexpr int XLD = 64 + 4;         // Xs[t][c]
  constexpr int NL = LP * 64 / 256;   // slice elements loaded per thread
  const int b = find_item(chunks, blockIdx.x);
  const Item& I = items[b];
  const int ch = blockIdx.x - chunks.prefix[b];
  extern __shared__ __align__(16) float apply_smem[];
  float* LsT = apply_smem;            // LP x LLD
  float* Xs = LsT + LP * LLD;         // LP x XLD
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  for (int e = tid; e < LP * LP; e += 256) {
    const int r = e / LP, t = e % LP;
    LsT[t * LLD + r] = I.LinvT[e];
  }
  const int64_t h = panel_h(I, src), ld = panel_ld(I, src);
  const int l = I.l;
  const float* X = panel(I, src);
  float* Y = panel(I, dst);
  bf16* Yb = write_bf16 ? (src < PN0 ? I.Qh : I.Zh) : nullptr;
  const int64_t c_begin = (int64_t)ch * AP;
  const int64_t c_end = c_begin + AP < h ? c_begin + AP : h;
  const bool vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(Y) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(Yb) & 7) == 0);
  float rx[NL];
  auto fetch = [&](int64_t c0) {
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = tid + 256 * q, r = e / 64, c = e % 64;
      rx[q] = (r < l && c0 + c < c_end) ? X[r * ld + c0 + c] : 0.f;
    }
  };
  fetch(c_begin);
  // L^{-1}[r][t] = 0 for t > r, and rows and columns past l are zero: rows
  // r >= l of the result are zero without a product
  const int tmax = RR * ti < l ? min(RR * ti + RR, l) : 0;
  for (int64_t c0 = c_begin; c0 < c_end; c0 += 64) {
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = tid + 256 * q, r = e / 64, c = e % 64;
      Xs[r * XLD + c] = rx[q];
    }
    __syncthreads();
    if (c0 + 64 < c_end) fetch(c0 + 64);
    float acc[RR][4];
#pragma unroll
    for (int q = 0; q < RR; ++q)
#pragma unroll
      for (int p = 0; p < 4; ++p) acc[q][p] = 0.f;
#pragma unroll 4
    for (int t = 0; t < tmax; ++t) {
      float a[RR];
#pragma unroll
      for (int q = 0; q < RR; q += 4) {
        const float4 a4 = *reinterpret_cast<const float4*>(&LsT[t * LLD + RR * ti + q]);
        a[q] = a4.x; a[q + 1] = a4.y; a[q + 2] = a4.z; a[q + 3] = a4.w;
      }
      const float4 b4 = *reinterpret_cast<const float4*>(&Xs[t * XLD + 4 * tj]);
      const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int q = 0; q < RR; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[q][p] = fmaf(a[q], bv[p], acc[q][p]);
    }
    const int64_t col = c0 + 4 * tj;
#pragma unroll
    for (int q = 0; q < RR; ++q) {
      const int64_t off = (int64_t)(RR * ti + q) * ld + col;
      if (vec && col + 3 < c_end) {
        *reinterpret_cast<float4*>(Y + off) = make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
        if (Yb) {
          bf16 hv[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) hv[p] = __float2bfloat16_rn(acc[q][p]);
          *reinterpret_cast<uint2*>(Yb + off) = *reinterpret_cast<const uint2*>(hv);
        }
      } else {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if (col + p >= c_end) break;
          Y[off + p] = acc[q][p];
          if (Yb) Yb[off + p] = __float2bfloat16_rn(acc[q][p]);
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Block leverage scores (Def. 2) straight from the factors: with Q_B (the
// panel in Pn0) and the right factor W of the small SVD, V_k^T = W_k^T Q_B^T,
// so column j of V_k^T is W_k^T q_j; the score of block g is the FP64 sum of
// the squares over the block's columns.  Row blocks use U~ and Q (Pm0).  One
// CTA per block, fixed order.
// ---------------------------------------------------------------------------
template <int LP>
__global__ void __launch_bounds__(128) scores_kernel(const Item* items, const bcur_batch_io_t* io,
                                                     Work blocks, int* status) {
  const int b = find_item(blocks, blockIdx.x);
  const Item& I = items[b];
  int g = blockIdx.x - blocks.prefix[b];
  const bool col = g < I.Gc;
  if (!col) g -= I.Gc;
  const float* F = col ? I.W : I.Ut;
  const float* P = col ? I.Pn0 : I.Pm0;
  const int64_t h = col ? I.n : I.m, ld = col ? I.ldn : I.ldm;
  const int k = I.k;
  extern __shared__ __align__(16) float FsT[];  // LP x LP, FsT[t][i] = F[i][t]
  __shared__ double red[4];
  for (int e = threadIdx.x; e < LP * LP; e += blockDim.x) {
    const int i = e / LP, t = e % LP;
    FsT[t * LP + i] = F[e];
  }
  __syncthreads();
  const int64_t j0 = (int64_t)g * I.s;
  const int64_t j1 = j0 + I.s < h ? j0 + I.s : h;
  double acc = 0.0;
  // Blocks narrower than the CTA split the k rows of V^T among thread groups
  // (group tg takes t = tg, tg + groups, ...); wider ones take a column per
  // thread.  The mapping depends only on s, so the order of every sum is a
  // function of the decomposition alone.
  const int nt = (int)blockDim.x;
  const int groups = I.s >= nt ? 1 : nt / I.s;
  const int span = groups == 1 ? nt : I.s;
  const int tg = groups == 1 ? 0 : (int)threadIdx.x / I.s;
  const int jc = groups == 1 ? (int)threadIdx.x : (int)threadIdx.x % I.s;
  // rows of the panel past l are zero: only the leading l4 are read
  const int l4 = (I.l + 3) & ~3;
  for (int64_t j = j0 + jc; tg < groups && j < j1; j += span) {
    float p[LP];
#pragma unroll
    for (int i = 0; i < LP; ++i) p[i] = i < l4 ? P[i * ld + j] : 0.f;
    for (int t = tg; t < k; t += groups) {
      float v = 0.f;
#pragma unroll
      for (int i = 0; i < LP; i += 4) {  // broadcast float4 reads of row t of F^T
        const float4 f = *reinterpret_cast<const float4*>(&FsT[t * LP + i]);
        v = fmaf(f.x, p[i], v);
        v = fmaf(f.y, p[i + 1], v);
        v = fmaf(f.z, p[i + 2], v);
        v = fmaf(f.w, p[i + 3], v);
      }
      acc = fma((double)v, (double)v, acc);
    }
  }
  const double sum = block_sum(acc, red);
  if (threadIdx.x == 0) {
    (col ? io[b].col_scores : io[b].row_scores)[g] = sum;
    if (!isfinite(sum)) dev_set_status(status, (int)BCUR_ENONFINITE);
  }
}

// ---------------------------------------------------------------------------
// Sampling (Alg. 1 step 2, without replacement) and the gather map: one
// thread per (decomposition, side).
// ---------------------------------------------------------------------------
__global__ void sample_kernel(const Item* items, const bcur_batch_io_t* io) {
  if (threadIdx.x != 0) return;
  const int b = blockIdx.x, side = blockIdx.y;
  const Item& I = items[b];
  const int G = side ? I.Gr : I.Gc, g = side ? I.gr : I.gc;
  const double* sc = side ? io[b].row_scores : io[b].col_scores;
  const double* u = side ? io[b].u_row : io[b].u_col;
  int32_t* idx = side ? io[b].row_idx : io[b].col_idx;
  sample_seq(sc, G, u, g, 0, idx, nullptr, I.remaining + (side ? I.Gc : 0));
  int* map = side ? I.rowmap : I.colmap;
  const int cap = side ? I.rpad : I.cpad;
  const int64_t h = side ? I.m : I.n;
  int base = 0;
  for (int t = 0; t < g; ++t) {
    const int64_t start = (int64_t)idx[t] * I.s;
    const int64_t size = (h - start) < I.s ? (h - start) : I.s;
    for (int64_t e = 0; e < size && base + e < cap; ++e) map[base + e] = (int)(start + e);
    base += (int)size;
  }
  for (int e = base; e < cap; ++e) map[e] = -1;
}

// C^T panel (cpad x m) and R (rpad x n) as BF16 pairs, straight from A.
// C^T of one decomposition as a BF16 pair, 64 x 64 tiles (rows i of A, gathered
// columns cc) through shared memory.  A tile whose 64 columns are consecutive
// in A and start on a 16-byte boundary reads float4 row pieces; other tiles
// (a block boundary inside the tile, blocks of 16 or 32 drawn out of order)
// read element by element.  Stores are two BF16 per thread and part.
__global__ void __launch_bounds__(256) gather_c_kernel(const Item* items,
                                                       const bcur_batch_io_t* io, Work tiles) {
  const int b = find_item(tiles, blockIdx.x);
  const Item& I = items[b];
  const int t = blockIdx.x - tiles.prefix[b];
  const int ti = (int)((I.m + 63) / 64);
  const int64_t i0 = (int64_t)(t % ti) * 64, c0 = (int64_t)(t / ti) * 64;
  __shared__ float tile[64][65];
  const int tid = threadIdx.x;
  const float* A = io[b].A;
  const int first = I.colmap[c0];
  int ok = first >= 0 && (first % 4) == 0 && c0 + 63 < I.cpad && (I.lda % 4) == 0 &&
           ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  if (ok) ok = I.colmap[c0 + (tid & 63)] == first + (tid & 63);
  ok = __syncthreads_and(ok);
  if (ok) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int r = (tid >> 4) + 16 * it, q = tid & 15;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i0 + r < I.m)
        v = __ldcs(reinterpret_cast<const float4*>(A + (i0 + r) * I.lda + first) + q);
      tile[r][4 * q] = v.x;
      tile[r][4 * q + 1] = v.y;
      tile[r][4 * q + 2] = v.z;
      tile[r][4 * q + 3] = v.w;
    }
  } else {
    for (int e = tid; e < 64 * 64; e += 256) {
      const int r = e >> 6, c = e & 63;
      const int64_t cc = c0 + c, i = i0 + r;
      const int col = cc < I.cpad ? I.colmap[cc] : -1;
      tile[r][c] = (col >= 0 && i < I.m) ? A[i * I.lda + col] : 0.f;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const int c = (tid >> 5) + 8 * it, ip = tid & 31;
    const int64_t cc = c0 + c, i = i0 + 2 * ip;
    if (cc >= I.cpad || i >= I.m) continue;
    bf16* dh = I.XCh[0] + cc * I.ldm + i;
    bf16* dl = I.XCl[0] + cc * I.ldm + i;
    const float v0 = tile[2 * ip][c];
    if (i + 1 < I.m) {
      const float v1 = tile[2 * ip + 1][c];
      const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
      const float2 f = __bfloat1622float2(h);
      *reinterpret_cast<__nv_bfloat162*>(dh) = h;
      *reinterpret_cast<__nv_bfloat162*>(dl) = __floats2bfloat162_rn(v0 - f.x, v1 - f.y);
    } else {
      const bf16 h = __float2bfloat16_rn(v0);
      dh[0] = h;
      dl[0] = __float2bfloat16_rn(v0 - __bfloat162float(h));
    }
  }
}

__global__ void __launch_bounds__(256) gather_r_kernel(const Item* items,
                                                       const bcur_batch_io_t* io, Work rows) {
  const int b = find_item(rows, blockIdx.x);
  const Item& I = items[b];
  const int rr = blockIdx.x - rows.prefix[b];
  const int row = I.rowmap[rr];
  const float* A = io[b].A;
  bf16* hr = I.XRh[0] + (int64_t)rr * I.ldn;
  bf16* lr = I.XRl[0] + (int64_t)rr * I.ldn;
  const float* src = A + (int64_t)(row >= 0 ? row : 0) * I.lda;
  // four per thread when the row is 16-byte aligned (n, lda, ldn multiples of 4)
  const bool v4 = ((reinterpret_cast<uintptr_t>(src) & 15) == 0) && (I.n % 4 == 0) &&
                  ((reinterpret_cast<uintptr_t>(hr) & 7) == 0) &&
                  ((reinterpret_cast<uintptr_t>(lr) & 7) == 0);
  if (v4) {
    for (int64_t j = 4 * (int64_t)threadIdx.x; j < I.n; j += 4 * (int64_t)blockDim.x) {
      const float4 v = row >= 0 ? *reinterpret_cast<const float4*>(src + j)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
      const float vv[4] = {v.x, v.y, v.z, v.w};
      bf16 h[4], l[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        h[q] = __float2bfloat16_rn(vv[q]);
        l[q] = __float2bfloat16_rn(vv[q] - __bfloat162float(h[q]));
      }
      *reinterpret_cast<uint2*>(hr + j) = *reinterpret_cast<const uint2*>(h);
      *reinterpret_cast<uint2*>(lr + j) = *reinterpret_cast<const uint2*>(l);
    }
    return;
  }
  for (int64_t j = threadIdx.x; j < I.n; j += blockDim.x) {
    const float v = row >= 0 ? src[j] : 0.f;
    const bf16 h = __float2bfloat16_rn(v);
    hr[j] = h;
    lr[j] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// ---------------------------------------------------------------------------
// Wide Cholesky G = L L^T (w x w, w <= WMAX, FP32, lower part of G) with the
// drop rule and L^{-1}, one CTA per (decomposition, side).  Right-looking by
// leaves of NB columns: factor the leaf (potrf_leaf), solve the panel below
// it (L_iJ = G_iJ L_JJ^{-T}, kept in shared memory), update the trailing
// lower triangle in place.  Then L^{-1} block row by block row:
// X_IJ = -X_II sum_{J <= K < I} L_IK X_KJ.  Writes L, L^{-1} (zeros above the
// diagonal) and L^{-1} as a BF16 pair.  Every 64 x 64 x 64 product reads its
// left operand k-major (A^T[t][row]) and its right operand row-major
// (B[t][col]) from shared memory, two float4 per k for a thread's 4 x 4
// outputs.
// ---------------------------------------------------------------------------
constexpr int WLD = NB + 4;   // leading dimension of every 64-wide tile (potrf_leaf's too)
// Shared memory: leaf L and L^{-1}, X^T, and the k-major panel below the leaf
// (its width depends on the largest w of the launch); the inverse phase
// reuses the first four tiles' worth.
constexpr int kWideBase = 3 * NB * WLD;
constexpr size_t wide_smem(int wmax) {
  return (size_t)(kWideBase + NB * (wmax - NB + 4)) * sizeof(float);
}
static_assert(4 * NB * WLD <= kWideBase + NB * (NB + 4), "inverse tiles must fit");

// acc[q][p] += sum_{t < kn} AT[t][4 ti + q] * B[t][4 tj + p]  (lda, ldb multiples of 4)
__device__ __forceinline__ void tile_acc_k(const float* AT, int lda, const float* B, int ldb,
                                           int ti, int tj, int kn, float (&acc)[4][4]) {
#pragma unroll 4
  for (int t = 0; t < kn; ++t) {
    const float4 a4 = *reinterpret_cast<const float4*>(&AT[t * lda + 4 * ti]);
    const float4 b4 = *reinterpret_cast<const float4*>(&B[t * ldb + 4 * tj]);
    const float a[4] = {a4.x, a4.y, a4.z, a4.w}, bb[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int p = 0; p < 4; ++p) acc[q][p] = fmaf(a[q], bb[p], acc[q][p]);
  }
}

// 64 x 64 tile of a row-major global matrix (ld) into shared memory:
// transposed (dst[c][r] = src[r][c]) or as is (dst[r][c]), ld of dst WLD.
__device__ __forceinline__ void load_tile(const float* src, int64_t ld, float* dst, bool transpose) {
  const int tid = threadIdx.x;
  float4 v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = tid + 256 * q, r = e >> 4, c4 = (e & 15) * 4;
    v[q] = *reinterpret_cast<const float4*>(src + (int64_t)r * ld + c4);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = tid + 256 * q, r = e >> 4, c4 = (e & 15) * 4;
    if (transpose) {
      dst[(c4 + 0) * WLD + r] = v[q].x;
      dst[(c4 + 1) * WLD + r] = v[q].y;
      dst[(c4 + 2) * WLD + r] = v[q].z;
      dst[(c4 + 3) * WLD + r] = v[q].w;
    } else {
      *reinterpret_cast<float4*>(&dst[r * WLD + c4]) = v[q];
    }
  }
}

__global__ void __launch_bounds__(256) wchol_kernel(const Item* items, const int* entries,
                                                    int pass, int gated) {
  extern __shared__ __align__(16) float sm[];
  float* S = sm;              // NB x WLD: leaf L
  float* X = S + NB * WLD;    // NB x WLD: leaf L^{-1}
  float* XT = X + NB * WLD;   // NB x WLD: XT[t][c] = X[c][t]
  float* PsT = XT + NB * WLD; // NB x pld: PsT[t][i] = panel row i, column t
  const int e0 = entries[blockIdx.x];
  const Item& I = items[e0 >> 1];
  if (gated && *I.refine == 0) return;  // uniform over the CTA
  const int side = e0 & 1;
  const int w = side ? I.rpad : I.cpad;
  const int pld = w - NB + 4;
  float* G = side ? I.GR : I.GC;
  float* L = side ? I.LR[pass] : I.LC[pass];
  float* Li = side ? I.LRi[pass] : I.LCi[pass];
  bf16* Lh = side ? I.LRih[pass] : I.LCih[pass];
  bf16* Ll = side ? I.LRil[pass] : I.LCil[pass];
  const int tid = threadIdx.x, ti = tid / 16, tj = tid % 16;
  __shared__ float s_red[8];
  __shared__ float s_tol;
  float mx = 0.f;
  for (int i = tid; i < w; i += 256) mx = fmaxf(mx, G[(int64_t)i * w + i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) s_red[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    float m2 = 0.f;
    for (int i = 0; i < 8; ++i) m2 = fmaxf(m2, s_red[i]);
    s_tol = (float)(64.0 * 1.1920928955078125e-07 * (double)m2);
  }
  __syncthreads();
  const float tol = s_tol;
  const int nbk = w / NB;
  int kept = 0;
  for (int J = 0; J < nbk; ++J) {
    const int j0 = J * NB;
    kept += potrf_leaf<float, NB>(G + (int64_t)j0 * w + j0, w, S, X, tol);
    for (int e = tid; e < NB * NB; e += 256) {
      const int i = e / NB, c = e % NB;
      L[(int64_t)(j0 + i) * w + j0 + c] = c <= i ? S[i * WLD + c] : 0.f;
      Li[(int64_t)(j0 + i) * w + j0 + c] = c <= i ? X[i * WLD + c] : 0.f;
      XT[c * WLD + i] = X[i * WLD + c];
    }
    const int R = w - j0 - NB;
    if (R > 0) {
      for (int r0 = 0; r0 < R; r0 += NB) {
        const float* src = G + (int64_t)(j0 + NB + r0) * w + j0;
        float4 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = tid + 256 * q, r = e >> 4, c4 = (e & 15) * 4;
          v[q] = *reinterpret_cast<const float4*>(src + (int64_t)r * w + c4);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = tid + 256 * q, r = e >> 4, c4 = (e & 15) * 4;
          PsT[(c4 + 0) * pld + r0 + r] = v[q].x;
          PsT[(c4 + 1) * pld + r0 + r] = v[q].y;
          PsT[(c4 + 2) * pld + r0 + r] = v[q].z;
          PsT[(c4 + 3) * pld + r0 + r] = v[q].w;
        }
      }
      __syncthreads();
      // panel: L_iJ = G_iJ X_JJ^T, 64 rows at a time, in place (k-major)
      for (int r0 = 0; r0 < R; r0 += NB) {
        float acc[4][4] = {};
        tile_acc_k(PsT + r0, pld, XT, WLD, ti, tj, NB, acc);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = r0 + 4 * ti + q;
          *reinterpret_cast<float4*>(&L[(int64_t)(j0 + NB + i) * w + j0 + 4 * tj]) =
              make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
#pragma unroll
          for (int p = 0; p < 4; ++p) PsT[(4 * tj + p) * pld + i] = acc[q][p];
        }
        __syncthreads();
      }
      // trailing update of the lower triangle, tile (bi, bj), bj <= bi
      const int nR = R / NB;
      for (int t = 0; t < nR * (nR + 1) / 2; ++t) {
        int bi = 0;
        while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
        const int bj = t - bi * (bi + 1) / 2;
        float acc[4][4] = {};
        // sum_t P[bi*NB + a][t] P[bj*NB + b][t]
        tile_acc_k(PsT + bi * NB, pld, PsT + bj * NB, pld, ti, tj, NB, acc);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t row = j0 + NB + bi * NB + 4 * ti + q;
          float4* g = reinterpret_cast<float4*>(&G[row * w + j0 + NB + bj * NB + 4 * tj]);
          float4 o = *g;
          o.x -= acc[q][0];
          o.y -= acc[q][1];
          o.z -= acc[q][2];
          o.w -= acc[q][3];
          *g = o;
        }
      }
    }
    __syncthreads();
  }
  // L^{-1}: off-diagonal blocks by block rows (tiles in the leaf area)
  float* TAT = sm;             // L_IK^T
  float* TB = sm + NB * WLD;   // X_KJ
  float* TT = sm + 2 * NB * WLD;  // sum_K L_IK X_KJ
  float* TXT = sm + 3 * NB * WLD; // X_II^T
  for (int Ib = 1; Ib < nbk; ++Ib) {
    load_tile(Li + (int64_t)(Ib * NB) * w + Ib * NB, w, TXT, true);
    for (int Jb = 0; Jb < Ib; ++Jb) {
      float acc[4][4] = {};
      for (int Kb = Jb; Kb < Ib; ++Kb) {
        load_tile(L + (int64_t)(Ib * NB) * w + Kb * NB, w, TAT, true);
        load_tile(Li + (int64_t)(Kb * NB) * w + Jb * NB, w, TB, false);
        __syncthreads();
        tile_acc_k(TAT, WLD, TB, WLD, ti, tj, NB, acc);
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(&TT[(4 * ti + q) * WLD + 4 * tj]) =
            make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
      __syncthreads();
      float acc2[4][4] = {};
      tile_acc_k(TXT, WLD, TT, WLD, ti, tj, NB, acc2);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(&Li[(int64_t)(Ib * NB + 4 * ti + q) * w + Jb * NB + 4 * tj]) =
            make_float4(-acc2[q][0], -acc2[q][1], -acc2[q][2], -acc2[q][3]);
      __syncthreads();
    }
  }
  // zeros above the block diagonal, then the BF16 pair of L^{-1} (four per thread)
  const int w4 = w / 4;
  for (int e = tid; e < w * w4; e += 256) {
    const int i = e / w4, c = (e - i * w4) * 4;
    const int64_t off = (int64_t)i * w + c;
    float4 lv = *reinterpret_cast<const float4*>(&Li[off]);
    if (c / NB > i / NB) {
      *reinterpret_cast<float4*>(&L[off]) = make_float4(0.f, 0.f, 0.f, 0.f);
      lv = make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4*>(&Li[off]) = lv;
    }
    const float vv[4] = {lv.x, lv.y, lv.z, lv.w};
    bf16 h[4], l[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      h[p] = __float2bfloat16_rn(vv[p]);
      l[p] = __float2bfloat16_rn(vv[p] - __bfloat162float(h[p]));
    }
    *reinterpret_cast<uint2*>(&Lh[off]) = *reinterpret_cast<const uint2*>(h);
    *reinterpret_cast<uint2*>(&Ll[off]) = *reinterpret_cast<const uint2*>(l);
  }
  if (tid == 0) I.kept[side * 2 + pass] = kept;
}

// U (cpad x rpad workspace) -> the caller's cmax x rmax output.
__global__ void copy_u_kernel(const Item* items, const bcur_batch_io_t* io, Work rows) {
  const int b = find_item(rows, blockIdx.x);
  const Item& I = items[b];
  float* U = io[b].U;
  if (!U) return;
  const int r = blockIdx.x - rows.prefix[b];
  for (int c = threadIdx.x; c < I.rmax; c += blockDim.x)
    U[(int64_t)r * I.rmax + c] = I.Uf[(int64_t)r * I.rpad + c];
}

// ||A - CUR||_F from the residual tiles' partial sums, fixed order.  refine =
// 0: from the one-term residual, and set the item's refinement flag
// (residual_needs_refine); refine = 1: from the three-term residual, only for
// items whose flag is set.
__global__ void __launch_bounds__(256) finish_kernel(const Item* items, const bcur_batch_io_t* io,
                                                     int refine) {
  const Item& I = items[blockIdx.x];
  if (refine && *I.refine == 0) return;
  __shared__ double red[8];
  const int64_t n = kResidSlots * I.res_units;
  double e2 = 0.0, x2 = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    e2 += I.partials[2 * i];
    x2 += I.partials[2 * i + 1];
  }
  const double se = block_sum(e2, red);
  __syncthreads();
  const double sx = block_sum(x2, red);
  if (threadIdx.x == 0) {
    double* err = io[blockIdx.x].err;
    const double fe = sqrt(se), fx = sqrt(sx);
    err[0] = fe;
    err[1] = fx > 0.0 ? fe / fx : 0.0;
    err[2] = fx;
    if (!refine) *I.refine = residual_needs_refine(err[1]) ? 1 : 0;
  }
}

}  // namespace

bcur_status_t split_inputs(const Item* items, const bcur_batch_io_t* io, Work rows8, int total8,
                           int B, int lp, cudaStream_t s, int mode) {
  if (mode < 0 || mode > 2) return BCUR_EINVAL;
  split_kernel<<<total8 + (mode == 2 ? 0 : B * (lp / 8)), 256, 0, s>>>(items, io, rows8, total8,
                                                                        lp, mode);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

namespace {
template <typename K>
bcur_status_t allow_smem(K kernel, size_t bytes, bool& done) {
  if (!done && bytes > 48 * 1024) {
    BCUR_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes));
  }
  done = true;
  return BCUR_OK;
}

template <int LP>
bcur_status_t gram_lp(const Item* items, Work chunks, int total, int sel, cudaStream_t s) {
  sgram_kernel<LP><<<total, 256, 0, s>>>(items, chunks, sel);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

template <int LP>
bcur_status_t chol_lp(const Item* items, int B, int sel, int pass, int want_lb, cudaStream_t s) {
  const size_t smem = (size_t)LP * (LP + 1) * sizeof(double);
  static bool attr = false;
  BCUR_TRY(allow_smem(schol_kernel<LP>, smem, attr));
  schol_kernel<LP><<<B, 256, smem, s>>>(items, sel, pass, want_lb);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

template <int LP>
bcur_status_t apply_lp(const Item* items, Work chunks, int total, int src, int dst,
                       int write_bf16, cudaStream_t s) {
  const size_t smem = (size_t)LP * (LP + 4 + 64 + 4) * sizeof(float);
  static bool attr = false;
  BCUR_TRY(allow_smem(sapply_kernel<LP>, smem, attr));
  sapply_kernel<LP><<<total, 256, smem, s>>>(items, chunks, src, dst, write_bf16);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

template <int LP>
bcur_status_t scores_lp(const Item* items, const bcur_batch_io_t* io, Work blocks, int total,
                        int* status, cudaStream_t s) {
  const size_t smem = (size_t)LP * LP * sizeof(float);
  static bool attr = false;
  BCUR_TRY(allow_smem(scores_kernel<LP>, smem, attr));
  scores_kernel<LP><<<total, 128, smem, s>>>(items, io, blocks, status);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}
}  // namespace

bcur_status_t skinny_gram(const Item* items, Work chunks, int total, int sel, int lp,
                          cudaStream_t s) {
  return lp == 64 ? gram_lp<64>(items, chunks, total, sel, s)
                  : gram_lp<128>(items, chunks, total, sel, s);
}

bcur_status_t skinny_chol(const Item* items, int B, int sel, int pass, int want_lb, int lp,
                          cudaStream_t s) {
  return lp == 64 ? chol_lp<64>(items, B, sel, pass, want_lb, s)
                  : chol_lp<128>(items, B, sel, pass, want_lb, s);
}

bcur_status_t skinny_apply(const Item* items, Work chunks, int total, int src, int dst,
                           int write_bf16, int lp, cudaStream_t s) {
  return lp == 64 ? apply_lp<64>(items, chunks, total, src, dst, write_bf16, s)
                  : apply_lp<128>(items, chunks, total, src, dst, write_bf16, s);
}

bcur_status_t scores(const Item* items, const bcur_batch_io_t* io, Work blocks, int total,
                     int* status, int lp, cudaStream_t s) {
  return lp == 64 ? scores_lp<64>(items, io, blocks, total, status, s)
                  : scores_lp<128>(items, io, blocks, total, status, s);
}

bcur_status_t sample(const Item* items, const bcur_batch_io_t* io, int B, cudaStream_t s) {
  sample_kernel<<<dim3(B, 2), 32, 0, s>>>(items, io);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

bcur_status_t gather(const Item* items, const bcur_batch_io_t* io, Work ctiles, int ctotal,
                     Work rrows, int rtotal, cudaStream_t s) {
  gather_c_kernel<<<ctotal, 256, 0, s>>>(items, io, ctiles);
  BCUR_LAUNCH_CHECK();
  gather_r_kernel<<<rtotal, 256, 0, s>>>(items, io, rrows);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

bcur_status_t wide_chol(const Item* items, const int* entries, int count, int wmax, int pass,
                        cudaStream_t s, int gated) {
  if (count < 1) return BCUR_OK;
  if (wmax < NB || wmax > WMAX) return BCUR_EINVAL;
  static bool attr = false;
  if (!attr) {
    BCUR_CUDA_TRY(cudaFuncSetAttribute(wchol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)wide_smem(WMAX)));
    attr = true;
  }
  wchol_kernel<<<count, 256, wide_smem(wmax), s>>>(items, entries, pass, gated);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

bcur_status_t copy_u(const Item* items, const bcur_batch_io_t* io, Work urows, int total,
                     cudaStream_t s) {
  copy_u_kernel<<<total, 256, 0, s>>>(items, io, urows);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

bcur_status_t finish(const Item* items, const bcur_batch_io_t* io, int B, int refine,
                     cudaStream_t s) {
  finish_kernel<<<B, 256, 0, s>>>(items, io, refine);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

__global__ void fit_terms_kernel(const Item* items, int B, int* terms) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
    terms[b] = *items[b].refine ? 3 : 1;
}

bcur_status_t fit_terms(const Item* items, int B, int* terms, cudaStream_t s) {
  if (B < 1) return BCUR_OK;
  fit_terms_kernel<<<(B + 255) / 256, 256, 0, s>>>(items, B, terms);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

}  // namespace batch
}  // namespace bcur
