// Device-visible description of one decomposition of a batch, shared by the
// batched kernels (batch.cu) and the batched plan (batch_api.cu).
#pragma once

#include <cuda_bf16.h>

#include "kernels.h"

namespace bcur {
namespace batch {

// Panel rows of a batch: 64 when every l = k + p <= 64, else 128; rows past
// an item's l stay zero.
constexpr int LP_MAX = 128;
constexpr int CH = 1024;    // columns per skinny-Gram chunk
constexpr int AP = 256;     // columns per skinny-apply chunk
constexpr int WMAX = 512;   // largest padded c or r
constexpr int NB = 64;      // leaf size of the wide Cholesky

using bf16 = __nv_bfloat16;

// Skinny panels of one decomposition, selected by number in the kernels.
enum PanelSel { PM0 = 0, PM1 = 1, PN0 = 2, PN1 = 3 };

struct Item {
  int64_t m, n, lda;
  int k, l, s;
  int lp;                    // panel rows of the batch (64 or 128)
  int Gc, Gr, gc, gr;
  int64_t ldm, ldn;          // panel leading dimensions (multiples of 64)
  int cpad, rpad;            // c and r padded to the leaf size
  int cmax, rmax;            // gc * s, gr * s: the U output is cmax x rmax
  int chunks_m, chunks_n;    // skinny-Gram chunks along m and n
  int64_t res_units;         // residual tiles (2 kResidSlots partial doubles each)
  // sketch
  bf16 *Ah, *Al;             // A as BF16 pair, m x ldn
  bf16* Om;                  // Omega^T, LP x ldn
  float *Pm0, *Pm1, *Pn0, *Pn1;
  bf16 *Qh, *Zh;             // BF16 copies of the orthonormal panels
  float* gpart;              // max(chunks_m, chunks_n) x LP x LP
  double *G64, *L64a, *L64b, *Linv64;
  float* LinvT;
  double* Lb;                // L_B (LP x LP) in the batch-contiguous Jacobi input
  float *Ut, *W;             // Jacobi outputs (LP x LP)
  unsigned char* remaining;  // Gc + Gr bytes for sampling
  int *colmap, *rowmap;      // cpad / rpad entries, -1 past c / r
  // fit
  bf16 *XCh[2], *XCl[2];     // C^T panels (cpad x ldm), ping-pong
  bf16 *XRh[2], *XRl[2];     // R panels (rpad x ldn)
  float *GC, *GR;            // Gram matrices
  float *LC[2], *LCi[2], *LR[2], *LRi[2];        // Cholesky factors and inverses per pass
  bf16 *LCih[2], *LCil[2], *LRih[2], *LRil[2];   // the inverses as BF16 pairs
  bf16 *Wh, *Wl;             // W = A Q_R^T, m x rpad
  float* Mf;                 // M = Q_C A Q_R^T (cpad x rpad)
  bf16 *Mh, *Ml;
  bf16 *U1h, *U1l, *U2h, *U2l;
  float* Uf;                 // U (cpad x rpad)
  bf16 *Ph, *Pl;             // P = Q_C^T M as a BF16 pair, m x rpad
  double* partials;          // 8 * res_units
  int* kept;                 // 4: C pass 0/1, R pass 0/1
  int* refine;               // 1: recompute the residual with BF16 pairs
};

// Work list: prefix sums of per-item unit counts (count + 1 entries).
struct Work {
  const int* prefix;
  int count;
};

__device__ __forceinline__ int find_item(const Work& w, int x) {
  int lo = 0, hi = w.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (w.prefix[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Launchers (batch.cu).  `items` / `io` are device tables of B entries.
bcur_status_t split_inputs(const Item* items, const bcur_batch_io_t* io, Work rows8, int total8,
                           int B, int lp, cudaStream_t s,
                           int mode = 0);
bcur_status_t skinny_gram(const Item* items, Work chunks, int total, int sel, int lp,
                          cudaStream_t s);
bcur_status_t skinny_chol(const Item* items, int B, int sel, int pass, int want_lb, int lp,
                          cudaStream_t s);
bcur_status_t skinny_apply(const Item* items, Work chunks, int total, int src, int dst,
                           int write_bf16, int lp, cudaStream_t s);
bcur_status_t scores(const Item* items, const bcur_batch_io_t* io, Work blocks, int total,
                     int* status, int lp, cudaStream_t s);
bcur_status_t sample(const Item* items, const bcur_batch_io_t* io, int B, cudaStream_t s);
bcur_status_t gather(const Item* items, const bcur_batch_io_t* io, Work ctiles, int ctotal,
                     Work rrows, int rtotal, cudaStream_t s);
// entries: (item << 1 | side) of the decompositions in this launch, all with
// w <= wmax (side 0: C^T with w = cpad, side 1: R with w = rpad).  gated: only
// the items whose refinement flag is set.
bcur_status_t wide_chol(const Item* items, const int* entries, int count, int wmax, int pass,
                        cudaStream_t s, int gated = 0);
bcur_status_t copy_u(const Item* items, const bcur_batch_io_t* io, Work urows, int total,
                     cudaStream_t s);
// terms[b] = 3 when item b's refinement flag is set, else 1 (device array).
bcur_status_t fit_terms(const Item* items, int B, int* terms, cudaStream_t s);
bcur_status_t finish(const Item* items, const bcur_batch_io_t* io, int B, int refine,
                     cudaStream_t s);

}  // namespace batch

// Batched Jacobi SVD (small.cu): `batch` independent w x w problems stored
// contiguously (X, Ut, W, jwork at stride w*w, sigma at stride w).  With
// wdim (device, one int per problem) only each problem's leading
// wdim[b] x wdim[b] block is factored (the rest of X must be zero); the
// outputs past it are zeros (W: identity there).
template <typename T>
bcur_status_t jacobi_svd_batched(const double* X, int w, T* Ut, T* W, double* sigma, T* jwork,
                                 int* status, int batch, cudaStream_t s,
                                 const int* wdim = nullptr);

}  // namespace bcur
