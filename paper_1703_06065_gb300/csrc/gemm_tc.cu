// Dense GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   D (Mm x Nm, FP32) = alpha * A (Mm x K) . B (Nm x K)^T        ("MMA space")
//
// Operands are BF16 (kind::f16), FP8 e4m3 (kind::f8f6f4, both operands
// K-major, with optional per-row / per-column output scales that undo a
// row-wise quantisation exactly), or FP32 read as TF32 (kind::tf32).  A BF16
// operand is either K-major (rows contiguous along K) or MN-major (contiguous
// along M / N); TF32 operands must be K-major (the MMA reads zeros for an
// MN-major TF32 operand on sm_103a, so such calls are refused).  TMA brings
// 128-byte-wide boxes into shared memory with the 128-byte swizzle, and the
// shared-memory matrix descriptors describe the same canonical layout to the
// MMA.  Accumulators live in tensor memory (TMEM), double-buffered so that
// the epilogue of one tile overlaps the main loop of the next.
//
// Split precision ("parts" = 3): an FP32 value x is carried as a BF16 pair
// hi = bf16(x), lo = bf16(x - hi), and A B is accumulated as
// A_hi B_hi + A_hi B_lo + A_lo B_hi, which keeps about 16 mantissa bits.  The
// three products are consecutive K-slices of one accumulation: iteration i
// of a tile's K loop handles K-block klo + i/3 with the operand pair i%3.
//
// CTA = 6 warps (10 for the grouped residual), persistent over a static tile
// schedule:
//   warp 0      TMA producer (one elected thread)
//   warp 1      TMEM allocator + MMA issuer (one elected thread)
//   warps 2..   epilogue: tcgen05.ld from TMEM (each warp owns the 32 TMEM
//               lanes of its rank within the warpgroup), then store, split-K
//               partial store, or fused residual reduction.
// Every mbarrier wait is bounded (2 s on %globaltimer); a wait that runs out
// records BCUR_ETIMEOUT, the kernel drains what it issued and returns.
//
// Grouped mode: one persistent launch over many independent GEMMs of
// different shapes (a batch of decompositions).  Each GEMM's tensor maps and
// parameters sit in a device table; the CTAs walk the concatenation of all
// GEMMs' tiles (heaviest GEMMs first, snake order across CTAs) and look up
// the owning GEMM of each tile by binary search over the tile prefix sums.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace bcur {
namespace tc {

constexpr int BM = 128;
// Epilogue warps: 4 (one per TMEM lane quarter).  The grouped residual,
// whose short-K tiles are bound by streaming X from HBM, has 8 (two warps per
// lane quarter, each on half the columns) and gives up a pipeline stage for
// their transpose tiles; the single-GEMM residual (long K, bound by the MMA
// feed) keeps 4 warps and the fourth stage.
template <int EPI, bool G> __host__ __device__ constexpr int epi_warps() {
  return (EPI == 2 && G) ? 8 : 4;
}
template <int EPI, bool G> __host__ __device__ constexpr int threads_of() {
  return 64 + 32 * epi_warps<EPI, G>();
}
constexpr int kStageABytes = BM * 128;  // 128 rows (or MN elements) x 128 bytes of K
// Bound of the waits that drain the kernel's own asynchronous work before it
// exits (copies and MMAs in flight): always the full 2 s.
constexpr uint64_t kWaitNs = 2000000000ull;
// Bound of the waits of the main loop (a stage, an accumulator); 2 s unless
// lowered from the host (bcur_set_wait_budget_ns), e.g. by a test that makes
// a wait run out on purpose.
__device__ unsigned long long g_wait_budget_ns = 2000000000ull;

enum Epi { EPI_STORE = 0, EPI_PARTIAL = 1, EPI_RESID = 2 };

struct Params {
  int Mm, Nm, K;
  int parts;             // 1, or 3 for the split-precision product
  int a_mn, b_mn;        // 1: operand is MN-major
  int tiles_m, tiles_n, ksplit, kblocks;
  int triA, triB;        // 1 lower / 2 upper (A: A(i,k)=0 for k>i / k<i; B: B(k,j)=0 for k<j / k>j)
  int tri_out;           // 1: keep row >= col, 2: keep row <= col (MMA space)
  int rev_m, rev_n;      // visit M / N tiles in reverse order (heaviest first)
  int batch;             // independent problems (third tensor-map coordinate)
  int64_t sD;            // element stride between the batch's outputs
  float alpha, beta;
  float* D;              // FP32 output (may be null)
  __nv_bfloat16* Dh;     // BF16 hi part of the output (may be null)
  __nv_bfloat16* Dl;     // BF16 lo part of the output (may be null)
  int64_t ldd;
  int transD;            // D stored as D^T (element (i,j) at D[j*ldd + i])
  float* part;           // split-K partial slices (Mm x Nm, row-major each)
  const float* X;        // residual reference matrix (Mm x Nm, ldx)
  int64_t ldx;
  double* partials;      // per-CTA {sum (X - acc)^2, sum X^2}
  int* status;
  const int* run_flag;   // when non-null and 0 at launch: nothing to do
  const int* parts_flag; // parts = 3, non-null and 0 at launch: one term (hi x hi)
  const float* scale_m;  // optional per-row / per-column factors of the output
  const float* scale_n;  //   (MMA space), applied after alpha
  // FP8 block scales (MMA space): the product of K block kb in M tile tm is
  // scaled by bscale[tm * bs_sm + kb * bs_sk] before it is added; each K block
  // is accumulated in its own TMEM buffer and summed in the epilogue.
  const float* bscale;
  int bs_sm, bs_sk;
};

template <int KIND> struct KindCfg;
template <> struct KindCfg<0> {  // TF32 from FP32 storage
  static constexpr int esize = 4, bk = 32, kstep_rows = 8, box_mn = 32;
};
template <> struct KindCfg<1> {  // BF16
  static constexpr int esize = 2, bk = 64, kstep_rows = 16, box_mn = 64;
};
template <> struct KindCfg<2> {  // FP8 e4m3 (K-major operands only)
  static constexpr int esize = 1, bk = 128, kstep_rows = 32, box_mn = 128;
};
__host__ __device__ constexpr int kind_bk(int kind) { return kind == 0 ? 32 : (kind == 1 ? 64 : 128); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the status word set) if the phase never completes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status,
                                          volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  const uint64_t budget = *(volatile unsigned long long*)&g_wait_budget_ns;
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (now_ns() - t0 > budget) {
      *abort_flag = 1;
      if (status) atomicCAS(status, 0, (int)BCUR_ETIMEOUT);
      return false;
    }
  }
}
// 3-D tile load: (x inner, y outer, z batch).  x is always a multiple of
// 128 bytes here, so every copy starts 16-byte aligned.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
template <int KIND>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  if constexpr (KIND == 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else if constexpr (KIND == 1) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}
// 32 lanes x 32 consecutive 32-bit columns: thread t of the warp receives
// lane (quarter*32 + t), columns [col, col+32).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, 128-byte swizzle, sm_100 format.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version
  d |= (uint64_t)2 << 61;  // SWIZZLE_128B
  return d;
}

// Instruction descriptor: FP32 accumulate, A/B format, majors, N, M.
__host__ __device__ inline uint32_t idesc(int kind, int a_mn, int b_mn, int M, int N) {
  uint32_t d = 0;
  d |= 1u << 4;                          // D format F32
  const uint32_t fmt = kind == 0 ? 2u : (kind == 1 ? 1u : 0u);  // TF32 : BF16 : E4M3
  d |= fmt << 7;
  d |= fmt << 10;
  d |= (uint32_t)(a_mn & 1) << 15;
  d |= (uint32_t)(b_mn & 1) << 16;
  d |= (uint32_t)(N >> 3) << 17;
  d |= (uint32_t)(M >> 4) << 24;
  return d;
}

// Tensor maps of the operands: [0] = hi (or the only part), [1] = lo.
struct Maps {
  CUtensorMap a[2];
  CUtensorMap b[2];
};

// One GEMM of a grouped launch (128-byte aligned: the tensor maps need 64).
struct alignas(128) GEntry {
  Maps maps;
  Params p;
};
struct Group {
  const GEntry* e;     // device table, `count` entries
  const int* starts;   // device, count + 1 prefix sums of the entries' units
  int count, total;
  int* status;
};

struct Unit {
  int m0, n0, z, b, klo, khi, skip, uu;
};

// CTA c takes units c, c + G, c + 2G, ...  Odd full rounds are walked in
// reverse ("snake"), so with units ordered heaviest first every CTA gets a
// similar amount of work.
__device__ __forceinline__ int snake(int u, int total) {
  const int G = gridDim.x;
  const int round = u / G, c = u % G;
  const int full_rounds = total / G;
  return (round < full_rounds && (round & 1)) ? round * G + (G - 1 - c) : u;
}

// BF16 terms of a GEMM's products: the producer and the MMA issuer read the
// same flag (written by an earlier launch) and so agree on the K loop.
__device__ __forceinline__ int terms_of(const Params& p) {
  return (p.parts == 3 && p.parts_flag && *p.parts_flag == 0) ? 1 : p.parts;
}

template <int BN, int KIND>
__device__ __forceinline__ Unit decode_unit(const Params& p, int uu) {
  constexpr int BK = KindCfg<KIND>::bk;
  Unit w;
  w.uu = uu;
  const int bt = uu / p.ksplit;
  w.z = uu % p.ksplit;
  w.b = bt / (p.tiles_m * p.tiles_n);
  const int tile = bt % (p.tiles_m * p.tiles_n);
  // grouped raster: 16 M-tiles per group for L2 reuse of the B panel
  const int GM = 16;
  const int per_group = GM * p.tiles_n;
  const int g = tile / per_group;
  const int first = g * GM;
  const int gm = min(GM, p.tiles_m - first);
  const int r = tile % per_group;
  int tm = first + r % gm;
  int tn = r / gm;
  if (p.rev_m) tm = p.tiles_m - 1 - tm;  // heavier tiles (longer K range) first
  if (p.rev_n) tn = p.tiles_n - 1 - tn;
  w.m0 = tm * BM;
  w.n0 = tn * BN;
  const int chunk = (p.kblocks + p.ksplit - 1) / p.ksplit;
  w.klo = w.z * chunk;
  w.khi = min(p.kblocks, w.klo + chunk);
  if (p.triA == 1) w.khi = min(w.khi, (w.m0 + BM + BK - 1) / BK);
  if (p.triA == 2) w.klo = max(w.klo, w.m0 / BK);
  if (p.triB == 1) w.klo = max(w.klo, w.n0 / BK);
  if (p.triB == 2) w.khi = min(w.khi, (w.n0 + BN + BK - 1) / BK);
  w.skip = 0;
  if (p.tri_out == 1 && w.m0 + BM - 1 < w.n0) w.skip = 1;
  if (p.tri_out == 2 && w.n0 + BN - 1 < w.m0) w.skip = 1;
  if (p.run_flag && *p.run_flag == 0) w.skip = 1;
  return w;
}

// The GEMM a thread looked up last and its unit range: consecutive units of
// a CTA's walk usually belong to the same GEMM, so the search (a chain of
// dependent global loads) is only repeated when the walk leaves the range.
struct LocCache {
  int entry = -1, begin = 0, end = 0;
};

// Unit u of this CTA's walk -> the GEMM that owns it (its parameters and
// tensor maps) and the decoded tile.
template <int BN, int KIND, bool GROUPED>
__device__ __forceinline__ Unit locate(const Maps& maps, const Params& p, const Group& grp, int u,
                                       int total, const Params*& P, const Maps*& M,
                                       LocCache& lc) {
  const int uu = snake(u, total);
  if constexpr (!GROUPED) {
    P = &p;
    M = &maps;
    return decode_unit<BN, KIND>(p, uu);
  } else {
    if (uu < lc.begin || uu >= lc.end) {
      int lo = 0, hi = grp.count - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (grp.starts[mid] <= uu) lo = mid; else hi = mid - 1;
      }
      lc.entry = lo;
      lc.begin = grp.starts[lo];
      lc.end = grp.starts[lo + 1];
    }
    P = &grp.e[lc.entry].p;
    M = &grp.e[lc.entry].maps;
    return decode_unit<BN, KIND>(*P, uu - lc.begin);
  }
}

template <int BN, int EPI, bool G> struct StageCfg {
  static constexpr int kStageBBytes = BN * 128;
  static constexpr int kStageBytes = kStageABytes + kStageBBytes;
  // 192 KB of stages and one 32 x 36 transpose tile per epilogue warp (an
  // eight-warp residual keeps 160 KB of stages)
  static constexpr int kStages = (epi_warps<EPI, G>() == 8 ? 163840 : 196608) / kStageBytes;
  static constexpr int kTmemCols = 2 * BN;
  static constexpr int kStageOut = epi_warps<EPI, G>() * 32 * 36 * 4;
  static constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 512 + kStageOut;
};

template <int BN, int KIND, int EPI, bool GROUPED>
__global__ void __launch_bounds__(threads_of<EPI, GROUPED>(), 1)
    tc_gemm_kernel(const __grid_constant__ Maps maps, const __grid_constant__ Params p,
                   const Group grp) {
  using SC = StageCfg<BN, EPI, GROUPED>;
  using KC = KindCfg<KIND>;
  constexpr int S = SC::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * SC::kStageBytes);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* red = reinterpret_cast<double*>(tmem_slot + 4);  // 2 per epilogue warp
  float* stage_out = reinterpret_cast<float*>(smem + S * SC::kStageBytes + 512);
  constexpr int EW = epi_warps<EPI, GROUPED>();
  int* const status = GROUPED ? grp.status : p.status;
  if constexpr (!GROUPED) {
    if (p.run_flag && *p.run_flag == 0) return;  // uniform: the whole CTA leaves
  }

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], EW);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if constexpr (!GROUPED) {
      for (int i = 0; i < 2; ++i) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.a[i])) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.b[i])) : "memory");
      }
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)SC::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int total = GROUPED ? grp.total : p.tiles_m * p.tiles_n * p.ksplit * p.batch;
  constexpr int BKR = KC::bk;  // K rows per stage for an MN-major operand

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      const Maps* last = nullptr;
      LocCache lcache;
      for (int u = blockIdx.x; u < total && ok; u += gridDim.x) {
        const Params* P;
        const Maps* M;
        const Unit w = locate<BN, KIND, GROUPED>(maps, p, grp, u, total, P, M, lcache);
        if (w.skip || w.klo >= w.khi) continue;
        if constexpr (GROUPED) {
          if (M != last) {  // maps written by the host into global memory
#pragma unroll
            for (int i = 0; i < 2; ++i) {
              asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(
                               reinterpret_cast<uint64_t>(&M->a[i]))
                           : "memory");
              asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(
                               reinterpret_cast<uint64_t>(&M->b[i]))
                           : "memory");
            }
            last = M;
          }
        }
        const int parts = terms_of(*P), a_mn = P->a_mn, b_mn = P->b_mn;
        const int n_it = (w.khi - w.klo) * parts;
        for (int i = 0; i < n_it; ++i, ++it) {
          const int kb = w.klo + i / parts, part = i % parts;
          const CUtensorMap* ma = &M->a[part == 2 ? 1 : 0];
          const CUtensorMap* mb = &M->b[part == 1 ? 1 : 0];
          const uint32_t stage = it % S, round = it / S;
          if (!mbar_wait(&empty[stage], (round & 1) ^ 1, status, abort_flag)) { ok = false; break; }
          uint8_t* sa = smem + stage * SC::kStageBytes;
          uint8_t* sb = sa + kStageABytes;
          mbar_expect_tx(&full[stage], SC::kStageBytes);
          if (!a_mn) {
            tma_load_3d(sa, ma, &full[stage], kb * KC::bk, w.m0, w.b);
          } else {
#pragma unroll
            for (int b = 0; b < BM / KC::box_mn; ++b)
              tma_load_3d(sa + b * (BKR * 128), ma, &full[stage], w.m0 + b * KC::box_mn, kb * BKR, w.b);
          }
          if (!b_mn) {
            tma_load_3d(sb, mb, &full[stage], kb * KC::bk, w.n0, w.b);
          } else {
#pragma unroll
            for (int b = 0; b < BN / KC::box_mn; ++b)
              tma_load_3d(sb + b * (BKR * 128), mb, &full[stage], w.n0 + b * KC::box_mn, kb * BKR, w.b);
          }
        }
      }
      // Drain: the last load issued on each stage must have landed before exit.
      const uint32_t n_last = it < (uint32_t)S ? it : (uint32_t)S;
      for (uint32_t j = 0; j < n_last; ++j) {
        const uint32_t i2 = it - 1 - j;
        const uint32_t stage = i2 % S, round = i2 / S;
        const uint64_t t0 = now_ns();
        while (!mbar_try_wait(&full[stage], round & 1) && now_ns() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t it = 0, tu = 0;
      bool ok = true;
      LocCache lcache;
      for (int u = blockIdx.x; u < total && ok; u += gridDim.x) {
        const Params* P;
        const Maps* M;
        const Unit w = locate<BN, KIND, GROUPED>(maps, p, grp, u, total, P, M, lcache);
        if (w.skip || w.klo >= w.khi) continue;
        const int parts = terms_of(*P), a_mn = P->a_mn, b_mn = P->b_mn;
        const uint32_t id = idesc(KIND, a_mn, b_mn, BM, BN);
        if constexpr (KIND == 2 && BN <= 128 && EPI == EPI_STORE && !GROUPED) {
          if (P->bscale) {
            // one K block (one stage) per TMEM buffer, each handed to the
            // epilogue on its own
            for (int i = 0; i < w.khi - w.klo; ++i, ++it) {
              const uint32_t acc = tu & 1, use = tu >> 1;
              if (!mbar_wait(&tempty[acc], (use & 1) ^ 1, status, abort_flag)) { ok = false; break; }
              tc_fence_after();
              const uint32_t stage = it % S, round = it / S;
              if (!mbar_wait(&full[stage], round & 1, status, abort_flag)) { ok = false; break; }
              tc_fence_after();
              const uint32_t sa = smem_u32(smem + stage * SC::kStageBytes);
              const uint32_t sb = sa + kStageABytes;
#pragma unroll
              for (int j = 0; j < 4; ++j)
                tc_mma<KIND>(tmem_base + acc * BN, sdesc(sa + j * 32, 16, 1024),
                             sdesc(sb + j * 32, 16, 1024), id, j > 0 ? 1u : 0u);
              tc_commit(&empty[stage]);
              tc_commit(&tfull[acc]);
              ++tu;
            }
            if (!ok) break;
            continue;
          }
        }
        const uint32_t acc = tu & 1, use = tu >> 1;
        if (!mbar_wait(&tempty[acc], (use & 1) ^ 1, status, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * BN;
        const int n_it = (w.khi - w.klo) * parts;
        for (int i = 0; i < n_it; ++i, ++it) {
          const uint32_t stage = it % S, round = it / S;
          if (!mbar_wait(&full[stage], round & 1, status, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * SC::kStageBytes);
          const uint32_t sb = sa + kStageABytes;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint64_t ad = a_mn ? sdesc(sa + j * KC::kstep_rows * 128, BKR * 128, 1024)
                                     : sdesc(sa + j * 32, 16, 1024);
            const uint64_t bd = b_mn ? sdesc(sb + j * KC::kstep_rows * 128, BKR * 128, 1024)
                                     : sdesc(sb + j * 32, 16, 1024);
            tc_mma<KIND>(d_tmem, ad, bd, id, (i > 0 || j > 0) ? 1u : 0u);
          }
          tc_commit(&empty[stage]);
        }
        if (!ok) break;
        tc_commit(&tfull[acc]);
        ++tu;
      }
      // All MMAs this thread issued complete before TMEM is released.
      tc_commit(done);
      const uint64_t t0 = now_ns();
      while (!mbar_try_wait(done, 0) && now_ns() - t0 < kWaitNs) {
      }
    }
  } else if constexpr (EPI == EPI_RESID) {
    // ---------------- residual epilogue (warps 2..9) ----------------
    // sum (X - alpha acc)^2 and sum X^2.  X is read coalesced: a lane loads
    // four consecutive floats, eight lanes one 128-byte row piece, a warp four
    // rows per instruction.  The accumulator chunk (lane = row in TMEM) is
    // brought into the same layout through a per-warp 32 x 36 shared tile.
    // The X loads of two chunks are issued before their accumulators are read.
    const int ew = warp - 2;
    const int quarter = warp & 3;  // TMEM lanes [32*quarter, 32*quarter + 32)
    constexpr int CW = BN / (EW / 4);  // columns per warp
    const int cbeg = (ew / 4) * CW;
    float* tile = stage_out + ew * (32 * 36);
    const int lr = lane >> 3, lc = (lane & 7) * 4;  // first row, column of this lane
    double e2 = 0.0, x2 = 0.0;
    uint32_t tu = 0;
    bool ok = true;
    LocCache lcache;
    for (int u = blockIdx.x; u < total && ok; u += gridDim.x) {
      const Params* P;
      const Maps* M;
      const Unit w = locate<BN, KIND, GROUPED>(maps, p, grp, u, total, P, M, lcache);
      if (w.skip) continue;
      const bool has_acc = w.klo < w.khi;
      const uint32_t acc = tu & 1, use = tu >> 1;
      const int Mm = P->Mm, Nm = P->Nm;
      const float alpha = P->alpha;
      const int64_t ldx = P->ldx;
      const int rbase = w.m0 + quarter * 32;
      const float* const Xp = P->X;
      const bool vec_ok = ((reinterpret_cast<uintptr_t>(Xp) & 15) == 0) && (ldx % 4 == 0);
      const bool whole = vec_ok && rbase + 32 <= Mm && w.n0 + cbeg + CW <= Nm;
      if (whole && lc == 0) {
        // X does not depend on the MMA: while the accumulator is still being
        // formed, ask L2 for every 128-byte row piece this warp will read
        // (one lane per piece, no registers held).
        const float* xr = Xp + (int64_t)(rbase + lr) * ldx + w.n0 + cbeg;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          for (int c = 0; c < CW; c += 32)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(xr + 4 * i * ldx + c));
      }
      if (has_acc) {
        // every lane polls; the warp goes on only if all of them saw the
        // phase (the tcgen05.ld and shuffles below need the whole warp)
        const bool got = mbar_wait(&tfull[acc], use & 1, status, abort_flag);
        if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
        tc_fence_after();
      }
      // rows rbase + lr + 4 i (i < 8), columns col0 + lc .. + 3
      auto load_x = [&](float4 (&xv)[8], int col0) {
        const int col = col0 + lc;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int row = rbase + lr + 4 * i;
          float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
          if (row < Mm) {
            const float* xr = Xp + (int64_t)row * ldx + col;
            // read once: stream past L1 so the GEMM table and parameters stay cached
            if (vec_ok && col + 4 <= Nm) {
              q = __ldcs(reinterpret_cast<const float4*>(xr));
            } else {
              if (col < Nm) q.x = __ldcs(xr);
              if (col + 1 < Nm) q.y = __ldcs(xr + 1);
              if (col + 2 < Nm) q.z = __ldcs(xr + 2);
              if (col + 3 < Nm) q.w = __ldcs(xr + 3);
            }
          }
          xv[i] = q;
        }
      };
      // accumulator chunk [c, c+32) of this warp's rows, in the X layout
      auto read_acc = [&](float4 (&av)[8], int c) {
        float v[32];
        __syncwarp();  // tcgen05.ld is warp-aligned: reconverge before it
        if (has_acc) {
          tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * BN + c, v);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(&tile[lane * 36 + 4 * q]) =
              make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 8; ++i)
          av[i] = *reinterpret_cast<const float4*>(&tile[(lr + 4 * i) * 36 + lc]);
        __syncwarp();
      };
      auto reduce = [&](const float4 (&xv)[8], const float4 (&av)[8], int col0) {
        const int col = col0 + lc;
        float se = 0.f, sx = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int row = rbase + lr + 4 * i;
          const bool rok = row < Mm;
          const float xs[4] = {xv[i].x, xv[i].y, xv[i].z, xv[i].w};
          const float as[4] = {av[i].x, av[i].y, av[i].z, av[i].w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float d = xs[j] - ((rok && col + j < Nm) ? alpha * as[j] : 0.f);
            se = fmaf(d, d, se);
            sx = fmaf(xs[j], xs[j], sx);
          }
        }
        e2 += (double)se;
        x2 += (double)sx;
      };
      // A whole tile (every row and column inside X, X 16-byte aligned) takes
      // the short path: one pointer per lane, no masks, d = x - alpha a by
      // one FMA, FP32 sums over the warp's share of the tile.
      if (whole) {
        const float* xl = Xp + (int64_t)(rbase + lr) * ldx + w.n0 + lc;
        const int64_t st4 = 4 * ldx;
        auto load_w = [&](float4 (&xv)[8], int c) {
#pragma unroll
          for (int i = 0; i < 8; ++i) xv[i] = __ldcs(reinterpret_cast<const float4*>(xl + i * st4 + c));
        };
        float se = 0.f, sx = 0.f;
        auto reduce_w = [&](const float4 (&xv)[8], const float4 (&av)[8]) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float xs[4] = {xv[i].x, xv[i].y, xv[i].z, xv[i].w};
            const float as[4] = {av[i].x, av[i].y, av[i].z, av[i].w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float d = fmaf(-alpha, as[j], xs[j]);
              se = fmaf(d, d, se);
              sx = fmaf(xs[j], xs[j], sx);
            }
          }
        };
#pragma unroll 1
        for (int c = cbeg; c < cbeg + CW; c += 64) {
          float4 xa[8], aa[8];
          if constexpr (CW >= 64) {
            float4 xb[8];
            load_w(xa, c);
            load_w(xb, c + 32);
            read_acc(aa, c);
            reduce_w(xa, aa);
            read_acc(aa, c + 32);
            reduce_w(xb, aa);
          } else {
            load_w(xa, c);
            read_acc(aa, c);
            reduce_w(xa, aa);
          }
        }
        e2 += (double)se;
        x2 += (double)sx;
      }
#pragma unroll 1
      for (int c = cbeg; !whole && c < cbeg + CW; c += 64) {
        float4 xa[8], aa[8];
        if constexpr (CW >= 64) {
          float4 xb[8];
          load_x(xa, w.n0 + c);
          load_x(xb, w.n0 + c + 32);
          read_acc(aa, c);
          reduce(xa, aa, w.n0 + c);
          read_acc(aa, c + 32);
          reduce(xb, aa, w.n0 + c + 32);
        } else {
          load_x(xa, w.n0 + c);
          read_acc(aa, c);
          reduce(xa, aa, w.n0 + c);
        }
      }
      if (has_acc) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[acc]);
        ++tu;
      }
      if constexpr (GROUPED) {
        // One partial pair per (tile, epilogue warp): the owning GEMM's sums
        // do not depend on which CTA ran the tile or what else was in the
        // launch.
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          e2 += __shfl_xor_sync(0xffffffffu, e2, o);
          x2 += __shfl_xor_sync(0xffffffffu, x2, o);
        }
        if (lane == 0) {
          P->partials[2 * (kResidSlots * (int64_t)w.uu + ew)] = e2;
          P->partials[2 * (kResidSlots * (int64_t)w.uu + ew) + 1] = x2;
          for (int sl = ew + EW; sl < kResidSlots; sl += EW) {  // slots no warp uses
            P->partials[2 * (kResidSlots * (int64_t)w.uu + sl)] = 0.0;
            P->partials[2 * (kResidSlots * (int64_t)w.uu + sl) + 1] = 0.0;
          }
        }
        e2 = 0.0;
        x2 = 0.0;
      }
    }
    if constexpr (!GROUPED) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        x2 += __shfl_xor_sync(0xffffffffu, x2, o);
      }
      if (lane == 0) {
        red[2 * ew] = e2;
        red[2 * ew + 1] = x2;
      }
    }
  } else {
    // ---------------- store epilogue (warps 2..5) ----------------
    const int quarter = warp & 3;  // TMEM lanes [32*quarter, 32*quarter + 32)
    uint32_t tu = 0;
    bool ok = true;
    LocCache lcache;
    for (int u = blockIdx.x; u < total && ok; u += gridDim.x) {
      const Params* P;
      const Maps* M;
      const Unit w = locate<BN, KIND, GROUPED>(maps, p, grp, u, total, P, M, lcache);
      if (w.skip) continue;
      if constexpr (KIND == 2 && BN <= 128 && EPI == EPI_STORE && !GROUPED) {
        if (P->bscale) {
          // block-scaled FP8: acc += scale(tile, kb) * (the K block's product),
          // in registers; each TMEM buffer is released as soon as it is read
          float racc[BN];
#pragma unroll
          for (int i = 0; i < BN; ++i) racc[i] = 0.f;
          const int64_t tm = w.m0 / BM;
          bool good = true;
          for (int i = 0; i < w.khi - w.klo; ++i) {
            const uint32_t a2 = tu & 1, u2 = tu >> 1;
            const bool got = mbar_wait(&tfull[a2], u2 & 1, status, abort_flag);
            if (!__all_sync(0xffffffffu, got)) { good = false; break; }
            tc_fence_after();
            const float sc = P->bscale[tm * P->bs_sm + (int64_t)(w.klo + i) * P->bs_sk];
#pragma unroll
            for (int c = 0; c < BN / 32; ++c) {
              float v[32];
              __syncwarp();
              tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + a2 * BN + c * 32, v);
#pragma unroll
              for (int j = 0; j < 32; ++j) racc[c * 32 + j] = fmaf(sc, v[j], racc[c * 32 + j]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[a2]);
            ++tu;
          }
          if (!good) { ok = false; break; }
          // D^T (the block-scaled product runs transposed): lane = row
          const int row = w.m0 + quarter * 32 + lane;
          if (row < P->Mm) {
            const int Nm = P->Nm;
            const int64_t ldd = P->ldd;
            const float f = P->alpha * (P->scale_m ? P->scale_m[row] : 1.f);
            const float* const sn = P->scale_n;
            float* const Dp = P->D + (int64_t)w.b * P->sD;
#pragma unroll
            for (int i = 0; i < BN; ++i) {
              const int col = w.n0 + i;
              if (col < Nm) Dp[(int64_t)col * ldd + row] = f * racc[i] * (sn ? sn[col] : 1.f);
            }
          }
          continue;
        }
      }
      const bool has_acc = w.klo < w.khi;
      const uint32_t acc = tu & 1, use = tu >> 1;
      if (has_acc) {
        const bool got = mbar_wait(&tfull[acc], use & 1, status, abort_flag);
        if (!__all_sync(0xffffffffu, got)) { ok = false; break; }  // warp-uniform, as above
        tc_fence_after();
      }
      const int Mm = P->Mm, Nm = P->Nm;
      const int row = w.m0 + quarter * 32 + lane;
      const bool row_ok = row < Mm;
      const float alpha = P->alpha, beta = P->beta;
      const int tri_out = P->tri_out;
      const int64_t ldd = P->ldd;
      // Every parameter the chunk loop needs is read here, once per tile: P
      // points into parameter (or table) memory that the compiler cannot tell
      // apart from D, so a read inside the loop would be repeated after every
      // store and serialise the row loop on its latency.
      const int transD = P->transD;
      const float* const scale_m = P->scale_m;
      const float* const scale_n = P->scale_n;
      float* const Dp = P->D ? P->D + (int64_t)w.b * P->sD : nullptr;
      __nv_bfloat16* const Dhp = P->Dh ? P->Dh + (int64_t)w.b * P->sD : nullptr;
      __nv_bfloat16* const Dlp = P->Dl ? P->Dl + (int64_t)w.b * P->sD : nullptr;
      const float sm_lane = (scale_m && row_ok) ? scale_m[row] : 1.f;  // row scale of this lane
      // four-wide stores need 16-byte rows (8-byte for the BF16 pair)
      const bool vec_ok = (ldd % 4 == 0) && ((reinterpret_cast<uintptr_t>(Dp) & 15) == 0) &&
                          ((reinterpret_cast<uintptr_t>(Dhp) & 7) == 0) &&
                          ((reinterpret_cast<uintptr_t>(Dlp) & 7) == 0);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        __syncwarp();  // tcgen05.ld is warp-aligned: reconverge before it
        if (has_acc) {
          tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * BN + c0, v);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = 0.f;
        }
        const int col0 = w.n0 + c0;
        if (col0 >= Nm) continue;
        if constexpr (EPI == EPI_STORE) {
          constexpr unsigned FULL = 0xffffffffu;
          // alpha and the scales are applied while the warp is converged (the
          // scale of the other index is shuffled), and the old values of D are
          // loaded before the first store.
          const float sn_lane = (scale_n && col0 + lane < Nm) ? scale_n[col0 + lane] : 1.f;
          if (transD) {
            // D^T: lane = row, consecutive lanes write consecutive addresses.
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              float o = alpha * v[i];
              if (scale_m) o *= sm_lane;
              if (scale_n) o *= __shfl_sync(FULL, sn_lane, i);
              v[i] = o;
            }
            if (!row_ok) continue;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const int col = col0 + i;
              if (col >= Nm) break;
              if (tri_out == 1 && row < col) continue;
              if (tri_out == 2 && row > col) continue;
              const int64_t off = (int64_t)col * ldd + row;
              float o = v[i];
              if (beta != 0.f) o = fmaf(beta, Dp[off], o);
              if (Dp) Dp[off] = o;
              if (Dhp) {
                const __nv_bfloat16 h = __float2bfloat16_rn(o);
                Dhp[off] = h;
                if (Dlp) Dlp[off] = __float2bfloat16_rn(o - __bfloat162float(h));
              }
            }
          } else {
            // Row-major D: the 32 x 32 chunk goes through a per-warp 32 x 36
            // shared tile (t[row * 36 + col]).  A chunk that is whole (inside
            // D, and wholly on the kept side of the diagonal) is written four
            // columns per lane: lane (lr, lc) takes columns lc..lc+3 of rows
            // lr + 4 i, so each store instruction writes four 128-byte row
            // pieces (a quarter of the instructions of one column per lane,
            // which is what bounds a short-K tile).  Other chunks: one column
            // per lane with per-element masks.
            float* t = stage_out + (warp - 2) * (32 * 36);
#pragma unroll
            for (int q = 0; q < 8; ++q)
              *reinterpret_cast<float4*>(&t[lane * 36 + 4 * q]) =
                  make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            __syncwarp();
            const int rbase = w.m0 + quarter * 32;
            const bool whole = vec_ok && rbase + 32 <= Mm && col0 + 32 <= Nm &&
                               (tri_out == 0 || (tri_out == 1 && rbase >= col0 + 31) ||
                                (tri_out == 2 && rbase + 31 <= col0));
            if (whole) {
              const int lr = lane >> 3, lc = (lane & 7) * 4;
              const int col = col0 + lc;
              float4 a[8];
#pragma unroll
              for (int i = 0; i < 8; ++i)
                a[i] = *reinterpret_cast<const float4*>(&t[(lr + 4 * i) * 36 + lc]);
              float sn[4] = {1.f, 1.f, 1.f, 1.f};
              if (scale_n)
#pragma unroll
                for (int j = 0; j < 4; ++j) sn[j] = scale_n[col + j];
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const float sm = scale_m ? scale_m[rbase + lr + 4 * i] : 1.f;
                float* e = &a[i].x;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  float o = alpha * e[j];
                  if (scale_m) o *= sm;
                  if (scale_n) o *= sn[j];
                  e[j] = o;
                }
              }
              if (beta != 0.f) {  // all loads issued before any store
                float4 old[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                  old[i] = *reinterpret_cast<const float4*>(
                      Dp + (int64_t)(rbase + lr + 4 * i) * ldd + col);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                  a[i].x = fmaf(beta, old[i].x, a[i].x);
                  a[i].y = fmaf(beta, old[i].y, a[i].y);
                  a[i].z = fmaf(beta, old[i].z, a[i].z);
                  a[i].w = fmaf(beta, old[i].w, a[i].w);
                }
              }
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const int64_t off = (int64_t)(rbase + lr + 4 * i) * ldd + col;
                if (Dp) *reinterpret_cast<float4*>(Dp + off) = a[i];
                if (Dhp) {
                  const float* e = &a[i].x;
                  __nv_bfloat16 h[4], l[4];
#pragma unroll
                  for (int j = 0; j < 4; ++j) {
                    h[j] = __float2bfloat16_rn(e[j]);
                    l[j] = __float2bfloat16_rn(e[j] - __bfloat162float(h[j]));
                  }
                  *reinterpret_cast<uint2*>(Dhp + off) = *reinterpret_cast<const uint2*>(h);
                  if (Dlp) *reinterpret_cast<uint2*>(Dlp + off) = *reinterpret_cast<const uint2*>(l);
                }
              }
            } else {
              const int col = col0 + lane;
              const bool col_ok = col < Nm;
#pragma unroll
              for (int r = 0; r < 32; ++r) {
                const int grow = rbase + r;
                bool ok = col_ok && grow < Mm;
                if (tri_out == 1 && grow < col) ok = false;
                if (tri_out == 2 && grow > col) ok = false;
                float o = alpha * t[r * 36 + lane];  // row rbase + r, column col
                if (scale_m) o *= __shfl_sync(FULL, sm_lane, r);
                if (scale_n) o *= sn_lane;
                if (ok) {
                  const int64_t off = (int64_t)grow * ldd + col;
                  if (beta != 0.f) o = fmaf(beta, Dp[off], o);
                  if (Dp) Dp[off] = o;
                  if (Dhp) {
                    const __nv_bfloat16 h = __float2bfloat16_rn(o);
                    Dhp[off] = h;
                    if (Dlp) Dlp[off] = __float2bfloat16_rn(o - __bfloat162float(h));
                  }
                }
              }
            }
            __syncwarp();
          }
        } else if constexpr (EPI == EPI_PARTIAL) {
          if (!row_ok) continue;
          float* prow = P->part + (int64_t)w.z * Mm * Nm + (int64_t)row * Nm;
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int col = col0 + i;
            if (col >= Nm) break;
            prow[col] = v[i];
          }
        }
      }
      if (has_acc) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[acc]);
        ++tu;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (EPI == EPI_RESID && !GROUPED) {
    if (threadIdx.x == 0) {
      double se = 0.0, sx = 0.0;
      for (int i = 0; i < EW; ++i) { se += red[2 * i]; sx += red[2 * i + 1]; }
      p.partials[2 * blockIdx.x] = se;
      p.partials[2 * blockIdx.x + 1] = sx;
    }
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"((uint32_t)SC::kTmemCols)
                 : "memory");
  }
}

// Sum the split-K slices in a fixed order and apply alpha / beta / layout.
__global__ void splitk_reduce_kernel(Params p) {
  if (p.run_flag && *p.run_flag == 0) return;
  const int64_t total = (int64_t)p.Mm * p.Nm;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / p.Nm), col = (int)(e % p.Nm);
    if (p.tri_out == 1 && row < col) continue;
    if (p.tri_out == 2 && row > col) continue;
    float s = 0.f;
    for (int z = 0; z < p.ksplit; ++z) s += p.part[(int64_t)z * total + e];
    const int64_t off = p.transD ? (int64_t)col * p.ldd + row : (int64_t)row * p.ldd + col;
    float o = p.alpha * s;
    if (p.beta != 0.f) o = fmaf(p.beta, p.D[off], o);
    if (p.D) p.D[off] = o;
    if (p.Dh) {
      const __nv_bfloat16 h = __float2bfloat16_rn(o);
      p.Dh[off] = h;
      if (p.Dl) p.Dl[off] = __float2bfloat16_rn(o - __bfloat162float(h));
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    else
      cudaGetLastError();
  });
  return fn;
}

int sm_count() {
  static int n = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      v = 148;
    }
    n = v;
  });
  return n;
}

bool tc_device_ok() {
  static int ok = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) == cudaSuccess)
      ok = (major == 10 && minor == 3) ? 1 : 0;
    else
      cudaGetLastError();
  });
  return ok == 1 && encode_fn() != nullptr;
}

// Operand in MMA space: rows = MN index when K-major (inner dim K), or
// rows = K index when MN-major (inner dim MN).
struct Operand {
  const void* ptr;
  int64_t ld;      // elements between consecutive outer-dimension entries
  int mn_major;
  int64_t mn, k;   // extents
};

bool make_map(CUtensorMap* map, const Operand& op, int kind, int box_rows_mn, int batch,
              int64_t sbatch) {
  const int esize = kind == 0 ? 4 : (kind == 1 ? 2 : 1);
  const int box_inner = 128 / esize;  // 128 bytes
  const uintptr_t a = reinterpret_cast<uintptr_t>(op.ptr);
  if (a % 16 != 0 || (op.ld * esize) % 16 != 0) return false;
  cuuint64_t dims[3];
  const int64_t outer = op.mn_major ? op.k : op.mn;
  const int64_t bstride = batch > 1 ? sbatch : op.ld * outer;
  if ((bstride * esize) % 16 != 0) return false;
  cuuint64_t strides[2] = {(cuuint64_t)(op.ld * esize), (cuuint64_t)(bstride * esize)};
  cuuint32_t box[3];
  cuuint32_t estr[3] = {1, 1, 1};
  dims[2] = (cuuint64_t)batch;
  box[2] = 1;
  if (!op.mn_major) {
    dims[0] = (cuuint64_t)op.k;
    dims[1] = (cuuint64_t)op.mn;
    box[0] = (cuuint32_t)box_inner;
    box[1] = (cuuint32_t)box_rows_mn;  // MN rows of the tile
  } else {
    dims[0] = (cuuint64_t)op.mn;
    dims[1] = (cuuint64_t)op.k;
    box[0] = (cuuint32_t)box_inner;   // MN elements per box
    box[1] = (cuuint32_t)kind_bk(kind);  // K rows per stage
  }
  if (op.ld < (int64_t)dims[0]) return false;
  auto fn = encode_fn();
  if (!fn) return false;
  CUresult r = fn(map, kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                            : (kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                         : CU_TENSOR_MAP_DATA_TYPE_UINT8),
                  3, const_cast<void*>(op.ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, int KIND, int EPI, bool GROUPED>
bcur_status_t launch_inst(const Maps& maps, const Params& p, const Group& grp, int grid,
                          cudaStream_t s) {
  using SC = StageCfg<BN, EPI, GROUPED>;
  static bool attr = false;
  if (!attr) {
    BCUR_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<BN, KIND, EPI, GROUPED>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SC::kSmemBytes));
    attr = true;
  }
  tc_gemm_kernel<BN, KIND, EPI, GROUPED><<<grid, threads_of<EPI, GROUPED>(), SC::kSmemBytes, s>>>(maps, p,
                                                                                     grp);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

template <int KIND, int EPI, bool GROUPED = false>
bcur_status_t launch_bn(int BN, const Maps& maps, const Params& p, int grid, cudaStream_t s,
                        const Group& grp = Group{}) {
  switch (BN) {
    case 64: return launch_inst<64, KIND, EPI, GROUPED>(maps, p, grp, grid, s);
    case 128: return launch_inst<128, KIND, EPI, GROUPED>(maps, p, grp, grid, s);
    case 256: return launch_inst<256, KIND, EPI, GROUPED>(maps, p, grp, grid, s);
  }
  return BCUR_EINVAL;
}

// Map one GEMM (GemmDesc convention, D row-major M x N) onto MMA space: the
// operands' tensor maps and the kernel parameters for tile width BN (0:
// chosen from the output width).  Split-K is not decided here.  Returns
// ENOTSUP if the operands cannot be described by TMA (alignment) or the
// device is not sm_103.
struct Prepared {
  Maps maps;
  Params p;
  int BN, kind;
};

// BCUR_DEBUG=1 in the environment: report why a GEMM is refused (stderr).
bool debug_on() {
  static const bool on = [] {
    const char* e = getenv("BCUR_DEBUG");
    return e && e[0] == '1';
  }();
  return on;
}

bcur_status_t prepare(const GemmDesc& d, int prec, int epi, int BN_force, Prepared* out) {
  // TF32 reads FP32 storage; BF16 / FP8 need that storage for both operands.
  if (!((prec == BCUR_TF32 && !d.ab_bf16 && !d.ab_fp8) ||
        (prec == BCUR_BF16 && d.ab_bf16 && !d.ab_fp8) || (prec == BCUR_FP8 && d.ab_fp8)))
    return BCUR_ENOTSUP;
  if (!tc_device_ok()) {
    if (debug_on()) fprintf(stderr, "bcur: tensor cores unavailable\n");
    return BCUR_ENOTSUP;
  }
  if (d.K <= 0 || d.M > INT32_MAX || d.N > INT32_MAX || d.K > INT32_MAX) {
    if (debug_on()) fprintf(stderr, "bcur: GEMM %lld x %lld x %lld out of range\n",
                            (long long)d.M, (long long)d.N, (long long)d.K);
    return BCUR_ENOTSUP;
  }
  if (d.ksplit > 1) return BCUR_ENOTSUP;
  const int kind = d.ab_fp8 ? 2 : (d.ab_bf16 ? 1 : 0);
  const int parts = d.parts == 3 ? 3 : 1;
  if (parts == 3 && (kind != 1 || !d.A_lo || !d.B_lo)) return BCUR_EINVAL;
  if (kind == 2 && epi != EPI_STORE) return BCUR_ENOTSUP;
  // Small M with a long N: compute D^T = B_op^T A_op^T so the long dimension
  // runs along the 128-row MMA tile and D is stored transposed.
  const bool swap = (epi == EPI_STORE) && d.M < 128 && d.N >= 2 * d.M;
  Operand A, B, Al, Bl;  // MMA-space A (Mm x K) and B (Nm x K), hi and lo
  int64_t Mm, Nm;
  int triA, triB, tri_out = d.out_lower ? 1 : 0;
  if (!swap) {
    Mm = d.M; Nm = d.N;
    A = {d.A, d.lda, d.transA ? 1 : 0, d.M, d.K};
    B = {d.B, d.ldb, d.transB ? 0 : 1, d.N, d.K};
    Al = {d.A_lo ? d.A_lo : d.A, d.lda, d.transA ? 1 : 0, d.M, d.K};
    Bl = {d.B_lo ? d.B_lo : d.B, d.ldb, d.transB ? 0 : 1, d.N, d.K};
    triA = d.triA;
    triB = d.triB;
  } else {
    Mm = d.N; Nm = d.M;
    A = {d.B, d.ldb, d.transB ? 0 : 1, d.N, d.K};
    B = {d.A, d.lda, d.transA ? 1 : 0, d.M, d.K};
    Al = {d.B_lo ? d.B_lo : d.B, d.ldb, d.transB ? 0 : 1, d.N, d.K};
    Bl = {d.A_lo ? d.A_lo : d.A, d.lda, d.transA ? 1 : 0, d.M, d.K};
    triA = d.triB == 1 ? 2 : (d.triB == 2 ? 1 : 0);
    triB = d.triA == 1 ? 2 : (d.triA == 2 ? 1 : 0);
    if (tri_out) tri_out = 2;
  }
  // TF32 operands must be K-major on this tensor core; FP8 is used K-major only.
  if (kind != 1 && (A.mn_major || B.mn_major)) return BCUR_ENOTSUP;
  const int BN = BN_force ? BN_force : (Nm <= 64 ? 64 : (Nm <= 128 ? 128 : 256));
  const int batch = d.batch > 1 ? d.batch : 1;
  const int64_t sAm = swap ? d.sB : d.sA, sBm = swap ? d.sA : d.sB;
  Maps& maps = out->maps;
  if (!make_map(&maps.a[0], A, kind, BM, batch, sAm) || !make_map(&maps.b[0], B, kind, BN, batch, sBm) ||
      !make_map(&maps.a[1], Al, kind, BM, batch, sAm) || !make_map(&maps.b[1], Bl, kind, BN, batch, sBm)) {
    if (debug_on())
      fprintf(stderr, "bcur: no tensor map for GEMM %lld x %lld x %lld (A %p ld %lld mn %d, B %p ld %lld mn %d)\n",
              (long long)d.M, (long long)d.N, (long long)d.K, A.ptr, (long long)A.ld, A.mn_major,
              B.ptr, (long long)B.ld, B.mn_major);
    return BCUR_ENOTSUP;
  }
  Params& p = out->p;
  p = Params{};
  p.Mm = (int)Mm; p.Nm = (int)Nm; p.K = (int)d.K;
  p.parts = parts;
  p.batch = batch;
  p.sD = d.sD;
  p.Dh = (__nv_bfloat16*)d.Dh;
  p.Dl = (__nv_bfloat16*)d.Dl;
  p.a_mn = A.mn_major; p.b_mn = B.mn_major;
  p.tiles_m = (int)ceil_div(Mm, BM);
  p.tiles_n = (int)ceil_div(Nm, BN);
  p.kblocks = (int)ceil_div(d.K, kind_bk(kind));
  p.triA = triA; p.triB = triB; p.tri_out = tri_out;
  p.rev_m = (triA == 1 || tri_out == 1) ? 1 : 0;
  p.rev_n = (triB == 2 || tri_out == 2) ? 1 : 0;
  p.alpha = (float)d.alpha; p.beta = (float)d.beta;
  p.D = (float*)d.D; p.ldd = d.ldd; p.transD = swap ? 1 : 0;
  p.X = (const float*)d.X; p.ldx = d.ldx; p.partials = d.partials;
  p.status = d.status;
  p.run_flag = d.run_flag;
  p.parts_flag = parts == 3 ? d.parts_flag : nullptr;
  p.scale_m = swap ? d.scale_n : d.scale_m;
  p.scale_n = swap ? d.scale_m : d.scale_n;
  p.ksplit = 1;
  if (d.bscale_b) {
    // op(B) becomes the MMA's A operand (128-row tiles = its 128-row blocks)
    // and a stage holds one 128-deep K block of e4m3
    if (kind != 2 || epi != EPI_STORE || !swap || BN > 128 || !d.D || d.Dh || d.Dl ||
        d.beta != 0.0 || tri_out || batch != 1 || d.bs_n > INT32_MAX || d.bs_k > INT32_MAX)
      return BCUR_ENOTSUP;
    p.bscale = d.bscale_b;
    p.bs_sm = (int)d.bs_n;
    p.bs_sk = (int)d.bs_k;
  }
  out->BN = BN;
  out->kind = kind;
  return BCUR_OK;
}

// Launch one GEMM.  `epi` selects store or residual.
bcur_status_t run(const GemmDesc& d, int prec, cudaStream_t s, int epi, int64_t* n_partials) {
  if (d.M <= 0 || d.N <= 0) {
    if (n_partials) *n_partials = 0;
    return BCUR_OK;
  }
  Prepared pr;
  BCUR_TRY(prepare(d, prec, epi, 0, &pr));
  Params& p = pr.p;
  const Maps& maps = pr.maps;
  const int BN = pr.BN, kind = pr.kind, batch = p.batch;
  const int sms = sm_count();
  const int tiles = p.tiles_m * p.tiles_n;
  // Split K when there are too few tiles to fill the GPU and a scratch
  // buffer for the partial slices is available.
  if (epi == EPI_STORE && kind != 2 && d.scratch && batch == 1 && tiles < sms &&
      p.kblocks >= 8) {
    int ks = std::min<int64_t>(std::max<int64_t>(1, (4 * sms) / tiles), p.kblocks / 4);
    const int64_t slice = (int64_t)p.Mm * p.Nm * 4;
    ks = (int)std::min<int64_t>(ks, (int64_t)d.scratch_bytes / slice);
    if (ks > 1) {
      p.ksplit = ks;
      p.part = (float*)d.scratch;
    }
  }
  const int units = tiles * p.ksplit * batch;
  const int grid = std::max(1, std::min(units, sms));
  if (epi == EPI_RESID) {
    if (n_partials) *n_partials = grid;
    return kind == 0 ? launch_bn<0, EPI_RESID>(BN, maps, p, grid, s)
                     : launch_bn<1, EPI_RESID>(BN, maps, p, grid, s);
  }
  if (p.ksplit > 1) {
    BCUR_TRY((kind == 0 ? launch_bn<0, EPI_PARTIAL>(BN, maps, p, grid, s)
                        : launch_bn<1, EPI_PARTIAL>(BN, maps, p, grid, s)));
    const int64_t total = (int64_t)p.Mm * p.Nm;
    const int blocks = (int)std::min<int64_t>(ceil_div(total, 256), 4 * sms);
    splitk_reduce_kernel<<<blocks, 256, 0, s>>>(p);
    BCUR_LAUNCH_CHECK();
    return BCUR_OK;
  }
  if (kind == 2) return launch_bn<2, EPI_STORE>(BN, maps, p, grid, s);
  return kind == 0 ? launch_bn<0, EPI_STORE>(BN, maps, p, grid, s)
                   : launch_bn<1, EPI_STORE>(BN, maps, p, grid, s);
}

// ---------------------------------------------------------------------------
// Grouped launches
// ---------------------------------------------------------------------------
size_t group_bytes(int count) {
  return (size_t)count * sizeof(GEntry) + (size_t)(2 * count + 1) * sizeof(int) + 256;
}

// X pointers of a residual group, read per launch from a caller table:
// entry i takes *(base + owner[i] * stride + offset).
__global__ void group_patch_x_kernel(GEntry* e, const int* owner, int count, const char* base,
                                     size_t stride, size_t offset) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  e[i].p.X = *reinterpret_cast<const float* const*>(base + (size_t)owner[i] * stride + offset);
}

bcur_status_t group_prepare(const GemmDesc* ds, int count, int epi, int BN_force, void* dev,
                            size_t bytes, int* status, TcGroup* out, cudaStream_t setup) {
  if (count < 1 || !dev || bytes < group_bytes(count)) return BCUR_EINVAL;
  if (epi != EPI_STORE && epi != EPI_RESID) return BCUR_EINVAL;
  if (reinterpret_cast<uintptr_t>(dev) % 128 != 0) return BCUR_EINVAL;
  // Tile width shared by the whole launch: the least padded MMA work, ties
  // going to the wider tile.
  int BN = BN_force;
  if (!BN) {
    double best = -1.0;
    for (int cand : {256, 128, 64}) {
      double work = 0.0;
      for (int i = 0; i < count; ++i) {
        Prepared pr;
        BCUR_TRY(prepare(ds[i], BCUR_BF16, epi, cand, &pr));
        work += (double)pr.p.tiles_m * pr.p.tiles_n * cand * pr.p.kblocks * pr.p.parts * pr.p.batch;
      }
      if (best < 0.0 || work < best) { best = work; BN = cand; }
    }
  }
  std::vector<GEntry> e(count);
  std::vector<int> order(count);
  std::vector<double> weight(count);
  for (int i = 0; i < count; ++i) {
    Prepared pr;
    BCUR_TRY(prepare(ds[i], BCUR_BF16, epi, BN, &pr));
    if (epi == EPI_RESID && (pr.p.tri_out || pr.p.batch != 1 || !ds[i].partials))
      return BCUR_EINVAL;
    e[i].maps = pr.maps;
    e[i].p = pr.p;
    order[i] = i;
    weight[i] = (double)pr.p.kblocks * pr.p.parts;
  }
  // heaviest units first
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return weight[x] > weight[y]; });
  std::vector<GEntry> sorted(count);
  std::vector<int> starts(count + 1, 0);
  int64_t total = 0;
  for (int i = 0; i < count; ++i) {
    sorted[i] = e[order[i]];
    starts[i] = (int)total;
    total += (int64_t)sorted[i].p.tiles_m * sorted[i].p.tiles_n * sorted[i].p.batch;
  }
  if (total > INT32_MAX) return BCUR_ENOTSUP;
  starts[count] = (int)total;
  char* base = static_cast<char*>(dev);
  // Pageable sources: each copy has been staged when the call returns.
  BCUR_CUDA_TRY(cudaMemcpyAsync(base, sorted.data(), (size_t)count * sizeof(GEntry),
                                cudaMemcpyHostToDevice, setup));
  int* d_starts = reinterpret_cast<int*>(base + (size_t)count * sizeof(GEntry));
  BCUR_CUDA_TRY(cudaMemcpyAsync(d_starts, starts.data(), (size_t)(count + 1) * sizeof(int),
                                cudaMemcpyHostToDevice, setup));
  BCUR_CUDA_TRY(cudaMemcpyAsync(d_starts + count + 1, order.data(), (size_t)count * sizeof(int),
                                cudaMemcpyHostToDevice, setup));
  BCUR_CUDA_TRY(cudaStreamSynchronize(setup));
  out->BN = BN;
  out->epi = epi;
  out->count = count;
  out->total = (int)total;
  out->grid = (int)std::max<int64_t>(1, std::min<int64_t>(total, sm_count()));
  out->table = dev;
  out->starts = d_starts;
  out->status = status;
  return BCUR_OK;
}

bcur_status_t group_patch_x(const TcGroup& g, const void* base, size_t stride, size_t offset,
                            cudaStream_t s) {
  if (g.count < 1) return BCUR_OK;
  group_patch_x_kernel<<<(g.count + 127) / 128, 128, 0, s>>>(
      static_cast<GEntry*>(g.table), g.starts + g.count + 1, g.count,
      static_cast<const char*>(base), stride, offset);
  BCUR_LAUNCH_CHECK();
  return BCUR_OK;
}

bcur_status_t group_run(const TcGroup& g, cudaStream_t s, int grid) {
  if (g.count < 1 || g.total < 1) return BCUR_OK;
  Group grp;
  grp.e = static_cast<const GEntry*>(g.table);
  grp.starts = g.starts;
  grp.count = g.count;
  grp.total = g.total;
  grp.status = g.status;
  Maps maps;
  memset(&maps, 0, sizeof(maps));
  Params p{};
  const int gr = grid > 0 ? std::min(grid, g.total) : g.grid;
  return g.epi == EPI_RESID ? launch_bn<1, EPI_RESID, true>(g.BN, maps, p, gr, s, grp)
                            : launch_bn<1, EPI_STORE, true>(g.BN, maps, p, gr, s, grp);
}

}  // namespace tc

bool gemm_tc_available() { return tc::tc_device_ok(); }

bcur_status_t gemm_tc_set_wait_budget(uint64_t ns) {
  const unsigned long long v = (unsigned long long)ns;
  BCUR_CUDA_TRY(cudaMemcpyToSymbol(tc::g_wait_budget_ns, &v, sizeof(v)));
  return BCUR_OK;
}

int64_t gemm_tc_resid_ctas(int64_t, int64_t) { return 1024; }

bcur_status_t gemm_tc(const GemmDesc& d, int prec, cudaStream_t s) {
  return tc::run(d, prec, s, tc::EPI_STORE, nullptr);
}

bcur_status_t gemm_tc_resid(const GemmDesc& d, int prec, cudaStream_t s, int64_t* n_partials) {
  if (d.batch != 1) return BCUR_ENOTSUP;
  return tc::run(d, prec, s, tc::EPI_RESID, n_partials);
}

size_t gemm_tc_group_bytes(int count) { return tc::group_bytes(count); }

bcur_status_t gemm_tc_group_prepare(const GemmDesc* ds, int count, int resid, int BN, void* dev,
                                    size_t bytes, int* status, TcGroup* out, cudaStream_t setup) {
  return tc::group_prepare(ds, count, resid ? tc::EPI_RESID : tc::EPI_STORE, BN, dev, bytes,
                           status, out, setup);
}

bcur_status_t gemm_tc_group_run(const TcGroup& g, cudaStream_t s, int grid) {
  return tc::group_run(g, s, grid);
}

bcur_status_t gemm_tc_group_patch_x(const TcGroup& g, const void* base, size_t stride,
                                    size_t offset, cudaStream_t s) {
  return tc::group_patch_x(g, base, stride, offset, s);
}

int64_t gemm_tc_units(const GemmDesc& d, int resid, int BN) {
  tc::Prepared pr;
  if (tc::prepare(d, BCUR_BF16, resid ? tc::EPI_RESID : tc::EPI_STORE, BN, &pr) != BCUR_OK)
    return -1;
  return (int64_t)pr.p.tiles_m * pr.p.tiles_n * pr.p.batch;
}

}  // namespace bcur
