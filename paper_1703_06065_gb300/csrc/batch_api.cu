// Batched plan of the C ABI: validation, workspace layout, the launch tables
// (grouped GEMMs and work lists) and the fixed launch sequence of one run.
// Every stage of the method is one launch over the whole batch; the host
// never synchronises inside a run, so the sequence can be captured in a CUDA
// graph and replayed.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "batch.h"

using namespace bcur;
using namespace bcur::batch;

namespace {

struct WorkList {
  std::vector<int> h;  // count + 1 prefix sums
  int* d = nullptr;
  int total = 0;
  Work w() const { return Work{d, (int)h.size() - 1}; }
};

}  // namespace

// Handles are opaque to callers: a tag as the first member lets every entry
// point refuse a handle of the other kind (a single-matrix plan) or a stale one.
constexpr uint32_t kBatchTag = 0x42435542u;  // "BUCB"

struct bcur_batch_s {
  uint32_t tag = kBatchTag;
  int B = 0, q = 0;
  int lp = 64;  // panel rows: 64, or 128 when some item has l > 64
  std::vector<bcur_batch_item_t> d;
  std::vector<Item> it;
  cudaStream_t stream = nullptr;
  size_t need = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool bound = false;
  // device tables
  Item* d_items = nullptr;
  bcur_batch_io_t* d_io = nullptr;
  int* d_status = nullptr;
  double* Lb_all = nullptr;
  float *Ut_all = nullptr, *W_all = nullptr, *jw_all = nullptr;
  double* sig_all = nullptr;
  int* d_l = nullptr;    // l = k + p of every item (the Jacobi's own width)
  bcur_batch_io_t* h_io = nullptr;  // pinned staging of the io table
  cudaEvent_t ev_io = nullptr;
  WorkList rows8, chunks_m, chunks_n, apply_m, apply_n, blocks, ctiles, rrows, urows;
  // wide Cholesky launches by size class (w <= 128, 256, 512): the shared
  // memory of a launch, and so the CTAs per SM, follows its largest w
  int* wide_entries[3] = {nullptr, nullptr, nullptr};
  int wide_count[3] = {0, 0, 0};
  // grouped GEMMs; each stage is split by output width into up to three
  // launches with 64-, 128- and 256-wide tiles
  struct MGroup {
    void* tab[3] = {nullptr, nullptr, nullptr};  // table memory per width slot
    TcGroup g[3];                                // the prepared launches
    int n = 0;
  };
  MGroup gY, gZ, gY2, gGram[2], gApply[2], gW, gM, gU[6], gP, gRes, gP3, gRes3;
  // adaptive fit: the second Cholesky-QR pass's Grams with one BF16 term
  // (the three-term gGram[1] then runs only for items the residual refines)
  MGroup gGram1;
  // adaptive split fit (BCUR_BF16X3A): one-term W, M and the products to M2;
  // the three-term groups above then run only for items whose one-term
  // residual asks for refinement
  int fit_prec = BCUR_BF16X3;
  MGroup gW1, gM1, gU1[4];
  int* d_terms = nullptr;  // per item: terms of its core products (bcur_batch_fit_terms)
  // graph mode: the sequence is captured on a stream of the plan's own and
  // joined to the caller's stream through events
  cudaStream_t gstream = nullptr;
  cudaStream_t sstream = nullptr;  // uploads of the launch tables (never waits on other work)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  // optional events between the launches of an eager run
  bool profile = false, marking = false;
  std::vector<cudaEvent_t> pev;
  std::vector<const char*> plabel;
  int pn = 0;
};

namespace {

bool batch_ok(const bcur_batch_s* P) { return P && P->tag == kBatchTag; }

// Bump allocator over the workspace; with base == nullptr it only measures.
struct Bump {
  char* base;
  size_t cur = 0;
  template <typename T> T* take(size_t count) {
    const size_t at = cur;
    cur += (count * sizeof(T) + 255) / 256 * 256;
    return base ? reinterpret_cast<T*>(base + at) : nullptr;
  }
};

void derive(Item& I, const bcur_batch_item_t& d) {
  I = Item{};
  I.m = d.m; I.n = d.n; I.lda = d.lda;
  I.k = d.k; I.l = d.k + d.p; I.s = d.block;
  I.Gc = (int)ceil_div(d.n, d.block);
  I.Gr = (int)ceil_div(d.m, d.block);
  I.gc = d.g_col; I.gr = d.g_row;
  I.ldm = round_up(d.m, 64);
  I.ldn = round_up(d.n, 64);
  I.cmax = d.g_col * d.block;
  I.rmax = d.g_row * d.block;
  I.cpad = (int)round_up(I.cmax, NB);
  I.rpad = (int)round_up(I.rmax, NB);
  I.chunks_m = (int)ceil_div(d.m, CH);
  I.chunks_n = (int)ceil_div(d.n, CH);
  I.res_units = ceil_div(d.m, 128) * ceil_div(d.n, 256);
}

// Lay out everything; pointers are assigned when P->ws is set.
size_t layout(bcur_batch_t P) {
  Bump bp{P->ws};
  const int B = P->B;
  P->d_items = bp.take<Item>(B);
  P->d_io = bp.take<bcur_batch_io_t>(B);
  P->d_status = bp.take<int>(1);
  const int64_t LP = P->lp;
  P->Lb_all = bp.take<double>((size_t)B * LP * LP);
  P->Ut_all = bp.take<float>((size_t)B * LP * LP);
  P->W_all = bp.take<float>((size_t)B * LP * LP);
  P->jw_all = bp.take<float>((size_t)B * LP * LP);
  P->sig_all = bp.take<double>((size_t)B * LP);
  P->d_l = bp.take<int>(B);
  WorkList* wls[] = {&P->rows8, &P->chunks_m, &P->chunks_n, &P->apply_m, &P->apply_n,
                     &P->blocks, &P->ctiles, &P->rrows, &P->urows};
  for (WorkList* w : wls) w->d = bp.take<int>(B + 1);
  for (int i = 0; i < 3; ++i) P->wide_entries[i] = bp.take<int>(2 * B);
  auto grp = [&](bcur_batch_s::MGroup& g, int count) {
    for (int i = 0; i < 3; ++i) g.tab[i] = bp.take<char>(gemm_tc_group_bytes(count));
  };
  grp(P->gY, B); grp(P->gZ, B); grp(P->gY2, B);
  for (int i = 0; i < 2; ++i) grp(P->gGram[i], 2 * B);
  grp(P->gGram1, 2 * B);
  grp(P->gApply[0], 2 * B);  // the second Cholesky-QR pass has no apply
  grp(P->gW, B); grp(P->gM, B);
  for (int i = 0; i < 6; ++i) grp(P->gU[i], B);
  grp(P->gP, B); grp(P->gRes, B); grp(P->gP3, B); grp(P->gRes3, B);
  grp(P->gW1, B); grp(P->gM1, B);
  for (int i = 0; i < 4; ++i) grp(P->gU1[i], B);
  P->d_terms = bp.take<int>(B);
  for (int b = 0; b < B; ++b) {
    Item& I = P->it[b];
    I.lp = P->lp;
    const int64_t m = I.m, n = I.n, ldm = I.ldm, ldn = I.ldn;
    const int64_t cp = I.cpad, rp = I.rpad;
    I.Ah = bp.take<bf16>(m * ldn);
    I.Al = bp.take<bf16>(m * ldn);
    I.Om = bp.take<bf16>(LP * ldn);
    I.Pm0 = bp.take<float>(LP * ldm);
    I.Pm1 = bp.take<float>(LP * ldm);
    I.Pn0 = bp.take<float>(LP * ldn);
    I.Pn1 = bp.take<float>(LP * ldn);
    I.Qh = bp.take<bf16>(LP * ldm);
    I.Zh = bp.take<bf16>(LP * ldn);
    I.gpart = bp.take<float>((size_t)std::max(I.chunks_m, I.chunks_n) * LP * LP);
    I.G64 = bp.take<double>(LP * LP);
    I.L64a = bp.take<double>(LP * LP);
    I.L64b = bp.take<double>(LP * LP);
    I.Linv64 = bp.take<double>(LP * LP);
    I.LinvT = bp.take<float>(LP * LP);
    I.remaining = bp.take<unsigned char>(I.Gc + I.Gr);
    I.colmap = bp.take<int>(cp);
    I.rowmap = bp.take<int>(rp);
    for (int i = 0; i < 2; ++i) {
      I.XCh[i] = bp.take<bf16>(cp * ldm);
      I.XCl[i] = bp.take<bf16>(cp * ldm);
      I.XRh[i] = bp.take<bf16>(rp * ldn);
      I.XRl[i] = bp.take<bf16>(rp * ldn);
    }
    I.GC = bp.take<float>(cp * cp);
    I.GR = bp.take<float>(rp * rp);
    for (int i = 0; i < 2; ++i) {
      I.LC[i] = bp.take<float>(cp * cp);
      I.LCi[i] = bp.take<float>(cp * cp);
      I.LR[i] = bp.take<float>(rp * rp);
      I.LRi[i] = bp.take<float>(rp * rp);
      I.LCih[i] = bp.take<bf16>(cp * cp);
      I.LCil[i] = bp.take<bf16>(cp * cp);
      I.LRih[i] = bp.take<bf16>(rp * rp);
      I.LRil[i] = bp.take<bf16>(rp * rp);
    }
    I.Wh = bp.take<bf16>(m * rp);
    I.Wl = bp.take<bf16>(m * rp);
    I.Mf = bp.take<float>(cp * rp);
    I.Mh = bp.take<bf16>(cp * rp);
    I.Ml = bp.take<bf16>(cp * rp);
    I.U1h = bp.take<bf16>(cp * rp);
    I.U1l = bp.take<bf16>(cp * rp);
    I.U2h = bp.take<bf16>(cp * rp);
    I.U2l = bp.take<bf16>(cp * rp);
    I.Uf = bp.take<float>(cp * rp);
    I.Ph = bp.take<bf16>(m * rp);
    I.Pl = bp.take<bf16>(m * rp);
    I.partials = bp.take<double>(2 * kResidSlots * I.res_units);
    I.kept = bp.take<int>(4);
    I.refine = bp.take<int>(1);
    if (P->ws) {
      I.Lb = P->Lb_all + (size_t)b * LP * LP;
      I.Ut = P->Ut_all + (size_t)b * LP * LP;
      I.W = P->W_all + (size_t)b * LP * LP;
    }
  }
  return bp.cur;
}

void build_list(WorkList& w, const std::vector<int>& per) {
  w.h.assign(per.size() + 1, 0);
  for (size_t i = 0; i < per.size(); ++i) w.h[i + 1] = w.h[i] + per[i];
  w.total = w.h.back();
}

GemmDesc g16(int64_t M, int64_t N, int64_t K, const void* A, const void* Alo, int64_t lda, int tA,
             const void* B, const void* Blo, int64_t ldb, int tB, int64_t ldd, int parts) {
  GemmDesc g;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.lda = lda; g.transA = tA;
  g.B = B; g.ldb = ldb; g.transB = tB;
  g.ldd = ldd;
  g.ab_bf16 = 1;
  g.parts = parts;
  if (parts == 3) { g.A_lo = Alo; g.B_lo = Blo; }
  return g;
}

// Tile width of every GEMM of a stage (from the autotuner, autotune.cu), then
// one grouped launch per width.
bcur_status_t prep(bcur_batch_t P, bcur_batch_s::MGroup& g, std::vector<GemmDesc>& ds, int resid,
                   const std::vector<int>& bns) {
  const int widths[3] = {64, 128, 256};
  g.n = 0;
  for (int wi = 0; wi < 3; ++wi) {
    std::vector<GemmDesc> part;
    for (size_t i = 0; i < ds.size(); ++i) {
      if (bns[i] != widths[wi]) continue;
      part.push_back(ds[i]);
      part.back().status = P->d_status;
    }
    if (part.empty()) continue;
    BCUR_TRY(gemm_tc_group_prepare(part.data(), (int)part.size(), resid, widths[wi], g.tab[wi],
                                   gemm_tc_group_bytes((int)ds.size()), P->d_status, &g.g[g.n],
                                   P->sstream));
    ++g.n;
  }
  return BCUR_OK;
}

bcur_status_t run_group(const bcur_batch_s::MGroup& g, cudaStream_t s) {
  for (int i = 0; i < g.n; ++i) BCUR_TRY(gemm_tc_group_run(g.g[i], s));
  return BCUR_OK;
}

bcur_status_t build_groups(bcur_batch_t P) {
  const int B = P->B;
  std::vector<GemmDesc> y, z, y2, w, mm, u[6], pp, res, pp3, res3, w1, mm1, u1[4];
  const bool adapt = P->fit_prec == BCUR_BF16X3A;
  std::vector<GemmDesc> gram[2], app[2], gram1;
  const int64_t LP = P->lp;
  for (int b = 0; b < B; ++b) {
    const Item& I = P->it[b];
    const int64_t m = I.m, n = I.n, ldm = I.ldm, ldn = I.ldn, cp = I.cpad, rp = I.rpad;
    GemmDesc d = g16(LP, m, n, I.Om, nullptr, ldn, 0, I.Ah, nullptr, ldn, 1, ldm, 1);
    d.D = I.Pm0;
    y.push_back(d);
    d = g16(LP, n, m, I.Qh, nullptr, ldm, 0, I.Ah, nullptr, ldn, 0, ldn, 1);
    d.D = I.Pn0;
    z.push_back(d);
    d = g16(LP, m, n, I.Zh, nullptr, ldn, 0, I.Ah, nullptr, ldn, 1, ldm, 1);
    d.D = I.Pm0;
    y2.push_back(d);
    for (int pass = 0; pass < 2; ++pass) {
      d = g16(cp, cp, m, I.XCh[pass], I.XCl[pass], ldm, 0, I.XCh[pass], I.XCl[pass], ldm, 1, cp, 3);
      d.D = I.GC;
      d.out_lower = 1;
      gram[pass].push_back(d);
      d = g16(rp, rp, n, I.XRh[pass], I.XRl[pass], ldn, 0, I.XRh[pass], I.XRl[pass], ldn, 1, rp, 3);
      d.D = I.GR;
      d.out_lower = 1;
      gram[pass].push_back(d);
      d = g16(cp, m, cp, I.LCih[pass], I.LCil[pass], cp, 0, I.XCh[pass], I.XCl[pass], ldm, 0, ldm, 3);
      d.Dh = I.XCh[1 - pass];
      d.Dl = I.XCl[1 - pass];
      d.triA = 1;
      app[pass].push_back(d);
      d = g16(rp, n, rp, I.LRih[pass], I.LRil[pass], rp, 0, I.XRh[pass], I.XRl[pass], ldn, 0, ldn, 3);
      d.Dh = I.XRh[1 - pass];
      d.Dl = I.XRl[1 - pass];
      d.triA = 1;
      app[pass].push_back(d);
    }
    if (adapt)  // one-term copies of the second pass's Grams; the pairs only on refinement
      for (size_t j = gram[1].size() - 2; j < gram[1].size(); ++j) {
        GemmDesc g1 = gram[1][j];
        g1.parts = 1;
        g1.A_lo = nullptr;
        g1.B_lo = nullptr;
        gram1.push_back(g1);
        gram[1][j].run_flag = I.refine;
      }
    // The second Cholesky-QR pass stops at L2 (no apply): Q1 = the pass-0
    // result (index 1), Q = Q1 L2^{-T}.  W1 = A Q1_R^T (m x r); M1 = Q1_C W1
    // (c x r); M2 = L2C^{-T} L2C^{-1} M1 L2R^{-T} L2R^{-1}, so that
    // Q_C M Q_R^T = Q1_C M2 Q1_R^T; U = L1C^{-T} M2 L1R^{-1}.
    d = g16(m, rp, n, I.Ah, I.Al, ldn, 0, I.XRh[1], I.XRl[1], ldn, 1, rp, 3);
    d.Dh = I.Wh;
    d.Dl = I.Wl;
    w.push_back(d);
    d = g16(cp, rp, m, I.XCh[1], I.XCl[1], ldm, 0, I.Wh, I.Wl, rp, 0, rp, 3);
    d.Dh = I.Mh;
    d.Dl = I.Ml;
    mm.push_back(d);
    d = g16(cp, rp, rp, I.Mh, I.Ml, rp, 0, I.LRih[1], I.LRil[1], rp, 1, rp, 3);  // M1 L2R^{-T}
    d.Dh = I.U1h; d.Dl = I.U1l; d.triB = 2;
    u[0].push_back(d);
    d = g16(cp, rp, rp, I.U1h, I.U1l, rp, 0, I.LRih[1], I.LRil[1], rp, 0, rp, 3);  // .. L2R^{-1}
    d.Dh = I.U2h; d.Dl = I.U2l; d.triB = 1;
    u[1].push_back(d);
    d = g16(cp, rp, cp, I.LCih[1], I.LCil[1], cp, 0, I.U2h, I.U2l, rp, 0, rp, 3);  // L2C^{-1} ..
    d.Dh = I.U1h; d.Dl = I.U1l; d.triA = 1;
    u[2].push_back(d);
    d = g16(cp, rp, cp, I.LCih[1], I.LCil[1], cp, 1, I.U1h, I.U1l, rp, 0, rp, 3);  // M2
    d.D = I.Mf; d.Dh = I.Mh; d.Dl = I.Ml; d.triA = 2;
    u[3].push_back(d);
    d = g16(cp, rp, rp, I.Mh, I.Ml, rp, 0, I.LRih[0], I.LRil[0], rp, 0, rp, 3);  // M2 L1R^{-1}
    d.Dh = I.U2h; d.Dl = I.U2l; d.triB = 1;
    u[4].push_back(d);
    d = g16(cp, rp, cp, I.LCih[0], I.LCil[0], cp, 1, I.U2h, I.U2l, rp, 0, rp, 3);  // U
    d.D = I.Uf; d.triA = 2;
    u[5].push_back(d);
    if (adapt) {
      // one-term copies of W1, M1 and the products to M2 (same outputs); the
      // three-term ones run only where the flag is set, and the last two
      // products (U) take the flag's term count
      auto one = [](GemmDesc g) {
        g.parts = 1;
        g.A_lo = nullptr;
        g.B_lo = nullptr;
        return g;
      };
      w1.push_back(one(w.back()));
      mm1.push_back(one(mm.back()));
      for (int i = 0; i < 4; ++i) u1[i].push_back(one(u[i].back()));
      w.back().run_flag = I.refine;
      mm.back().run_flag = I.refine;
      for (int i = 0; i < 4; ++i) u[i].back().run_flag = I.refine;
      u[4].back().parts_flag = I.refine;
      u[5].back().parts_flag = I.refine;
    }
    // P = Q1_C^T M2 (m x r), then sum (A - P Q1_R)^2: one BF16 term, and the
    // BF16-pair version for the items the first result flags
    d = g16(m, rp, cp, I.XCh[1], nullptr, ldm, 1, I.Mh, nullptr, rp, 0, rp, 1);
    d.Dh = I.Ph;
    pp.push_back(d);
    d = g16(m, n, rp, I.Ph, nullptr, rp, 0, I.XRh[1], nullptr, ldn, 0, 0, 1);
    d.X = nullptr;  // set per run from the io table
    d.ldx = I.lda;
    d.partials = I.partials;
    res.push_back(d);
    d = g16(m, rp, cp, I.XCh[1], I.XCl[1], ldm, 1, I.Mh, I.Ml, rp, 0, rp, 3);
    d.Dh = I.Ph;
    d.Dl = I.Pl;
    d.run_flag = I.refine;
    pp3.push_back(d);
    d = g16(m, n, rp, I.Ph, I.Pl, rp, 0, I.XRh[1], I.XRl[1], ldn, 0, 0, 3);
    d.X = nullptr;
    d.ldx = I.lda;
    d.partials = I.partials;
    d.run_flag = I.refine;
    res3.push_back(d);
  }
  // The tables are independent: encode them on parallel host threads (the
  // tensor-map encoding is pure host work; the uploads share the plan's setup
  // stream, whose use from several threads is ordered by the runtime).
  // Candidate tile widths per stage: the skinny sketch products (64 or 128
  // output rows) try 64 and 128; the residual keeps 256 (its epilogue streams
  // A, and A is only known per run); every other product tries all three.
  struct Job {
    bcur_batch_s::MGroup* g;
    std::vector<GemmDesc>* ds;
    int resid;
    const char* stage;
    std::vector<int> cands;
    std::vector<int> bns;
  };
  const std::vector<int> all = {64, 128, 256}, narrow = {64, 128}, wide = {256};
  std::vector<Job> jobs = {{&P->gY, &y, 0, "sketch_y", narrow, {}},
                           {&P->gZ, &z, 0, "sketch_z", narrow, {}},
                           {&P->gY2, &y2, 0, "sketch_y2", narrow, {}},
                           {&P->gW, &w, 0, "w", all, {}},
                           {&P->gM, &mm, 0, "m", all, {}},
                           {&P->gP, &pp, 0, "p", all, {}},
                           {&P->gRes, &res, 1, "res", wide, {}},
                           {&P->gP3, &pp3, 0, "p3", all, {}},
                           {&P->gRes3, &res3, 1, "res3", wide, {}}};
  static const char* gram_names[2] = {"gram0", "gram1"};
  static const char* u_names[6] = {"u0", "u1", "u2", "u3", "u4", "u5"};
  for (int i = 0; i < 2; ++i) {
    jobs.push_back({&P->gGram[i], &gram[i], 0, gram_names[i], all, {}});
    if (i == 0) jobs.push_back({&P->gApply[i], &app[i], 0, "apply0", all, {}});  // no second apply
  }
  for (int i = 0; i < 6; ++i) jobs.push_back({&P->gU[i], &u[i], 0, u_names[i], all, {}});
  if (adapt) {
    jobs.push_back({&P->gGram1, &gram1, 0, "gram1", all, {}});
    jobs.push_back({&P->gW1, &w1, 0, "w", all, {}});
    jobs.push_back({&P->gM1, &mm1, 0, "m", all, {}});
    for (int i = 0; i < 4; ++i) jobs.push_back({&P->gU1[i], &u1[i], 0, u_names[i], all, {}});
  }
  // Measuring launches write their tables into the BF16 lo copy of the
  // largest A (not yet filled: the workspace holds no data before a run).
  {
    TuneScratch sc;
    size_t big = 0;
    for (int b = 1; b < B; ++b)
      if (P->it[b].m * P->it[b].ldn > P->it[big].m * P->it[big].ldn) big = b;
    sc.table = P->it[big].Al;
    sc.table_bytes = (size_t)P->it[big].m * P->it[big].ldn * sizeof(bf16);
    sc.status = P->d_status;
    sc.stream = P->sstream;
    int dev = 0;
    BCUR_CUDA_TRY(cudaGetDevice(&dev));
    BCUR_CUDA_TRY(cudaDeviceGetAttribute(&sc.sms, cudaDevAttrMultiProcessorCount, dev));
    for (Job& j : jobs) BCUR_TRY(tune_widths(j.stage, *j.ds, j.resid, j.cands, sc, &j.bns));
    BCUR_CUDA_TRY(cudaMemsetAsync(P->d_status, 0, sizeof(int), P->sstream));
    BCUR_CUDA_TRY(cudaStreamSynchronize(P->sstream));
  }
  std::vector<bcur_status_t> st(jobs.size(), BCUR_OK);
  const unsigned hw = std::max(1u, std::min(8u, std::thread::hardware_concurrency()));
  int dev = 0;
  BCUR_CUDA_TRY(cudaGetDevice(&dev));
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < hw; ++t)
    pool.emplace_back([&, t] {
      // a new host thread has no current context: bind the caller's device
      // (the tensor-map encoder validates addresses against it)
      if (cudaSetDevice(dev) != cudaSuccess) {
        for (size_t j = t; j < jobs.size(); j += hw) st[j] = BCUR_ECUDA;
        return;
      }
      for (size_t j = t; j < jobs.size(); j += hw)
        st[j] = prep(P, *jobs[j].g, *jobs[j].ds, jobs[j].resid, jobs[j].bns);
    });
  for (auto& th : pool) th.join();
  for (bcur_status_t e : st) BCUR_TRY(e);
  return BCUR_OK;
}

// Profiling marker: an event after the launch(es) just enqueued.
bcur_status_t mark(bcur_batch_t P, cudaStream_t s, const char* label) {
  if (!P->marking) return BCUR_OK;
  if (P->pn >= (int)P->pev.size()) {
    cudaEvent_t e;
    BCUR_CUDA_TRY(cudaEventCreate(&e));
    P->pev.push_back(e);
    P->plabel.push_back(nullptr);
  }
  BCUR_CUDA_TRY(cudaEventRecord(P->pev[P->pn], s));
  P->plabel[P->pn] = label;
  ++P->pn;
  return BCUR_OK;
}

bcur_status_t orth(bcur_batch_t P, int s0, int s1, bool want_lb, cudaStream_t s) {
  const bool m_side = s0 < PN0;
  const WorkList& ch = m_side ? P->chunks_m : P->chunks_n;
  const WorkList& ap = m_side ? P->apply_m : P->apply_n;
  const int lp = P->lp;
  BCUR_TRY(skinny_gram(P->d_items, ch.w(), ch.total, s0, lp, s));
  BCUR_TRY(mark(P, s, "skinny_gram"));
  BCUR_TRY(skinny_chol(P->d_items, P->B, s0, 0, 0, lp, s));
  BCUR_TRY(mark(P, s, "skinny_chol"));
  BCUR_TRY(skinny_apply(P->d_items, ap.w(), ap.total, s0, s1, 0, lp, s));
  BCUR_TRY(mark(P, s, "skinny_apply"));
  BCUR_TRY(skinny_gram(P->d_items, ch.w(), ch.total, s1, lp, s));
  BCUR_TRY(mark(P, s, "skinny_gram"));
  BCUR_TRY(skinny_chol(P->d_items, P->B, s1, 1, want_lb ? 1 : 0, lp, s));
  BCUR_TRY(mark(P, s, "skinny_chol"));
  BCUR_TRY(skinny_apply(P->d_items, ap.w(), ap.total, s1, s0, 1, lp, s));
  BCUR_TRY(mark(P, s, "skinny_apply"));
  return BCUR_OK;
}

// The wide Cholesky of pass `pass` for every item (gated: only the items whose
// refinement flag is set), one launch per size class.
bcur_status_t wide_chol_all(bcur_batch_t P, int pass, cudaStream_t s, int gated) {
  const int wmax[3] = {128, 256, 512};
  for (int c = 0; c < 3; ++c)
    BCUR_TRY(wide_chol(P->d_items, P->wide_entries[c], P->wide_count[c], wmax[c], pass, s, gated));
  return BCUR_OK;
}

// The fit and residual of the adaptive split fit: W1, M1 and M2 and the
// residual with one BF16 term (after a second Cholesky-QR pass with one
// term); the finish sets each item's refinement flag (residual_needs_refine);
// the three-term launches redo the second pass, those products and the
// residual for the flagged items only; the two products that give U take the
// flag's term count.
bcur_status_t enqueue_adaptive_fit(bcur_batch_t P, cudaStream_t s) {
  const int B = P->B;
  BCUR_TRY(run_group(P->gW1, s));
  BCUR_TRY(mark(P, s, "w_gemm"));
  BCUR_TRY(run_group(P->gM1, s));
  BCUR_TRY(mark(P, s, "m_gemm"));
  for (int i = 0; i < 4; ++i) {
    BCUR_TRY(run_group(P->gU1[i], s));
    BCUR_TRY(mark(P, s, "u_gemm"));
  }
  BCUR_TRY(run_group(P->gP, s));
  BCUR_TRY(mark(P, s, "p_gemm"));
  BCUR_TRY(run_group(P->gRes, s));
  BCUR_TRY(mark(P, s, "residual"));
  BCUR_TRY(finish(P->d_items, P->d_io, B, 0, s));
  BCUR_TRY(mark(P, s, "finish"));
  BCUR_TRY(split_inputs(P->d_items, P->d_io, P->rows8.w(), P->rows8.total, B, P->lp, s, 2));
  BCUR_TRY(mark(P, s, "split"));
  // the second Cholesky-QR pass again with three terms, for the refined items
  BCUR_TRY(run_group(P->gGram[1], s));
  BCUR_TRY(mark(P, s, "qr_gram"));
  BCUR_TRY(wide_chol_all(P, 1, s, 1));
  BCUR_TRY(mark(P, s, "wide_chol"));
  BCUR_TRY(run_group(P->gW, s));
  BCUR_TRY(mark(P, s, "w_gemm"));
  BCUR_TRY(run_group(P->gM, s));
  BCUR_TRY(mark(P, s, "m_gemm"));
  for (int i = 0; i < 4; ++i) {
    BCUR_TRY(run_group(P->gU[i], s));
    BCUR_TRY(mark(P, s, "u_gemm"));
  }
  BCUR_TRY(run_group(P->gP3, s));
  BCUR_TRY(mark(P, s, "p_gemm"));
  BCUR_TRY(run_group(P->gRes3, s));
  BCUR_TRY(mark(P, s, "residual"));
  BCUR_TRY(finish(P->d_items, P->d_io, B, 1, s));
  BCUR_TRY(mark(P, s, "finish"));
  for (int i = 4; i < 6; ++i) {
    BCUR_TRY(run_group(P->gU[i], s));
    BCUR_TRY(mark(P, s, "u_gemm"));
  }
  BCUR_TRY(copy_u(P->d_items, P->d_io, P->urows.w(), P->urows.total, s));
  BCUR_TRY(mark(P, s, "copy_u"));
  return BCUR_OK;
}

// The launch sequence of one run (the io table is already being copied).
bcur_status_t enqueue(bcur_batch_t P, cudaStream_t s) {
  const int B = P->B;
  if (P->marking) P->pn = 0;
  BCUR_TRY(mark(P, s, "start"));
  for (const auto* g : {&P->gRes, &P->gRes3})
    for (int i = 0; i < g->n; ++i)
      BCUR_TRY(gemm_tc_group_patch_x(g->g[i], P->d_io, sizeof(bcur_batch_io_t),
                                     offsetof(bcur_batch_io_t, A), s));
  // the adaptive fit splits A's lo half later, for the items it refines
  BCUR_TRY(split_inputs(P->d_items, P->d_io, P->rows8.w(), P->rows8.total, B, P->lp, s,
                        P->fit_prec == BCUR_BF16X3A ? 1 : 0));
  BCUR_TRY(mark(P, s, "split"));
  // scores: randomized range finder with q subspace iterations (Sec. 3.1)
  BCUR_TRY(run_group(P->gY, s));
  BCUR_TRY(mark(P, s, "sketch_gemm"));
  BCUR_TRY(orth(P, PM0, PM1, false, s));
  for (int i = 0; i < P->q; ++i) {
    BCUR_TRY(run_group(P->gZ, s));
    BCUR_TRY(mark(P, s, "sketch_gemm"));
    BCUR_TRY(orth(P, PN0, PN1, false, s));
    BCUR_TRY(run_group(P->gY2, s));
    BCUR_TRY(mark(P, s, "sketch_gemm"));
    BCUR_TRY(orth(P, PM0, PM1, false, s));
  }
  BCUR_TRY(run_group(P->gZ, s));
  BCUR_TRY(mark(P, s, "sketch_gemm"));
  BCUR_TRY(orth(P, PN0, PN1, true, s));
  BCUR_TRY(jacobi_svd_batched<float>(P->Lb_all, P->lp, P->Ut_all, P->W_all, P->sig_all,
                                     P->jw_all, P->d_status, B, s, P->d_l));
  BCUR_TRY(mark(P, s, "jacobi"));
  BCUR_TRY(scores(P->d_items, P->d_io, P->blocks.w(), P->blocks.total, P->d_status, P->lp, s));
  BCUR_TRY(mark(P, s, "scores"));
  // sampling (Alg. 1 step 2) and the gathers
  BCUR_TRY(sample(P->d_items, P->d_io, B, s));
  BCUR_TRY(mark(P, s, "sample"));
  BCUR_TRY(gather(P->d_items, P->d_io, P->ctiles.w(), P->ctiles.total, P->rrows.w(),
                  P->rrows.total, s));
  BCUR_TRY(mark(P, s, "gather"));
  // Cholesky-QR2 of C^T and R, both sides in each launch (the adaptive fit
  // takes the second pass's Grams with one term first)
  for (int pass = 0; pass < 2; ++pass) {
    const bool one = pass == 1 && P->fit_prec == BCUR_BF16X3A;
    BCUR_TRY(run_group(one ? P->gGram1 : P->gGram[pass], s));
    BCUR_TRY(mark(P, s, "qr_gram"));
    BCUR_TRY(wide_chol_all(P, pass, s, 0));
    BCUR_TRY(mark(P, s, "wide_chol"));
    if (pass == 0) {  // the second pass stops at L2 (see build_groups)
      BCUR_TRY(run_group(P->gApply[pass], s));
      BCUR_TRY(mark(P, s, "qr_apply"));
    }
  }
  if (P->fit_prec == BCUR_BF16X3A) return enqueue_adaptive_fit(P, s);
  // U = C^+ A R^+
  BCUR_TRY(run_group(P->gW, s));
  BCUR_TRY(mark(P, s, "w_gemm"));
  BCUR_TRY(run_group(P->gM, s));
  BCUR_TRY(mark(P, s, "m_gemm"));
  for (int i = 0; i < 6; ++i) {
    BCUR_TRY(run_group(P->gU[i], s));
    BCUR_TRY(mark(P, s, "u_gemm"));
  }
  BCUR_TRY(copy_u(P->d_items, P->d_io, P->urows.w(), P->urows.total, s));
  BCUR_TRY(mark(P, s, "copy_u"));
  // ||A - CUR||_F
  BCUR_TRY(run_group(P->gP, s));
  BCUR_TRY(mark(P, s, "p_gemm"));
  BCUR_TRY(run_group(P->gRes, s));
  BCUR_TRY(mark(P, s, "residual"));
  BCUR_TRY(finish(P->d_items, P->d_io, B, 0, s));
  BCUR_TRY(mark(P, s, "finish"));
  BCUR_TRY(run_group(P->gP3, s));
  BCUR_TRY(mark(P, s, "p_gemm"));
  BCUR_TRY(run_group(P->gRes3, s));
  BCUR_TRY(mark(P, s, "residual"));
  BCUR_TRY(finish(P->d_items, P->d_io, B, 1, s));
  BCUR_TRY(mark(P, s, "finish"));
  return BCUR_OK;
}

bool item_ok(const bcur_batch_item_t& d) {
  if (d.m < 1 || d.n < 1 || d.lda < d.n || d.lda % 4 != 0) return false;
  if (d.m > INT32_MAX / 2 || d.n > INT32_MAX / 2) return false;
  if (d.k < 1 || d.p < 0 || d.k + d.p > LP_MAX || d.k + d.p > d.m || d.k + d.p > d.n) return false;
  if (d.block < 1) return false;
  const int64_t Gc = ceil_div(d.n, d.block), Gr = ceil_div(d.m, d.block);
  if (Gc > 32768 || Gr > 32768) return false;
  if (d.g_col < 1 || d.g_row < 1 || d.g_col > Gc || d.g_row > Gr) return false;
  if ((int64_t)d.g_col * d.block > WMAX || (int64_t)d.g_row * d.block > WMAX) return false;
  return true;
}

}  // namespace

extern "C" {

bcur_status_t bcur_batch_plan(const bcur_batch_item_t* items, int32_t count, int32_t q,
                              void* stream, bcur_batch_t* out, size_t* workspace_bytes) {
  if (!items || !out || !workspace_bytes || count < 1 || q < 0 || q > 16) return BCUR_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!item_ok(items[i])) return BCUR_EINVAL;
  bcur_batch_t P = new (std::nothrow) bcur_batch_s();
  if (!P) return BCUR_ENOMEM;
  P->B = count;
  P->q = q;
  P->d.assign(items, items + count);
  P->it.resize(count);
  for (int i = 0; i < count; ++i) {
    derive(P->it[i], items[i]);
    if (P->it[i].l > 64) P->lp = 128;
  }
  P->stream = static_cast<cudaStream_t>(stream);
  P->need = layout(P);
  *out = P;
  *workspace_bytes = P->need;
  return BCUR_OK;
}

bcur_status_t bcur_batch_set_workspace(bcur_batch_t P, void* ws, size_t bytes) {
  if (!batch_ok(P) || !ws || reinterpret_cast<uintptr_t>(ws) % 256 != 0) return BCUR_EINVAL;
  if (bytes < P->need) return BCUR_ENOMEM;
  if (!gemm_tc_available()) return BCUR_ENOTSUP;
  if (P->exec) { cudaGraphExecDestroy(P->exec); P->exec = nullptr; }
  if (P->graph) { cudaGraphDestroy(P->graph); P->graph = nullptr; }
  if (!P->sstream) BCUR_CUDA_TRY(cudaStreamCreateWithFlags(&P->sstream, cudaStreamNonBlocking));
  P->ws = static_cast<char*>(ws);
  P->ws_bytes = bytes;
  layout(P);
  const int B = P->B;
  std::vector<int> r8(B), cm(B), cn(B), am(B), an(B), bl(B), ct(B), rr(B), ur(B);
  for (int b = 0; b < B; ++b) {
    const Item& I = P->it[b];
    r8[b] = (int)ceil_div(I.m, 8);
    cm[b] = I.chunks_m;
    cn[b] = I.chunks_n;
    am[b] = (int)ceil_div(I.m, AP);
    an[b] = (int)ceil_div(I.n, AP);
    bl[b] = I.Gc + I.Gr;
    ct[b] = (int)(ceil_div(I.cpad, 64) * ceil_div(I.m, 64));
    rr[b] = I.rpad;
    ur[b] = I.cmax;
  }
  build_list(P->rows8, r8); build_list(P->chunks_m, cm); build_list(P->chunks_n, cn);
  build_list(P->apply_m, am); build_list(P->apply_n, an); build_list(P->blocks, bl);
  build_list(P->ctiles, ct); build_list(P->rrows, rr); build_list(P->urows, ur);
  WorkList* wls[] = {&P->rows8, &P->chunks_m, &P->chunks_n, &P->apply_m, &P->apply_n,
                     &P->blocks, &P->ctiles, &P->rrows, &P->urows};
  for (WorkList* w : wls)
    BCUR_CUDA_TRY(cudaMemcpyAsync(w->d, w->h.data(), w->h.size() * sizeof(int),
                                  cudaMemcpyHostToDevice, P->sstream));
  {
    std::vector<int> cls[3];
    for (int b = 0; b < B; ++b)
      for (int side = 0; side < 2; ++side) {
        const int w = side ? P->it[b].rpad : P->it[b].cpad;
        cls[w <= 128 ? 0 : (w <= 256 ? 1 : 2)].push_back(b << 1 | side);
      }
    for (int c = 0; c < 3; ++c) {
      P->wide_count[c] = (int)cls[c].size();
      if (!cls[c].empty())
        BCUR_CUDA_TRY(cudaMemcpyAsync(P->wide_entries[c], cls[c].data(),
                                      cls[c].size() * sizeof(int), cudaMemcpyHostToDevice,
                                      P->sstream));
    }
  }
  BCUR_CUDA_TRY(cudaMemcpyAsync(P->d_items, P->it.data(), (size_t)B * sizeof(Item),
                                cudaMemcpyHostToDevice, P->sstream));
  std::vector<int> ls(B);
  for (int b = 0; b < B; ++b) ls[b] = P->it[b].l;
  BCUR_CUDA_TRY(cudaMemcpyAsync(P->d_l, ls.data(), (size_t)B * sizeof(int),
                                cudaMemcpyHostToDevice, P->sstream));
  BCUR_CUDA_TRY(cudaMemsetAsync(P->d_status, 0, sizeof(int), P->sstream));
  BCUR_CUDA_TRY(cudaMemsetAsync(P->d_io, 0, (size_t)B * sizeof(bcur_batch_io_t), P->sstream));
  BCUR_CUDA_TRY(cudaStreamSynchronize(P->sstream));
  if (!P->h_io) {
    BCUR_CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&P->h_io),
                                (size_t)B * sizeof(bcur_batch_io_t), cudaHostAllocDefault));
    BCUR_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_io, cudaEventDisableTiming));
  }
  BCUR_TRY(build_groups(P));
  P->bound = true;
  return BCUR_OK;
}

bcur_status_t bcur_batch_run(bcur_batch_t P, const bcur_batch_io_t* io, int32_t use_graph) {
  if (!batch_ok(P) || !io) return BCUR_EINVAL;
  if (!P->bound) return BCUR_ESTATE;
  for (int b = 0; b < P->B; ++b) {
    const bcur_batch_io_t& e = io[b];
    if (!e.A || !e.omega || !e.u_col || !e.u_row || !e.col_scores || !e.row_scores ||
        !e.col_idx || !e.row_idx || !e.err)
      return BCUR_EINVAL;
  }
  // the previous run's copy of the staging buffer must have finished
  BCUR_CUDA_TRY(cudaEventSynchronize(P->ev_io));
  memcpy(P->h_io, io, (size_t)P->B * sizeof(bcur_batch_io_t));
  cudaStream_t s = P->stream;
  if (use_graph && P->exec) {
    BCUR_CUDA_TRY(cudaEventRecord(P->ev_in, s));
    BCUR_CUDA_TRY(cudaStreamWaitEvent(P->gstream, P->ev_in, 0));
    BCUR_CUDA_TRY(cudaGraphLaunch(P->exec, P->gstream));
    BCUR_CUDA_TRY(cudaEventRecord(P->ev_out, P->gstream));
    BCUR_CUDA_TRY(cudaStreamWaitEvent(s, P->ev_out, 0));
    return BCUR_OK;
  }
  const uint64_t l0 = bcur_launch_count();
  BCUR_CUDA_TRY(cudaMemcpyAsync(P->d_io, P->h_io, (size_t)P->B * sizeof(bcur_batch_io_t),
                                cudaMemcpyHostToDevice, s));
  BCUR_CUDA_TRY(cudaEventRecord(P->ev_io, s));
  P->marking = P->profile;
  const bcur_status_t st0 = enqueue(P, s);
  P->marking = false;
  BCUR_TRY(st0);
  P->launches = (int64_t)(bcur_launch_count() - l0);
  if (use_graph && !P->exec) {
    // Capture the same sequence (on the plan's own stream) for later runs.
    if (!P->gstream) {
      BCUR_CUDA_TRY(cudaStreamCreateWithFlags(&P->gstream, cudaStreamNonBlocking));
      BCUR_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming));
      BCUR_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming));
    }
    cudaStream_t g = P->gstream;
    BCUR_CUDA_TRY(cudaStreamBeginCapture(g, cudaStreamCaptureModeThreadLocal));
    bcur_status_t st = BCUR_OK;
    if (cudaMemcpyAsync(P->d_io, P->h_io, (size_t)P->B * sizeof(bcur_batch_io_t),
                        cudaMemcpyHostToDevice, g) != cudaSuccess ||
        cudaEventRecordWithFlags(P->ev_io, g, cudaEventRecordExternal) != cudaSuccess)
      st = BCUR_ECUDA;
    if (st == BCUR_OK) st = enqueue(P, g);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(g, &graph);
    if (st != BCUR_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    BCUR_CUDA_TRY(e);
    P->graph = graph;
    BCUR_CUDA_TRY(cudaGraphInstantiate(&P->exec, graph, 0));
  }
  return BCUR_OK;
}

bcur_status_t bcur_batch_set_stream(bcur_batch_t P, void* stream) {
  if (!batch_ok(P)) return BCUR_EINVAL;
  if (P->exec) {  // a captured graph belongs to the old stream's sequence: recapture
    cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
  }
  if (P->graph) {
    cudaGraphDestroy(P->graph);
    P->graph = nullptr;
  }
  P->stream = static_cast<cudaStream_t>(stream);
  return BCUR_OK;
}

bcur_status_t bcur_batch_dims(bcur_batch_t P, int32_t i, int64_t* cmax, int64_t* rmax,
                              int64_t* launches_per_run) {
  if (!batch_ok(P) || i < 0 || i >= P->B) return BCUR_EINVAL;
  if (cmax) *cmax = P->it[i].cmax;
  if (rmax) *rmax = P->it[i].rmax;
  if (launches_per_run) *launches_per_run = P->launches;
  return BCUR_OK;
}

bcur_status_t bcur_batch_set_fit(bcur_batch_t P, int32_t fit_prec) {
  if (!batch_ok(P)) return BCUR_EINVAL;
  if (fit_prec != BCUR_BF16X3 && fit_prec != BCUR_BF16X3A) return BCUR_EINVAL;
  if (P->bound) return BCUR_ESTATE;
  P->fit_prec = fit_prec;
  return BCUR_OK;
}

bcur_status_t bcur_batch_fit_terms(bcur_batch_t P, int32_t* terms) {
  if (!batch_ok(P) || !terms) return BCUR_EINVAL;
  if (!P->bound) return BCUR_ESTATE;
  if (P->fit_prec != BCUR_BF16X3A) {
    for (int b = 0; b < P->B; ++b) terms[b] = 3;
    return BCUR_OK;
  }
  BCUR_TRY(fit_terms(P->d_items, P->B, P->d_terms, P->stream));
  BCUR_CUDA_TRY(cudaMemcpyAsync(terms, P->d_terms, (size_t)P->B * sizeof(int),
                                cudaMemcpyDeviceToHost, P->stream));
  BCUR_CUDA_TRY(cudaStreamSynchronize(P->stream));
  return BCUR_OK;
}

bcur_status_t bcur_batch_sync_status(bcur_batch_t P) {
  if (!batch_ok(P)) return BCUR_EINVAL;
  BCUR_CUDA_TRY(cudaStreamSynchronize(P->stream));
  if (!P->bound) return BCUR_OK;
  int st = 0;
  BCUR_CUDA_TRY(cudaMemcpyAsync(&st, P->d_status, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  BCUR_CUDA_TRY(cudaStreamSynchronize(P->stream));
  if (st) {
    BCUR_CUDA_TRY(cudaMemsetAsync(P->d_status, 0, sizeof(int), P->stream));
    BCUR_CUDA_TRY(cudaStreamSynchronize(P->stream));
  }
  return (bcur_status_t)st;
}

bcur_status_t bcur_batch_profile(bcur_batch_t P, int32_t enable) {
  if (!batch_ok(P)) return BCUR_EINVAL;
  P->profile = enable != 0;
  return BCUR_OK;
}

int32_t bcur_batch_profile_count(bcur_batch_t P) { return batch_ok(P) ? (P->pn > 0 ? P->pn - 1 : 0) : 0; }

bcur_status_t bcur_batch_profile_entry(bcur_batch_t P, int32_t i, const char** label, double* ms) {
  if (!batch_ok(P) || i < 0 || i + 1 >= P->pn || !label || !ms) return BCUR_EINVAL;
  float t = 0.f;
  BCUR_CUDA_TRY(cudaEventElapsedTime(&t, P->pev[i], P->pev[i + 1]));
  *label = P->plabel[i + 1];
  *ms = (double)t;
  return BCUR_OK;
}

void bcur_batch_destroy(bcur_batch_t P) {
  if (!batch_ok(P)) return;
  for (cudaEvent_t e : P->pev) cudaEventDestroy(e);
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  if (P->ev_io) cudaEventDestroy(P->ev_io);
  if (P->ev_in) cudaEventDestroy(P->ev_in);
  if (P->ev_out) cudaEventDestroy(P->ev_out);
  if (P->gstream) cudaStreamDestroy(P->gstream);
  if (P->sstream) cudaStreamDestroy(P->sstream);
  if (P->h_io) cudaFreeHost(P->h_io);
  P->tag = 0;
  delete P;
}

}  // extern "C"
