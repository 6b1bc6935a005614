// Tile-width autotuner for the grouped tensor-core GEMMs of the batched path.
//
// A batched stage launches the GEMMs of all its decompositions at once, split
// by tile width (64, 128 or 256 output columns per 128-row tile).  Which width
// is fastest depends on the GEMM's own shape: a narrow output pads a wide
// tile, a short K loop is bound by the epilogue, a long one by the MMA feed.
// The tuner measures that instead of guessing: for every GEMM shape class it
// has not seen, it times a grouped launch of copies of one representative
// GEMM of the class at each candidate width (CUDA events, after a warm-up
// launch) and keeps the fastest.
//
// The choice is keyed by the GEMM's own shape class (stage, output width,
// rows, K, precision terms, operand layouts, triangular flags), never by the
// rest of the batch, so a decomposition gets the same tile widths alone or in
// any mix (and the width does not change any sum: each output element is
// accumulated over K in the same order whatever the tile's width).
//
// Results live in a process-wide table; with BCUR_AUTOTUNE_CACHE=<path> they
// are also read from and written back to a JSON file, so that later
// processes skip the measurements.  BCUR_AUTOTUNE=0 turns measuring off (the
// fixed widths are used for shapes not in the table).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"

namespace bcur {
namespace {

std::mutex g_mu;
std::map<std::string, int> g_table;
bool g_loaded = false;
int g_measured = 0;

const char* cache_path() {
  const char* p = getenv("BCUR_AUTOTUNE_CACHE");
  return (p && p[0]) ? p : nullptr;
}

bool tuning_on() {
  const char* e = getenv("BCUR_AUTOTUNE");
  return !(e && e[0] == '0');
}

std::string device_tag() {
  int dev = 0, sms = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return "sm?";
  }
  char b[48];
  snprintf(b, sizeof(b), "sm%d%dx%d", major, minor, sms);
  return b;
}

// The cache file is a flat JSON object {"key": width, ...}.  Keys contain
// only [A-Za-z0-9_|=.-], so the reader needs no escapes.
void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = cache_path();
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  fclose(f);
  size_t i = 0;
  while (true) {
    const size_t q0 = text.find('"', i);
    if (q0 == std::string::npos) break;
    const size_t q1 = text.find('"', q0 + 1);
    if (q1 == std::string::npos) break;
    const size_t colon = text.find(':', q1);
    if (colon == std::string::npos) break;
    const std::string key = text.substr(q0 + 1, q1 - q0 - 1);
    const int v = atoi(text.c_str() + colon + 1);
    if (v == 64 || v == 128 || v == 256) g_table[key] = v;
    i = colon + 1;
  }
}

void save_locked() {
  const char* path = cache_path();
  if (!path) return;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t j = 0;
  for (const auto& kv : g_table)
    fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++j < g_table.size() ? "," : "");
  fprintf(f, "}\n");
  fclose(f);
  rename(tmp.c_str(), path);
}

int64_t pow2_at_least(int64_t x, int64_t lo) {
  int64_t p = lo;
  while (p < x) p <<= 1;
  return p;
}

// Output width, rows and layout of the GEMM in MMA space (the kernel stores
// D^T when M < 128 and N >= 2M, so the long side runs along the tile rows).
void mma_space(const GemmDesc& d, int resid, int64_t* Mm, int64_t* Nm, int* swap) {
  *swap = (!resid && d.M < 128 && d.N >= 2 * d.M) ? 1 : 0;
  *Mm = *swap ? d.N : d.M;
  *Nm = *swap ? d.M : d.N;
}

}  // namespace

std::string tune_key(const char* stage, const GemmDesc& d, int resid) {
  int64_t Mm, Nm;
  int swap;
  mma_space(d, resid, &Mm, &Nm, &swap);
  const int64_t nb = Nm <= 512 ? (Nm + 63) / 64 * 64 : pow2_at_least(Nm, 1024);
  char b[200];
  snprintf(b, sizeof(b), "%s|%s|N=%lld|M=%lld|K=%lld|p=%d|t=%d%d%d|tri=%d%d%d", stage,
           device_tag().c_str(), (long long)nb, (long long)pow2_at_least(Mm, 128),
           (long long)pow2_at_least(d.K, 64), d.parts == 3 ? 3 : 1, d.transA ? 1 : 0,
           d.transB ? 1 : 0, swap, d.triA, d.triB, d.out_lower);
  return b;
}

int tune_fixed_bn(const GemmDesc& d, int resid) {
  int64_t Mm, Nm;
  int swap;
  mma_space(d, resid, &Mm, &Nm, &swap);
  return Nm <= 64 ? 64 : (Nm <= 128 ? 128 : 256);
}

bcur_status_t tune_widths(const char* stage, const std::vector<GemmDesc>& ds, int resid,
                          const std::vector<int>& cands, const TuneScratch& sc,
                          std::vector<int>* out) {
  out->assign(ds.size(), 0);
  std::lock_guard<std::mutex> lock(g_mu);
  load_locked();
  const bool measure = tuning_on() && sc.table && cands.size() > 1;
  bool changed = false;
  struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  cudaEvent_t& e0 = ev.a;
  cudaEvent_t& e1 = ev.b;
  for (size_t i = 0; i < ds.size(); ++i) {
    const std::string key = tune_key(stage, ds[i], resid);
    auto it = g_table.find(key);
    if (it != g_table.end()) { (*out)[i] = it->second; continue; }
    int pick = cands.size() == 1 ? cands[0] : tune_fixed_bn(ds[i], resid);
    if (std::find(cands.begin(), cands.end(), pick) == cands.end()) pick = cands.back();
    if (measure) {
      if (!e0) {
        BCUR_CUDA_TRY(cudaEventCreate(&e0));
        BCUR_CUDA_TRY(cudaEventCreate(&e1));
      }
      // Copies of the representative GEMM, enough for about two waves of
      // persistent CTAs at the widest candidate (they all write the same
      // output: only the time is kept).
      const int64_t units = std::max<int64_t>(1, gemm_tc_units(ds[i], resid, 256));
      int copies = (int)std::min<int64_t>(
          64, std::max<int64_t>(1, (2 * (int64_t)sc.sms + units - 1) / units));
      while (copies > 1 && gemm_tc_group_bytes(copies) > sc.table_bytes) copies /= 2;
      std::vector<GemmDesc> rep(copies, ds[i]);
      for (auto& r : rep) {
        r.status = sc.status;
        r.run_flag = nullptr;    // a conditional GEMM is timed as if it runs,
        r.parts_flag = nullptr;  // with all the terms its class names
      }
      std::vector<std::pair<int, float>> timed;
      for (int bn : cands) {
        TcGroup g;
        if (gemm_tc_group_prepare(rep.data(), copies, resid, bn, sc.table, sc.table_bytes,
                                  sc.status, &g, sc.stream) != BCUR_OK)
          continue;
        BCUR_TRY(gemm_tc_group_run(g, sc.stream));  // warm-up
        BCUR_CUDA_TRY(cudaEventRecord(e0, sc.stream));
        for (int r = 0; r < 3; ++r) BCUR_TRY(gemm_tc_group_run(g, sc.stream));
        BCUR_CUDA_TRY(cudaEventRecord(e1, sc.stream));
        BCUR_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        BCUR_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        timed.push_back({bn, ms});
      }
      if (!timed.empty()) {
        // the widest tile within 3% of the fastest (fewer tiles and epilogues)
        float best = timed[0].second;
        for (const auto& t : timed) best = std::min(best, t.second);
        int widest = 0;
        for (const auto& t : timed)
          if (t.second <= 1.03f * best) widest = std::max(widest, t.first);
        pick = widest;
      }
      ++g_measured;
      g_table[key] = pick;
      changed = true;
    }
    (*out)[i] = pick;
  }
  if (changed) save_locked();
  return BCUR_OK;
}

int tune_measured_count() {
  std::lock_guard<std::mutex> lock(g_mu);
  return g_measured;
}

}  // namespace bcur

extern "C" int32_t bcur_autotune_measured(void) { return bcur::tune_measured_count(); }
