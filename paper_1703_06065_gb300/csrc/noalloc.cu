// Frobenius residual without any device allocation.
//
// bcur_residual needs a caller-provided scratch buffer for its per-CTA
// partial sums.  Some callers cannot provide one: code that runs while every
// byte of device memory is owned by another framework's pool, latency-bound
// request loops that must not call cudaMalloc/cudaFree (cudaFree synchronises
// the whole device), and plug-ins that are handed only input and output
// pointers.  For them this file keeps the partial sums in a fixed array that
// lives in the library's own device image, so a call touches no allocator.
#include <algorithm>
#include <mutex>

#include "kernels.h"

namespace bcur {
namespace {

// Largest number of per-CTA partial pairs one call can reduce.  Two doubles
// per CTA: 1 MiB of device memory on every GPU that loads this library, held
// until the process exits.
constexpr int64_t kMaxPartials = 65536;
static __device__ __align__(256) double g_residual_scratch[2 * kMaxPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
struct Cached {
  void* ctx = nullptr;   // context the address was looked up in
  double* addr = nullptr;
};
Cached g_scratch_addr[kMaxDevices];

using CtxGetCurrentFn = int (*)(void**);  // cuCtxGetCurrent(CUcontext*)
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(ptr);
    else
      cudaGetLastError();
  });
  return fn;
}

// Device address of the array for the current device.  The name above is only
// a host-side stand-in; the address must come from the runtime, with that
// device current.  It is looked up once per device and again whenever the
// device's current context has changed since (after cudaDeviceReset the
// module is loaded anew, possibly at another address).
bcur_status_t scratch_address(double** out) {
  int dev = 0;
  BCUR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return BCUR_ENOTSUP;
  auto current = []() -> void* {
    void* ctx = nullptr;
    if (auto fn = ctx_get_current()) {
      if (fn(&ctx) != 0) ctx = nullptr;
    }
    return ctx;
  };
  void* ctx = current();
  std::lock_guard<std::mutex> lock(g_mutex);
  Cached& c = g_scratch_addr[dev];
  if (c.addr == nullptr || ctx == nullptr || c.ctx != ctx) {
    void* p = nullptr;
    BCUR_CUDA_TRY(cudaGetSymbolAddress(&p, g_residual_scratch));
    c.addr = static_cast<double*>(p);
    c.ctx = current();  // the lookup makes the device's primary context current
  }
  *out = c.addr;
  return BCUR_OK;
}

}  // namespace
}  // namespace bcur

using namespace bcur;

extern "C" bcur_status_t bcur_residual_noalloc(const void* X, int64_t ldx, const void* P,
                                               int64_t ldp, const void* Q, int64_t ldq, int64_t m,
                                               int64_t n, int64_t r, int32_t dtype, int32_t prec,
                                               double* out, void* stream) {
  if (!X || !out || m < 1 || n < 1 || r < 0) return BCUR_EINVAL;
  if (r > 0 && (!P || !Q)) return BCUR_EINVAL;
  if (ldx < n || ldp < r || ldq < n) return BCUR_EINVAL;
  if (dtype == BCUR_F64 && prec != BCUR_F64) return BCUR_EINVAL;
  if (dtype == BCUR_F32 && (prec < BCUR_F32 || prec > BCUR_BF16)) return BCUR_EINVAL;
  if (dtype == BCUR_BF16 && prec != BCUR_BF16) return BCUR_EINVAL;
  if (dtype != BCUR_F64 && dtype != BCUR_F32 && dtype != BCUR_BF16) return BCUR_EINVAL;
  // Every kernel that may serve the call must fit its partials in the array.
  int64_t need = 0;
  if (dtype == BCUR_F64) {
    need = gemm_simt_resid_ctas<double>(m, n);
  } else if (dtype == BCUR_BF16) {
    need = gemm_tc_resid_ctas(m, n);
  } else {
    need = gemm_simt_resid_ctas<float>(m, n);
    if (prec != BCUR_F32) need = std::max(need, gemm_tc_resid_ctas(m, n));
  }
  if (need > kMaxPartials) return BCUR_ENOMEM;

  double* scratch = nullptr;
  BCUR_TRY(scratch_address(&scratch));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GemmDesc g;
  g.M = m; g.N = n; g.K = r;
  g.A = P; g.lda = ldp; g.transA = 0;
  g.B = Q; g.ldb = ldq; g.transB = 0;
  g.X = X; g.ldx = ldx;
  g.partials = scratch;
  int64_t np = 0;
  if (dtype == BCUR_F64) {
    BCUR_TRY(gemm_simt_resid<double>(g, s, &np));
  } else if (dtype == BCUR_BF16) {  // X FP32, P and Q BF16: tensor cores only
    g.ab_bf16 = 1;
    BCUR_TRY(gemm_tc_resid(g, prec, s, &np));
  } else {
    bcur_status_t st = BCUR_ENOTSUP;
    if (prec == BCUR_TF32 || prec == BCUR_BF16) st = gemm_tc_resid(g, prec, s, &np);
    if (st == BCUR_ENOTSUP) st = gemm_simt_resid<float>(g, s, &np);
    BCUR_TRY(st);
  }
  // Each CTA overwrote its own slot above, and the reduction reads exactly
  // those slots, so nothing left from an earlier call is ever read.
  return finish_residual(scratch, np, out, 1, s);
}
