// tcgen05 tensor-core GEMM (placeholder until the kernel lands).
#include "kernels.h"

namespace bcur {
bool gemm_tc_available() { return false; }
int64_t gemm_tc_resid_ctas(int64_t, int64_t) { return 0; }
bcur_status_t gemm_tc(const GemmDesc&, int, cudaStream_t) { return BCUR_ENOTSUP; }
bcur_status_t gemm_tc_resid(const GemmDesc&, int, cudaStream_t, int64_t*) { return BCUR_ENOTSUP; }
}  // namespace bcur
