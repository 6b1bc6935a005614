// Shared definitions for the Block CUR CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/bcur.h"

namespace bcur {

// Device-side status word values (a subset of bcur_status_t).
enum : int { kDevOk = 0 };

#define BCUR_CUDA_TRY(expr)                                                   \
  do {                                                                        \
    cudaError_t e__ = (expr);                                                 \
    if (e__ != cudaSuccess) {                                                 \
      bcur::set_last_cuda_error(e__, #expr, __FILE__, __LINE__);              \
      return BCUR_ECUDA;                                                      \
    }                                                                         \
  } while (0)

#define BCUR_LAUNCH_CHECK()                                                   \
  do {                                                                        \
    bcur::count_launch();                                                     \
    cudaError_t e__ = cudaGetLastError();                                     \
    if (e__ != cudaSuccess) {                                                 \
      bcur::set_last_cuda_error(e__, "kernel launch", __FILE__, __LINE__);    \
      return BCUR_ECUDA;                                                      \
    }                                                                         \
  } while (0)

#define BCUR_TRY(expr)                                                        \
  do {                                                                        \
    bcur_status_t s__ = (expr);                                               \
    if (s__ != BCUR_OK) return s__;                                           \
  } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
// Process-wide count of kernels this library has launched.
void count_launch();

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Record the first device-detected error into a status word.
__device__ __forceinline__ void dev_set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

}  // namespace bcur
