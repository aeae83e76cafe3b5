// common.cuh -- shared device/host helpers of the GB300 ensemble-SDE library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/sde.h"

namespace sde {

// Device-side error word bits (latched in the context, reported by
// sde_observables).
enum : uint32_t {
  kErrNonFinite = 1u,  // a path or oscillator state became NaN/Inf
  kErrTimeout = 2u,    // a bounded wait expired
};

// Philox stream tags (fourth counter word), one per kind of draw.
enum : uint32_t {
  kTagJosephson = 1u,  // noise of Eq. 1: counter (n/4, path, point, 1)
  kTagKuramoto = 2u,   // noise of Eq. 2: counter (n/4, oscillator, replica, 2)
};

// Thread-local last-error message (sde_last_error).
void set_error(const std::string &msg);
void clear_error();

sde_status cuda_fail(cudaError_t e, const char *what);

// cudaMalloc of the library's workspaces, through the allocation-failure
// injection of sde_debug_fail_allocation.
cudaError_t device_alloc(void **p, size_t bytes);
// True when the injection says the allocation being made fails (abi.cu).
bool injected_alloc_failure();
// Disarm the injection (the end of every create call).
void alloc_injection_disarm();

#define SDE_CUDA_TRY(expr)                                    \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return ::sde::cuda_fail(e_, #expr); \
  } while (0)

#define SDE_CHECK_ARG(cond, msg)                 \
  do {                                           \
    if (!(cond)) {                               \
      ::sde::set_error(std::string("invalid argument: ") + (msg)); \
      return SDE_ERR_INVALID_ARG;                \
    }                                            \
  } while (0)

inline int ceil_div_i64(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace sde
