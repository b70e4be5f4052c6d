// Shared helpers of the GPU library: error reporting across the C ABI,
// CUDA call checking, small device utilities.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstdarg>
#include <string>

#include "anderson_jd.h"

namespace ajd {

// Thread-local message behind jd_last_error().
void set_error_msg(const char* fmt, ...);

// Record an error message and return the code (for `return fail(...)`).
int fail(int code, const char* fmt, ...);

}  // namespace ajd

// Evaluate a CUDA runtime call; on failure record the message and return
// JD_EDEVICE from the enclosing int-returning function.
#define AJD_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      return ::ajd::fail(JD_EDEVICE, "%s:%d %s: %s", __FILE__, __LINE__,      \
                         #call, cudaGetErrorString(e_));                      \
    }                                                                         \
  } while (0)

// Propagate a non-zero status code.
#define AJD_TRY(expr)                                                         \
  do {                                                                        \
    int ajd_rc_ = (expr);                                                     \
    if (ajd_rc_ != JD_OK) return ajd_rc_;                                     \
  } while (0)

#define AJD_CHECK_LAUNCH() AJD_CUDA(cudaGetLastError())

namespace ajd {

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Number of SMs of the current device (cached per process; one GPU).
int sm_count();

// Kernel launches issued by this library on the calling thread (monotone).
int64_t& launch_counter();
inline void count_launches(int k = 1) { launch_counter() += k; }

}  // namespace ajd
