// Internal state of a preconditioner handle.
#pragma once
#include <cstring>

#include "common.cuh"
#include "ildl_setup.h"

namespace ajd {

// Device copy of a HostFactor in one precision.
template <typename T>
struct DevFactor {
  bool ready = false;
  int* perm = nullptr;
  T* scale = nullptr;
  int* Lptr = nullptr;
  int* Lcol = nullptr;
  T* Lval = nullptr;
  int* Uptr = nullptr;
  int* Ucol = nullptr;
  T* Uval = nullptr;
  T* dd = nullptr;
  T* dof = nullptr;
  int* partner = nullptr;
  T* dense = nullptr;
  T* w = nullptr;  // work vectors in position space
  T* z = nullptr;
  int4* phases = nullptr;  // persistent-apply phase list (kind, p0, p1, G)
  int nphase = 0;
  unsigned* bar = nullptr;   // [64] timeout flag of the apply's waits
  unsigned* done = nullptr;  // completion counters of the apply's phases
  int grid = 0;
  int4* units = nullptr;  // dataflow-apply unit segments (kind | G << 8, p0, p1, first unit)
  int nseg = 0;
  int nunits = 0;
  int form = 0;  // apply form: 0 level counters (phases), 1 dataflow (units)
  float2* wdf = nullptr;  // float-float work vectors of the mixed apply (binary32 copy only)
  float2* zdf = nullptr;
};

}  // namespace ajd

struct ildl_s {
  ajd::HostFactor F;
  int device = 0;
  ajd::DevFactor<double> d64;
  ajd::DevFactor<float> d32;  // also the mixed apply (float-float work vectors)
  template <typename T>
  const ajd::DevFactor<T>& dev() const {
    if constexpr (sizeof(T) == 8) return d64;
    else return d32;
  }
};

namespace ajd {

// x = K^{-1} b on `stream` (device pointers, n elements).
template <typename T>
int ildl_apply_dev(const ildl_s* f, const T* b, T* out, cudaStream_t stream);

// x = K^{-1} b with the binary32 factor, float-float work vectors and
// sums, binary64 b and x.
int ildl_apply_dev_mixed(const ildl_s* f, const double* b, double* out, cudaStream_t stream);

// Device copies of a factor: binary64, binary32 (which the mixed apply
// shares: binary32 values, float-float work vectors).
constexpr int kCopyF64 = 1, kCopyF32 = 2, kCopyAll = 3;

// The copy a solve in `precision` (JD_FP64, JD_FP32, JD_MIXED) applies.
inline int copy_for_precision(int precision) {
  return precision == JD_FP32 || precision == JD_MIXED ? kCopyF32 : kCopyF64;
}

// ildl_create with its device work on stream `st`, uploading only the
// device copies in `copies`.
int ildl_create_on_stream(anderson_t h, double sigma, const ildl_params* p, ildl_t* out, cudaStream_t st,
                          int copies = kCopyAll);

// JD_EDEVICE if a device-side wait of an apply timed out (reads a flag).
int ildl_check_device_error(const ildl_s* f, cudaStream_t s);

}  // namespace ajd
