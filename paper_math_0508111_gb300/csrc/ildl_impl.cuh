// Internal state of a preconditioner handle.
#pragma once
#include <cstring>

#include "common.cuh"
#include "ildl_setup.h"

namespace ajd {

// A binary64 value stored as its upper 32 bits (sign, 11-bit exponent, 20
// mantissa bits), rounded to nearest-even from the full value: half the
// bytes of a binary64 entry, the full binary64 range, 21 significant bits,
// and widening back to binary64 is a register move (no conversion
// instruction).  Used for the factor values of the mixed apply.
struct hi32_t {
  unsigned u = 0;
  hi32_t() = default;
  explicit hi32_t(double x) {
    uint64_t b;
    std::memcpy(&b, &x, sizeof(b));
    b += 0x7FFFFFFFull + ((b >> 32) & 1ull);  // round the dropped low word, ties to even
    u = (unsigned)(b >> 32);
  }
};

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
  unsigned* bar = nullptr;  // [0] arrivals, [32] generation, [64] timeout flag
  int grid = 0;
  double* w64 = nullptr;  // binary64 work vectors of the mixed apply (hi32_t factor)
  double* z64 = nullptr;
};

}  // namespace ajd

struct ildl_s {
  ajd::HostFactor F;
  int device = 0;
  ajd::DevFactor<double> d64;
  ajd::DevFactor<float> d32;
  ajd::DevFactor<ajd::hi32_t> dh;  // mixed apply: binary64 sums over hi32_t values
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

// x = K^{-1} b with the factor values stored as hi32_t, binary64 vectors
// and sums.
int ildl_apply_dev_mixed(const ildl_s* f, const double* b, double* out, cudaStream_t stream);

// Device copies of a factor: binary64, binary32, mixed (hi32_t values).
constexpr int kCopyF64 = 1, kCopyF32 = 2, kCopyMixed = 4, kCopyAll = 7;

// The copy a solve in `precision` (JD_FP64, JD_FP32, JD_MIXED) applies.
inline int copy_for_precision(int precision) {
  return precision == JD_FP32 ? kCopyF32 : precision == JD_MIXED ? kCopyMixed : kCopyF64;
}

// ildl_create with its device work on stream `st`, uploading only the
// device copies in `copies`.
int ildl_create_on_stream(anderson_t h, double sigma, const ildl_params* p, ildl_t* out, cudaStream_t st,
                          int copies = kCopyAll);

// JD_EDEVICE if a device-side wait of an apply timed out (reads a flag).
int ildl_check_device_error(const ildl_s* f);

}  // namespace ajd
