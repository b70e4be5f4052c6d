// Internal state of an Anderson lattice handle and the stencil launchers
// shared by the preconditioner and the eigensolver translation units.
#pragma once
#include "common.cuh"

struct anderson_s {
  int L = 0;
  int64_t n = 0;
  double W = 0.0;
  uint64_t seed = 0;
  int bc = JD_PERIODIC;
  int device = 0;
  double hop = -1.0;        // nearest-neighbour hopping of Eq. (1)
  double* eps64 = nullptr;  // on-site energies, binary64, device
  float* eps32 = nullptr;   // binary32 copy, device
  double max_abs_eps = 0.0;
  // off-diagonal model (Section 7): hopping of the bond from site s to its
  // +x/+y/+z neighbour at [3s + d] (0 for bonds a hard wall removes);
  // nullptr for Eq. (1), whose hopping is `hop` on every bond
  double* bond64 = nullptr;
  float* bond32 = nullptr;
  double max_abs_bond = 1.0;
  // Gershgorin bound max|diagonal| + 6 max|hopping|: the ||A|| of the
  // relative tolerances (6 + max|eps| for Eq. (1))
  double norm_bound() const { return max_abs_eps + 6.0 * max_abs_bond; }
};

namespace ajd {

// y = (A - shift I) x for m column-major vectors of length n (device
// pointers), on `stream`.  T is double or float.
template <typename T>
int stencil_apply(const anderson_s* h, T shift, const T* x, T* y, int m,
                  cudaStream_t stream);

}  // namespace ajd
