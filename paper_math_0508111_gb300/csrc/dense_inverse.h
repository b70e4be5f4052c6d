// Device inverse of the preconditioner's dense trailing block.
#pragma once
#include <cuda_runtime.h>

namespace ajd {

// X = A^{-1} for the m x m row-major binary64 matrix A (device; overwritten),
// m <= 8192, by blocked Gauss-Jordan elimination with partial pivoting, then
// X symmetrised.  *bad (device, zeroed by the caller) is set to 1 on a zero
// or non-finite pivot.  Synchronises `st`.
int dense_inverse_device(double* A, double* X, int m, int* bad, cudaStream_t st);

}  // namespace ajd
