// First Gram-Schmidt pass on the tensor cores with BF16 operands
// (gram_bf16.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace ajd {

// Leading dimension (elements) of a BF16 shadow of n-row columns: n rounded
// up to the 64-row chunk of the projection kernel (the rows beyond n are 0).
int64_t gram_bf16_ld(int64_t n);

// Most columns one projection handles.
int gram_bf16_max_cols();

// Xb[:, j] = BF16(X[:, j]), j0 <= j < j1 (X binary64, leading dimension ldx).
int gram_bf16_convert(const double* X, int64_t ldx, int j0, int j1, void* Xb, int64_t ldb, int64_t n,
                      cudaStream_t s);

// out = [X1 X2]^T BF16(t) with BF16 columns (c1 + c2 <= max cols) and FP32
// tensor-core accumulation, summed over CTAs in binary64.  partial holds
// nparts * (c1 + c2) doubles; *err is set if a wait of the kernel timed out.
int gram_bf16_dots(const void* X1, int c1, const void* X2, int c2, int64_t ldb, const double* t, int64_t n,
                   double* partial, int nparts, double* out, int* err, cudaStream_t s);

}  // namespace ajd
