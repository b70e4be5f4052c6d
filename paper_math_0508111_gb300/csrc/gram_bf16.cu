// First pass of the block Gram-Schmidt of the search-space expansion
// (Section 4.2: t is orthogonalised against [Q, V] before it extends V) on
// the 5th-generation tensor cores: the projection c = Xb^T tb with Xb a BF16
// shadow of the columns of [Q, V] and tb = BF16(t), FP32 accumulation in
// tensor memory -- a quarter of the bytes of the binary64 projection.  The
// update t -= X c uses the binary64 columns (jd.cu), so the BF16 error of c
// stays inside span(X), and the second, binary64 pass removes it.
//
// gram_bf16_kernel: each CTA (128 threads) walks a slab of rows in chunks of
// 64.  Per chunk the A operand (the columns as rows: up to 128 x 64 BF16, the
// matrix X^T, K-major) and the B operand (tb as the first of 16 rows, the
// rest zero) are written to shared memory in the canonical no-swizzle
// K-major layout -- 8-row x 16-byte core matrices, K-adjacent ones 128 B
// apart, 8-row groups 1024 B apart -- and one thread issues four
// tcgen05.mma (M = 128, N = 16, K = 16 each) accumulating into tensor memory;
// tcgen05.commit signals an mbarrier when they are done with the buffer
// (two buffers alternate).  At the end each warp reads its 32 rows of the
// accumulator (tcgen05.ld) and writes the CTA's partial sums.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "gram_bf16.h"

namespace ajd {
namespace {

constexpr int kGramThreads = 128;
constexpr int kGramChunk = 64;    // rows (the K extent) per chunk
constexpr int kGramM = 128;       // columns of X handled (MMA M)
constexpr int kGramN = 16;        // MMA N (tb plus 15 zero rows)
constexpr int kATileBytes = kGramM * kGramChunk * 2;  // 16 KiB
constexpr int kBTileBytes = kGramN * kGramChunk * 2;  // 2 KiB
constexpr unsigned kGramSpinLimit = 1u << 24;

// instruction descriptor of tcgen05.mma kind::f16: D in FP32, A and B BF16,
// both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kGramN >> 3) << 17) |
                            ((uint32_t)(kGramM >> 4) << 24);

// shared-memory matrix descriptor: no swizzle, K-adjacent core matrices 128 B
// apart (leading byte offset), 8-row groups 1024 B apart (stride byte
// offset), descriptor version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46);
}

// byte offset of element (row, k) of a K-major tile in the canonical layout
__device__ __forceinline__ int tile_off(int row, int k) {
  return ((row >> 3) * 8 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (unsigned it = 0; it < kGramSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// X = [X1 X2]: the first c1 columns from X1, the next c2 from X2 (the locked
// vectors Q and the search space V), both with leading dimension ldb
__global__ void __launch_bounds__(kGramThreads)
gram_bf16_kernel(const __nv_bfloat16* __restrict__ X1, int c1, const __nv_bfloat16* __restrict__ X2, int c2,
                 int64_t ldb, const double* __restrict__ t, int64_t n, int64_t rows_per_cta,
                 double* __restrict__ partial, int* __restrict__ err) {
  const int c = c1 + c2;
  __shared__ __align__(1024) unsigned char sA[2][kATileBytes];
  __shared__ __align__(1024) unsigned char sB[2][kBTileBytes];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // zero both buffers: the rows of A beyond c and the rows 1..15 of B stay 0
  for (int i = tid; i < 2 * kATileBytes / 16; i += kGramThreads) reinterpret_cast<uint4*>(&sA[0][0])[i] = uint4{0, 0, 0, 0};
  for (int i = tid; i < 2 * kBTileBytes / 16; i += kGramThreads) reinterpret_cast<uint4*>(&sB[0][0])[i] = uint4{0, 0, 0, 0};
  const uint32_t mbar0 = (uint32_t)__cvta_generic_to_shared(&mbar[0]);
  const uint32_t mbar1 = (uint32_t)__cvta_generic_to_shared(&mbar[1]);
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_tmem);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(dst) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = std::min<int64_t>(n, r0 + rows_per_cta);
  const int nchunks = r1 > r0 ? (int)((r1 - r0 + kGramChunk - 1) / kGramChunk) : 0;
  // the next chunk's operands are loaded into registers while the tensor
  // cores work on the current one: A as 16-byte pieces (8 rows of one
  // column of X; the shadow is zero-padded to ldb), B as one value of t
  constexpr int kPieces = kGramM * 8 / kGramThreads;  // 16-byte pieces per thread
  uint4 pre[kPieces];
  double tv = 0.0;
  auto load_chunk = [&](int k) {
    const int64_t i0 = r0 + (int64_t)k * kGramChunk;
#pragma unroll
    for (int q = 0; q < kPieces; ++q) {
      const int idx = tid + q * kGramThreads;
      if (idx < c * 8) {
        const int j = idx >> 3, kk = (idx & 7) * 8;
        const __nv_bfloat16* col = j < c1 ? X1 + (int64_t)j * ldb : X2 + (int64_t)(j - c1) * ldb;
        pre[q] = *reinterpret_cast<const uint4*>(col + i0 + kk);
      }
    }
    if (tid < kGramChunk) tv = i0 + tid < n ? t[i0 + tid] : 0.0;
  };
  if (nchunks > 0) load_chunk(0);
  for (int k = 0; k < nchunks; ++k) {
    const int buf = k & 1;
    const uint32_t mb = buf ? mbar1 : mbar0;
    if (k >= 2 && !mbar_wait(mb, (uint32_t)(((k - 2) >> 1) & 1))) {
      if (tid == 0) s_fail = 1;
    }
    __syncthreads();
    if (s_fail) break;
    // A: column j of X, rows of the chunk, as row j of the tile; B: tb as row 0
#pragma unroll
    for (int q = 0; q < kPieces; ++q) {
      const int idx = tid + q * kGramThreads;
      if (idx < c * 8) *reinterpret_cast<uint4*>(&sA[buf][tile_off(idx >> 3, (idx & 7) * 8)]) = pre[q];
    }
    if (tid < kGramChunk) *reinterpret_cast<__nv_bfloat16*>(&sB[buf][tile_off(0, tid)]) = __double2bfloat16(tv);
    // the generic-proxy writes above become visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (k + 1 < nchunks) load_chunk(k + 1);
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(&sA[buf][0]);
      const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(&sB[buf][0]);
#pragma unroll
      for (int ks = 0; ks < kGramChunk / 16; ++ks) {
        const uint64_t ad = smem_desc(a0 + ks * 256), bd = smem_desc(b0 + ks * 256);
        const uint32_t acc = (k > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
    }
  }
  // the last commit covers every MMA of this CTA
  if (nchunks > 0 && !s_fail) {
    const int kl = nchunks - 1;
    if (!mbar_wait((kl & 1) ? mbar1 : mbar0, (uint32_t)((kl >> 1) & 1)) && tid == 0) s_fail = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  float v = 0.f;
  if (nchunks > 0 && !s_fail) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    v = __uint_as_float(r);
  }
  const int j = warp * 32 + lane;
  if (j < c) partial[(int64_t)blockIdx.x * c + j] = (double)v;
  if (tid == 0 && s_fail) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

// out[j] = sum over the CTAs' partial sums (binary64, fixed order)
__global__ void gram_reduce_kernel(const double* __restrict__ partial, int nblocks, int c, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < c; j += nw) {
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partial[(int64_t)b * c + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[j] = s;
  }
}

// Xb[:, j] = BF16(X[:, j]) for columns j0 .. j1 - 1, rows n .. ldb - 1 zero
__global__ void to_bf16_kernel(const double* __restrict__ X, int64_t ldx, int j0, int j1, __nv_bfloat16* __restrict__ Xb,
                               int64_t ldb, int64_t n) {
  const int64_t total = (int64_t)(j1 - j0) * ldb;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int j = j0 + (int)(q / ldb);
    const int64_t i = q - (q / ldb) * ldb;
    Xb[(int64_t)j * ldb + i] = __double2bfloat16(i < n ? X[(int64_t)j * ldx + i] : 0.0);
  }
}

}  // namespace

int64_t gram_bf16_ld(int64_t n) { return (n + kGramChunk - 1) / kGramChunk * kGramChunk; }

int gram_bf16_max_cols() { return kGramM; }

int gram_bf16_convert(const double* X, int64_t ldx, int j0, int j1, void* Xb, int64_t ldb, int64_t n,
                      cudaStream_t s) {
  if (j1 <= j0) return JD_OK;
  const int grid = std::max(1, std::min(ceil_div((int64_t)(j1 - j0) * ldb, 256), 8 * sm_count()));
  to_bf16_kernel<<<grid, 256, 0, s>>>(X, ldx, j0, j1, static_cast<__nv_bfloat16*>(Xb), ldb, n);
  count_launches();
  AJD_CHECK_LAUNCH();
  return JD_OK;
}

int gram_bf16_dots(const void* X1, int c1, const void* X2, int c2, int64_t ldb, const double* t, int64_t n,
                   double* partial, int nparts, double* out, int* err, cudaStream_t s) {
  const int c = c1 + c2;
  if (c <= 0) return JD_OK;
  if (c > kGramM) return fail(JD_EINVAL, "gram_bf16: %d columns exceed %d", c, kGramM);
  // rows per CTA: a multiple of the chunk, spread over at most nparts CTAs
  int64_t per = (n + nparts - 1) / nparts;
  per = (per + kGramChunk - 1) / kGramChunk * kGramChunk;
  const int grid = (int)std::max<int64_t>(1, (n + per - 1) / per);
  gram_bf16_kernel<<<grid, kGramThreads, 0, s>>>(static_cast<const __nv_bfloat16*>(X1), c1,
                                                 static_cast<const __nv_bfloat16*>(X2), c2, ldb, t, n, per, partial,
                                                 err);
  gram_reduce_kernel<<<1, 256, 0, s>>>(partial, grid, c, out);
  count_launches(2);
  AJD_CHECK_LAUNCH();
  return JD_OK;
}

}  // namespace ajd

using namespace ajd;

extern "C" int jd_gram_bf16(const double* X, int64_t ldx, int c, const double* t, int64_t n, double* out,
                            void* stream) {
  if (!X || !t || !out || n < 1 || c < 0 || ldx < n)
    return fail(JD_EINVAL, "jd_gram_bf16: bad arguments");
  if (c > kGramM) return fail(JD_EINVAL, "jd_gram_bf16: at most %d columns", kGramM);
  if (c == 0) return JD_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t ldb = gram_bf16_ld(n);
  const int nparts = 4 * sm_count();
  void* Xb = nullptr;
  double *partial = nullptr, *dout = nullptr;
  int* err = nullptr;
  int rc = JD_OK;
  cudaError_t e = cudaMalloc(&Xb, (size_t)c * ldb * 2);
  if (e == cudaSuccess) e = cudaMalloc(&partial, sizeof(double) * (size_t)nparts * c);
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double) * c);
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e != cudaSuccess) rc = fail(JD_EDEVICE, "jd_gram_bf16: %s", cudaGetErrorString(e));
  if (rc == JD_OK) rc = gram_bf16_convert(X, ldx, 0, c, Xb, ldb, n, s);
  if (rc == JD_OK) rc = gram_bf16_dots(Xb, c, nullptr, 0, ldb, t, n, partial, nparts, dout, err, s);
  int herr = 0;
  if (rc == JD_OK) {
    e = cudaMemcpyAsync(out, dout, sizeof(double) * c, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = fail(JD_EDEVICE, "jd_gram_bf16: %s", cudaGetErrorString(e));
    else if (herr) rc = fail(JD_EDEVICE, "jd_gram_bf16: a tensor-core wait timed out");
  }
  cudaFree(Xb);
  cudaFree(partial);
  cudaFree(dout);
  cudaFree(err);
  return rc;
}
