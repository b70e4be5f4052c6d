// Inverse of the preconditioner's dense trailing block on the device:
// Gauss-Jordan elimination with partial pivoting (rows), in panels of
// kGjPanel columns.
//
// The augmented matrix [A | X] (m x 2m, row-major, X = I at the start) is
// reduced to [I | A^{-1}].  For a panel of w columns c0..c0+w-1:
//   1. gj_panel_kernel, one thread-block cluster of kGjCluster CTAs (each
//      owning a contiguous range of rows): for each column c of the panel,
//      the pivot is the largest |A[r][c]|, r >= c (lowest row on ties; each
//      CTA's candidate goes to the others through distributed shared
//      memory), rows c and the pivot row are swapped, row c is scaled by
//      1/pivot and every other row r loses A[r][c] times row c -- on the
//      panel's columns only.  The same steps are applied to H, an m x w
//      record of the transformation: column k of H starts as the unit vector
//      e_c when column c = c0 + k is pivoted, so that in the end H holds the
//      pivot columns of the whole panel's elimination E (E differs from I
//      only there, once the swaps are taken out in front; a swap of rows c
//      and p >= c commutes past the earlier steps when it also swaps their
//      rows of H).  Two cluster barriers per column; no other waits.
//   2. gj_swap_kernel: the panel's swaps, in order, on every other column of
//      [A | X] (A's columns right of the panel and all of X; the columns
//      left of it are unit vectors with zeros in the swapped rows).
//   3. gj_rows_kernel copies the panel's pivot rows R of those columns.
//   4. gj_update_kernel: M <- M + (H - I_P) R on those columns (a rank-w
//      update, tiled through shared memory, column tiles whose R is zero
//      skipped -- most of X early on); pivot rows become H R.
// Per panel four launches instead of two per column, and the trailing
// update reads and writes each element once per panel instead of once per
// column.  Ordinary launches (the cluster needs 8 SMs), so the setup of one
// problem shares the GPU with the solves of others.  A zero or non-finite
// pivot sets *bad.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include <cooperative_groups.h>

#include "common.cuh"
#include "dense_inverse.h"

namespace cg = cooperative_groups;

namespace ajd {
namespace {

constexpr int kGjPanel = 32;    // columns per panel
constexpr int kGjCluster = 8;   // CTAs of the panel kernel (one cluster)
constexpr int kGjThreads = 512;
constexpr int kGjMaxRowsPerCta = 1024;  // rows of one CTA: m <= 8 * 1024 (the dense tail is at most 8000 rows)

__device__ __forceinline__ bool better(double v, int i, double bv, int bi) {
  // larger |value| first, then the lower row; i < 0: no candidate
  if (i < 0) return false;
  if (bi < 0) return true;
  const double a = fabs(v), b = fabs(bv);
  return a > b || (a == b && i < bi);
}

__global__ void __cluster_dims__(kGjCluster, 1, 1) __launch_bounds__(kGjThreads)
gj_panel_kernel(double* __restrict__ A, int m, int c0, int w, double* __restrict__ H, int* __restrict__ piv,
                int* __restrict__ bad) {
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int r0 = (int)((int64_t)m * q / kGjCluster), r1 = (int)((int64_t)m * (q + 1) / kGjCluster);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double s_bv;  // this CTA's pivot candidate (read by the others)
  __shared__ int s_bi;
  __shared__ double wv[kGjThreads / 32];
  __shared__ int wi[kGjThreads / 32];
  __shared__ double s_pc[2 * kGjPanel];  // old row c: panel columns, then H
  __shared__ double s_pp[2 * kGjPanel];  // old pivot row
  __shared__ int s_piv;
  __shared__ double s_inv;
  __shared__ double s_f[kGjMaxRowsPerCta];  // the multipliers of this CTA's rows
  for (int64_t t = (int64_t)r0 * kGjPanel + threadIdx.x; t < (int64_t)r1 * kGjPanel; t += blockDim.x) H[t] = 0.0;
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    const int c = c0 + k;
    // 1. this CTA's candidate among its rows r >= c
    double bv = 0.0;
    int bi = -1;
    for (int r = max(r0, c) + threadIdx.x; r < r1; r += blockDim.x) {
      const double a = A[(int64_t)r * m + c];
      if (better(a, r, bv, bi)) { bv = a; bi = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (better(v2, i2, bv, bi)) { bv = v2; bi = i2; }
    }
    if (lane == 0) { wv[warp] = bv; wi[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = 0.0;
      int i = -1;
      for (int j = 0; j < kGjThreads / 32; ++j)
        if (better(wv[j], wi[j], b, i)) { b = wv[j]; i = wi[j]; }
      s_bv = b;
      s_bi = i;
    }
    // the candidates, and every row written in the previous step, visible
    // to the whole cluster
    cluster.sync();
    if (threadIdx.x == 0) {
      double b = 0.0;
      int i = -1;
      for (int j = 0; j < kGjCluster; ++j) {
        const double* pv = cluster.map_shared_rank(&s_bv, j);
        const int* pi = cluster.map_shared_rank(&s_bi, j);
        if (better(*pv, *pi, b, i)) { b = *pv; i = *pi; }
      }
      const bool ok = i >= 0 && fabs(b) > 0.0 && isfinite(b);
      if (!ok && q == 0) *bad = 1;
      s_piv = i >= 0 ? i : c;
      s_inv = ok ? 1.0 / b : 1.0;
      if (q == 0) piv[k] = s_piv;
    }
    __syncthreads();
    const int pr = s_piv;
    const double inv = s_inv;
    // 2. the old rows c and pr (panel columns k..w-1, H columns 0..k-1)
    for (int j = threadIdx.x; j < 2 * kGjPanel; j += blockDim.x) {
      double vc = 0.0, vp = 0.0;
      if (j < kGjPanel) {
        if (j >= k && j < w) {
          vc = __ldcg(A + (int64_t)c * m + c0 + j);
          vp = __ldcg(A + (int64_t)pr * m + c0 + j);
        }
      } else if (j - kGjPanel < k) {
        vc = __ldcg(H + (int64_t)c * kGjPanel + (j - kGjPanel));
        vp = __ldcg(H + (int64_t)pr * kGjPanel + (j - kGjPanel));
      }
      s_pc[j] = vc;
      s_pp[j] = vp;
    }
    __syncthreads();
    // the multipliers f_r = A[r][c] of this CTA's rows (for the old row c,
    // which moves to pr: its own A[c][c]), read before any is overwritten
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x)
      s_f[r - r0] = (r == pr && r != c) ? s_pc[k] : A[(int64_t)r * m + c];
    // every CTA has read rows c and pr before their owners overwrite them
    cluster.sync();
    // 3. the new row c is the old pivot row with H's column k set to 1,
    //    scaled; every other row r loses f_r times it; column c of the
    //    others becomes exactly 0
    const int span = (w - k) + (k + 1);  // panel columns k..w-1, H columns 0..k
    for (int64_t t = threadIdx.x; t < (int64_t)(r1 - r0) * span; t += blockDim.x) {
      const int r = r0 + (int)(t / span);
      const int j = (int)(t % span);
      const bool in_a = j < w - k;
      const int ja = k + j;            // panel column (relative) when in_a
      const int jh = j - (w - k);      // H column otherwise
      // pivot-row value of this column
      const double prow =
          in_a ? __dmul_rn(s_pp[ja], inv) : __dmul_rn(jh < k ? s_pp[kGjPanel + jh] : 1.0, inv);
      if (r == c) {
        if (in_a) A[(int64_t)r * m + c0 + ja] = prow;
        else H[(int64_t)r * kGjPanel + jh] = prow;
        continue;
      }
      const bool moved = r == pr;  // holds the old row c
      const double f = s_f[r - r0];
      if (!moved && f == 0.0) continue;
      double old;
      if (in_a) old = moved ? s_pc[ja] : A[(int64_t)r * m + c0 + ja];
      else old = moved ? (jh < k ? s_pc[kGjPanel + jh] : 0.0) : H[(int64_t)r * kGjPanel + jh];
      const double nv = (in_a && ja == k) ? 0.0 : __dsub_rn(old, __dmul_rn(f, prow));
      if (in_a) A[(int64_t)r * m + c0 + ja] = nv;
      else H[(int64_t)r * kGjPanel + jh] = nv;
    }
    __syncthreads();
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// Apply the panel's swaps (rows c0 + k <-> piv[k], k = 0..w-1, in order) to
// the columns of [A | X] outside the panel: A's columns c0 + w .. m-1 and all
// of X's; one thread per column.
__global__ void gj_swap_kernel(double* __restrict__ A, double* __restrict__ X, int m, int c0, int w,
                               const int* __restrict__ piv) {
  const int na = m - (c0 + w);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < na + m; t += gridDim.x * blockDim.x) {
    double* col = t < na ? A + c0 + w + t : X + (t - na);
    for (int k = 0; k < w; ++k) {
      const int c = c0 + k, p = piv[k];
      if (p == c) continue;
      const double a = col[(int64_t)c * m], b = col[(int64_t)p * m];
      col[(int64_t)c * m] = b;
      col[(int64_t)p * m] = a;
    }
  }
}

// R[k][t] = row c0 + k of the columns outside the panel (t < na: A's column
// c0 + w + t; else X's column t - na); R has kGjPanel rows of na + m.
__global__ void gj_rows_kernel(const double* __restrict__ A, const double* __restrict__ X, int m, int c0, int w,
                               double* __restrict__ R) {
  const int na = m - (c0 + w), width = na + m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)w * width;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / width), j = (int)(t % width);
    const int64_t row = (int64_t)(c0 + k) * m;
    R[(int64_t)k * width + j] = j < na ? A[row + c0 + w + j] : X[row + (j - na)];
  }
}

// M[r][j] = (r a pivot row ? 0 : M[r][j]) + sum_k H[r][k] R[k][j] on the
// columns outside the panel; 64 x 64 tiles, each thread 4 x 4 outputs.
constexpr int kTile = 64;
__global__ void __launch_bounds__(256)
gj_update_kernel(double* __restrict__ A, double* __restrict__ X, int m, int c0, int w,
                 const double* __restrict__ H, const double* __restrict__ R) {
  __shared__ double sh[kTile][kGjPanel + 1];
  __shared__ double sr[kGjPanel][kTile];
  __shared__ int s_any;
  const int na = m - (c0 + w), width = na + m;
  const int tiles_c = (width + kTile - 1) / kTile, tiles_r = (m + kTile - 1) / kTile;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int tile = blockIdx.x; tile < tiles_c * tiles_r; tile += gridDim.x) {
    const int tr = tile / tiles_c, tc = tile % tiles_c;
    const int rb = tr * kTile, cb = tc * kTile;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    bool nz = false;
    for (int t = threadIdx.x; t < kGjPanel * kTile; t += blockDim.x) {
      const int k = t / kTile, j = t % kTile;
      const double v = (k < w && cb + j < width) ? R[(int64_t)k * width + cb + j] : 0.0;
      sr[k][j] = v;
      nz |= v != 0.0;
    }
    for (int t = threadIdx.x; t < kTile * kGjPanel; t += blockDim.x) {
      const int i = t / kGjPanel, k = t % kGjPanel;
      sh[i][k] = (k < w && rb + i < m) ? H[(int64_t)(rb + i) * kGjPanel + k] : 0.0;
    }
    if (nz) s_any = 1;
    __syncthreads();
    const bool any = s_any != 0;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    if (any) {
      for (int k = 0; k < w; ++k) {
        double hv[4], rv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) hv[a] = sh[ty * 4 + a][k];
#pragma unroll
        for (int b = 0; b < 4; ++b) rv[b] = sr[k][tx * 4 + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(hv[a], rv[b], acc[a][b]);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = rb + ty * 4 + a;
      if (r >= m) continue;
      const bool pivot_row = r >= c0 && r < c0 + w;
      if (!any && !pivot_row) continue;  // zero update
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int j = cb + tx * 4 + b;
        if (j >= width) continue;
        double* p = j < na ? A + (int64_t)r * m + c0 + w + j : X + (int64_t)r * m + (j - na);
        *p = pivot_row ? acc[a][b] : *p + acc[a][b];
      }
    }
    __syncthreads();  // sh, sr reused by the next tile
  }
}

__global__ void gj_identity_kernel(double* __restrict__ X, int m) {
  const int64_t total = (int64_t)m * m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    X[t] = (t / m == t % m) ? 1.0 : 0.0;
}

__global__ void gj_symmetrize_kernel(double* __restrict__ X, int m) {
  const int64_t total = (int64_t)m * m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / m), j = (int)(t % m);
    if (j <= i) continue;
    const double sym = 0.5 * (X[(int64_t)i * m + j] + X[(int64_t)j * m + i]);
    X[(int64_t)i * m + j] = sym;
    X[(int64_t)j * m + i] = sym;
  }
}

}  // namespace

int dense_inverse_device(double* A, double* X, int m, int* bad, cudaStream_t st) {
  if (m <= 0) return JD_OK;
  double *H = nullptr, *R = nullptr;
  int* piv = nullptr;
  cudaError_t e = cudaMalloc(&H, (size_t)m * kGjPanel * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&R, (size_t)kGjPanel * 2 * m * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&piv, kGjPanel * sizeof(int));
  int launches = 0;
  if (e == cudaSuccess) {
    const int gb = std::max(1, std::min(ceil_div((int64_t)m * m, 256), 8 * sm_count()));
    gj_identity_kernel<<<gb, 256, 0, st>>>(X, m);
    ++launches;
    for (int c0 = 0; c0 < m; c0 += kGjPanel) {
      const int w = std::min(kGjPanel, m - c0);
      const int na = m - (c0 + w), width = na + m;
      gj_panel_kernel<<<kGjCluster, kGjThreads, 0, st>>>(A, m, c0, w, H, piv, bad);
      gj_swap_kernel<<<std::max(1, std::min(ceil_div(width, 256), 4 * sm_count())), 256, 0, st>>>(A, X, m, c0, w,
                                                                                                   piv);
      gj_rows_kernel<<<std::max(1, std::min(ceil_div((int64_t)w * width, 256), 4 * sm_count())), 256, 0, st>>>(
          A, X, m, c0, w, R);
      const int tiles = ceil_div(width, kTile) * ceil_div(m, kTile);
      gj_update_kernel<<<std::max(1, std::min(tiles, 4 * sm_count())), 256, 0, st>>>(A, X, m, c0, w, H, R);
      launches += 4;
    }
    gj_symmetrize_kernel<<<gb, 256, 0, st>>>(X, m);
    ++launches;
    count_launches(launches);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(H);
  cudaFree(R);
  cudaFree(piv);
  if (e != cudaSuccess) return fail(JD_EDEVICE, "ildl dense inverse: %s", cudaGetErrorString(e));
  return JD_OK;
}

}  // namespace ajd
