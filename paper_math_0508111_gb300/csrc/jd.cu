// Jacobi–Davidson for the k eigenpairs of the Anderson matrix nearest sigma
// (Section 4.2), with the correction equation (4.1) solved by simplified QMR
// and the multilevel ILDL^T preconditioner of Sections 5-6.
//
// Division of work: every O(n) operation runs in the kernels of this file
// (or the stencil and preconditioner kernels): Gram–Schmidt, the Rayleigh
// quotient matrix H = V^T A V, Ritz vectors, residuals, restarts and every
// SQMR step.  The m x m (m <= 64) symmetric eigenproblem of H is solved by a
// one-CTA Jacobi kernel.  The host only sequences the steps and reads a few
// scalars back once per outer step (Ritz value, residual norm, convergence
// flags).  The outer quantities are binary64; the inner solve runs in the
// precision the caller selects.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>
#include <cstdio>
#include <cstdlib>
#include <limits>
#include <type_traits>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>

#include <omp.h>

#include "anderson_impl.cuh"
#include "ildl_impl.cuh"
#include "gram_bf16.h"
#include "jd_impl.cuh"

namespace ajd {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxCols = 160;  // columns of one multi-dot (k + jmax + 2)
constexpr int kMaxM = 64;      // largest Rayleigh–Ritz problem

int vec_blocks(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads * 4 - 1) / (kThreads * 4), 4 * sm_count()));
}

template <typename T>
struct Cols {
  const T* p = nullptr;
  int64_t ld = 0;
  int c = 0;
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// partial[b*ncols + j] = block b's share of (column j of [X1 X2 extra])^T v
template <typename T>
__global__ void __launch_bounds__(kThreads)
multidot_kernel(Cols<T> X1, Cols<T> X2, const T* __restrict__ extra, const T* __restrict__ v, int64_t n,
                double* __restrict__ partial, int ncols, const int* done) {
  if (done && *done) return;
  __shared__ double sh[kThreads / 32];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = 0; j < ncols; ++j) {
    const T* x;
    if (j < X1.c) x = X1.p + (int64_t)j * X1.ld;
    else if (j < X1.c + X2.c) x = X2.p + (int64_t)(j - X1.c) * X2.ld;
    else x = extra;
    T acc = T(0);
    for (int64_t i = i0; i < n; i += stride) acc += x[i] * v[i];
    const double s = block_sum((double)acc, sh);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * ncols + j] = s;
  }
}

// partial[b*ncols + j] = block b's share of (AV_j - sigma V_j)^T (AV_c - sigma V_c),
// j = 0..ncols-1, c = ncols - 1: the new column of G = W^T W, W = AV - sigma V,
// formed from the shifted vectors themselves (no cancellation of
// (AV)^T AV - 2 sigma V^T AV + sigma^2 I)
__global__ void __launch_bounds__(kThreads)
shifted_dots_kernel(const double* __restrict__ V, const double* __restrict__ AV, int64_t ld, int ncols,
                    double sigma, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[kThreads / 32];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = ncols - 1;
  for (int j = 0; j < ncols; ++j) {
    double acc = 0.0;
    for (int64_t i = i0; i < n; i += stride) {
      const double wc = AV[(int64_t)c * ld + i] - sigma * V[(int64_t)c * ld + i];
      const double wj = AV[(int64_t)j * ld + i] - sigma * V[(int64_t)j * ld + i];
      acc = fma(wj, wc, acc);
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * ncols + j] = s;
  }
}

// out[j] = sum_b partial[b*ncols + j]: one warp per column, lanes striding
// over the blocks, then a shuffle tree (fixed order, deterministic)
constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum_partials(const double* __restrict__ partial, int nblocks, int stride,
                                                    int j) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partial[(int64_t)b * stride + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

__global__ void __launch_bounds__(kRedThreads)
reduce_partials_kernel(const double* __restrict__ partial, int nblocks, int ncols, double* __restrict__ out,
                       const int* done) {
  if (done && *done) return;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < ncols; j += nw) {
    const double s = warp_sum_partials(partial, nblocks, ncols, j);
    if ((threadIdx.x & 31) == 0) out[j] = s;
  }
}

// v -= X1 h1 + X2 h2 (h from device memory), optionally y = alpha_scale * v
template <typename T>
__global__ void __launch_bounds__(kThreads)
multiaxpy_kernel(Cols<T> X1, Cols<T> X2, const double* __restrict__ h, T* __restrict__ v, int64_t n) {
  __shared__ double hs[kMaxCols];
  const int c = X1.c + X2.c;
  for (int j = threadIdx.x; j < c; j += blockDim.x) hs[j] = h[j];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T acc = v[i];
    for (int j = 0; j < X1.c; ++j) acc -= X1.p[(int64_t)j * X1.ld + i] * (T)hs[j];
    for (int j = 0; j < X2.c; ++j) acc -= X2.p[(int64_t)j * X2.ld + i] * (T)hs[X1.c + j];
    v[i] = acc;
  }
}

// out_j = sum_k X[:, k] Y[k, j] for j < mo (Y column-major with leading dim ldy);
// outputs in tiles of 8 so each row's X values are re-read from L1
__global__ void __launch_bounds__(kThreads)
lincomb_kernel(const double* __restrict__ X, int64_t ldx, int m, const double* __restrict__ Y, int ldy,
               int mo, double* __restrict__ out, int64_t ldo, int64_t n) {
  __shared__ double ys[kMaxM * kMaxM];
  for (int t = threadIdx.x; t < m * mo; t += blockDim.x) {
    const int k = t % m, j = t / m;
    ys[j * m + k] = Y[(int64_t)j * ldy + k];
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int j0 = 0; j0 < mo; j0 += 8) {
      double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      const int jn = min(8, mo - j0);
      for (int k = 0; k < m; ++k) {
        const double x = X[(int64_t)k * ldx + i];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          if (jj < jn) acc[jj] = fma(x, ys[(j0 + jj) * m + k], acc[jj]);
      }
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if (jj < jn) out[(int64_t)(j0 + jj) * ldo + i] = acc[jj];
    }
  }
}

// y = a * x with a = scal[ia] (or 1/sqrt(scal[ia]) when inv_sqrt)
__global__ void scale_copy_kernel(const double* __restrict__ x, double* __restrict__ y, int64_t n,
                                  const double* __restrict__ scal, int ia, int inv_sqrt) {
  double a = scal[ia];
  if (inv_sqrt) a = 1.0 / sqrt(a);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// r = Au - theta u with theta = scal[0]
__global__ void residual_kernel(const double* __restrict__ Au, const double* __restrict__ u,
                                const double* __restrict__ theta, double* __restrict__ r, int64_t n) {
  const double th = *theta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = Au[i] - th * u[i];
}

template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ x, D* __restrict__ y, int64_t n, double a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (D)(a * (double)x[i]);
}

// start vector: uniform in [-1/2, 1/2) from SplitMix64 (counter form)
__global__ void random_kernel(double* __restrict__ v, int64_t n, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + ((uint64_t)i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = (double)(z >> 11) * 0x1.0p-53 - 0.5;
  }
}

// H[:, col] and H[col, :] from the dot results (symmetric), ld = ldh
__global__ void set_h_column_kernel(double* __restrict__ H, int ldh, int col, const double* __restrict__ d) {
  for (int i = threadIdx.x; i <= col; i += blockDim.x) {
    double v = d[i];
    H[(int64_t)col * ldh + i] = v;
    H[(int64_t)i * ldh + col] = v;
  }
}

// Symmetric eigenproblem of H (m x m, m <= kMaxM) by the cyclic Jacobi method
// with the round-robin (tournament) ordering, m/2 rotations per round applied
// in parallel.  Output: theta[j] and Y[:, j] ordered by |theta - sigma|
// (ties: theta ascending).
__global__ void __launch_bounds__(kThreads)
rr_eig_kernel(const double* __restrict__ H, int ldh, int m, double sigma, double* __restrict__ theta,
              double* __restrict__ Y, int ldy) {
  extern __shared__ double smem[];
  const int mp = (m + 1) & ~1;  // padded to even
  double* A = smem;             // mp x mp, column-major
  double* V = A + mp * mp;      // mp x mp
  double* cs = V + mp * mp;     // cos/sin per pair
  int* pr = reinterpret_cast<int*>(cs + mp);  // pairs
  __shared__ double red[kThreads / 32];
  __shared__ int stop;
  for (int t = threadIdx.x; t < mp * mp; t += blockDim.x) {
    const int i = t % mp, j = t / mp;
    A[t] = (i < m && j < m) ? 0.5 * (H[(int64_t)j * ldh + i] + H[(int64_t)i * ldh + j]) : 0.0;
    V[t] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int half = mp / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, fro = 0.0;
    for (int t = threadIdx.x; t < mp * mp; t += blockDim.x) {
      const int i = t % mp, j = t / mp;
      fro += A[t] * A[t];
      if (i != j) off += A[t] * A[t];
    }
    off = block_sum(off, red);
    __syncthreads();
    fro = block_sum(fro, red);
    if (threadIdx.x == 0) stop = (off <= 1e-30 * fro) || fro == 0.0;
    __syncthreads();
    if (stop) break;
    for (int round = 0; round < mp - 1; ++round) {
      // pairs of the circle method: index 0 fixed, others rotate
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        auto pos = [&](int q) { return q == 0 ? 0 : ((q - 1 + round) % (mp - 1)) + 1; };
        int p = pos(k), q = pos(mp - 1 - k);
        if (p > q) { int tmp = p; p = q; q = tmp; }
        pr[2 * k] = p;
        pr[2 * k + 1] = q;
        const double apq = A[q * mp + p];
        double c = 1.0, s = 0.0;
        if (p < m && q < m && apq != 0.0) {
          const double tau = (A[q * mp + q] - A[p * mp + p]) / (2.0 * apq);
          double t;
          if (fabs(tau) > 1e150) t = 0.5 / tau;
          else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int t = threadIdx.x; t < half * mp; t += blockDim.x) {
        const int k = t / mp, i = t % mp;
        const int p = pr[2 * k], q = pr[2 * k + 1];
        const double c = cs[2 * k], s = cs[2 * k + 1];
        const double ap = A[p * mp + i], aq = A[q * mp + i];
        A[p * mp + i] = c * ap - s * aq;
        A[q * mp + i] = s * ap + c * aq;
        const double vp = V[p * mp + i], vq = V[q * mp + i];
        V[p * mp + i] = c * vp - s * vq;
        V[q * mp + i] = s * vp + c * vq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int t = threadIdx.x; t < half * mp; t += blockDim.x) {
        const int k = t / mp, j = t % mp;
        const int p = pr[2 * k], q = pr[2 * k + 1];
        const double c = cs[2 * k], s = cs[2 * k + 1];
        const double ap = A[j * mp + p], aq = A[j * mp + q];
        A[j * mp + p] = c * ap - s * aq;
        A[j * mp + q] = s * ap + c * aq;
      }
      __syncthreads();
    }
  }
  // order by |theta - sigma|, then theta: rank of each eigenvalue
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double ti = A[i * mp + i], di = fabs(ti - sigma);
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const double tj = A[j * mp + j], dj = fabs(tj - sigma);
      if (dj < di || (dj == di && (tj < ti || (tj == ti && j < i)))) ++rank;
    }
    theta[rank] = ti;
    for (int r = 0; r < m; ++r) Y[(int64_t)rank * ldy + r] = V[i * mp + r];
  }
}

// ---------------------------------------------------------------- SQMR ---
// scalar slots of the inner solver (double)
enum {
  S_RHO = 0, S_SIGMA, S_ALPHA, S_THETA, S_TAU, S_CD, S_CQ, S_BETA, S_BNORM, S_TOL, S_IT,
  S_NSCAL
};

// Projected matrix-vector step: after t = (A - theta^ I) q, dots[0..c) =
// Qt^T t and dots[c] = q^T t.  Then:
//   alpha = rho / sigma;  r -= alpha (t - Qt h);  partial ||r||^2
template <typename T>
__global__ void __launch_bounds__(kThreads)
sqmr_update_r_kernel(Cols<T> Qt, const double* __restrict__ dots, const T* __restrict__ t, T* __restrict__ r,
                     int64_t n, double* __restrict__ scal, double* __restrict__ partial, const int* done) {
  if (*done) return;
  __shared__ double hs[kMaxCols];
  __shared__ double sh[kThreads / 32];
  const int c = Qt.c;
  for (int j = threadIdx.x; j < c; j += blockDim.x) hs[j] = dots[j];
  __syncthreads();
  const double sigma = dots[c];
  const T alpha = (T)(scal[S_RHO] / sigma);
  T acc = T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T ti = t[i];
    for (int j = 0; j < c; ++j) ti -= Qt.p[(int64_t)j * Qt.ld + i] * (T)hs[j];
    const T ri = r[i] - alpha * ti;
    r[i] = ri;
    acc += ri * ri;
  }
  const double s = block_sum((double)acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// After ||r||^2: theta_k, c_k, tau_k and the convergence test (one thread).
__global__ void sqmr_scalar_theta_kernel(const double* __restrict__ partial, int nblocks,
                                         const double* __restrict__ dots, int c, double* __restrict__ scal,
                                         int* done, int* breakdown) {
  if (*done) return;
  const double rr = warp_sum_partials(partial, nblocks, 1, 0);  // one warp; lane 0 goes on
  if (threadIdx.x != 0) return;
  const double sigma = dots[c];
  if (sigma == 0.0 || !isfinite(sigma)) {
    *breakdown = 1;
    *done = 1;
    return;
  }
  const double alpha = scal[S_RHO] / sigma;
  const double theta_old = scal[S_THETA];
  const double theta = sqrt(rr) / scal[S_TAU];
  const double c2 = 1.0 / (1.0 + theta * theta);
  const double tau = scal[S_TAU] * theta * sqrt(c2);
  scal[S_ALPHA] = alpha;
  scal[S_SIGMA] = sigma;
  scal[S_CD] = c2 * theta_old * theta_old;
  scal[S_CQ] = c2 * alpha;
  scal[S_THETA] = theta;
  scal[S_TAU] = tau;
  const double it = scal[S_IT] + 1.0;
  scal[S_IT] = it;
  if (sqrt(it + 1.0) * tau <= scal[S_TOL] || !isfinite(tau)) *done = 2;  // 2: stop after x update
}

// d = cd d + cq q ; x += d
template <typename T>
__global__ void sqmr_update_dx_kernel(T* __restrict__ d, T* __restrict__ x, const T* __restrict__ q, int64_t n,
                                      const double* __restrict__ scal, const int* done) {
  if (*done == 1) return;
  const T cd = (T)scal[S_CD], cq = (T)scal[S_CQ];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T di = cd * d[i] + cq * q[i];
    d[i] = di;
    x[i] += di;
  }
}

__global__ void sqmr_mark_done_kernel(int* done) {
  if (*done == 2) *done = 1;
}

// g = Minv (Qt^T y) (small, one thread block)
__global__ void small_matvec_kernel(const double* __restrict__ Minv, int c, const double* __restrict__ g,
                                    double* __restrict__ out, const int* done) {
  if (done && *done) return;
  for (int i = threadIdx.x; i < c; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < c; ++j) s += Minv[(int64_t)j * c + i] * g[j];
    out[i] = s;
  }
}

// u = y - W gg ; partial r^T u
template <typename T>
__global__ void __launch_bounds__(kThreads)
sqmr_update_u_kernel(Cols<T> W, const double* __restrict__ gg, const T* __restrict__ y, const T* __restrict__ r,
                     T* __restrict__ u, int64_t n, double* __restrict__ partial, const int* done) {
  if (done && *done) return;
  __shared__ double hs[kMaxCols];
  __shared__ double sh[kThreads / 32];
  for (int j = threadIdx.x; j < W.c; j += blockDim.x) hs[j] = gg[j];
  __syncthreads();
  T acc = T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T ui = y[i];
    for (int j = 0; j < W.c; ++j) ui -= W.p[(int64_t)j * W.ld + i] * (T)hs[j];
    u[i] = ui;
    acc += r[i] * ui;
  }
  const double s = block_sum((double)acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// rho' = r^T u ; beta = rho'/rho (first call: just rho)
__global__ void sqmr_scalar_beta_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ scal,
                                        int first, int* done, int* breakdown) {
  if (*done) return;
  const double rho = warp_sum_partials(partial, nblocks, 1, 0);  // one warp; lane 0 goes on
  if (threadIdx.x != 0) return;
  if (first) {
    scal[S_BETA] = 0.0;
  } else {
    if (scal[S_RHO] == 0.0) {
      *breakdown = 1;
      *done = 1;
      return;
    }
    scal[S_BETA] = rho / scal[S_RHO];
  }
  scal[S_RHO] = rho;
  if (rho == 0.0 || !isfinite(rho)) {
    *breakdown = 1;
    *done = 1;
  }
}

// q = u + beta q
template <typename T>
__global__ void sqmr_update_q_kernel(const T* __restrict__ u, T* __restrict__ q, int64_t n,
                                     const double* __restrict__ scal, const int* done) {
  if (*done) return;
  const T beta = (T)scal[S_BETA];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    q[i] = u[i] + beta * q[i];
}

// init: r = b, x = d = q = 0, partial ||r||^2.  q must hold numbers before
// the first q = u + beta q (beta = 0): a buffer that held other data may
// contain NaN bit patterns, and 0 * NaN is NaN.
template <typename T>
__global__ void __launch_bounds__(kThreads)
sqmr_init_kernel(const T* __restrict__ b, T* __restrict__ r, T* __restrict__ x, T* __restrict__ d,
                 T* __restrict__ q, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[kThreads / 32];
  T acc = T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T bi = b[i];
    r[i] = bi;
    x[i] = T(0);
    d[i] = T(0);
    q[i] = T(0);
    acc += bi * bi;
  }
  const double s = block_sum((double)acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void sqmr_scalar_init_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ scal,
                                        double rel_tol, int* done, int* breakdown) {
  const double rr = warp_sum_partials(partial, nblocks, 1, 0);  // one warp; lane 0 goes on
  if (threadIdx.x != 0) return;
  const double bn = sqrt(rr);
  for (int i = 0; i < S_NSCAL; ++i) scal[i] = 0.0;
  scal[S_TAU] = bn;
  scal[S_BNORM] = bn;
  scal[S_TOL] = rel_tol * bn;
  *breakdown = 0;
  *done = (bn == 0.0 || !isfinite(bn)) ? 1 : 0;
}

// Sign convention of an eigenvector: the largest |x_i| (lowest index on
// ties).  Pass 1: max |x| via an atomic max on the IEEE bits (monotone for
// non-negative doubles); pass 2: smallest index attaining it.
__global__ void max_abs_bits_kernel(const double* __restrict__ x, int64_t n, unsigned long long* out) {
  unsigned long long best = 0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(x[i]));
    best = b > best ? b : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
    best = v > best ? v : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

__global__ void first_index_kernel(const double* __restrict__ x, int64_t n, const unsigned long long* bits,
                                   unsigned long long* out) {
  const double m = __longlong_as_double((long long)*bits);
  unsigned long long best = ~0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (fabs(x[i]) == m && (unsigned long long)i < best) best = (unsigned long long)i;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
    best = v < best ? v : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMin(out, best);
}

}  // namespace

// ------------------------------------------- small dense algebra (host) ---
// Matrices of order m <= 64, column-major with leading dimension m.
namespace hostla {

// Cyclic Jacobi eigen-decomposition of the symmetric A: A = V diag(w) V^T.
void jacobi_eig(int m, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)j * m + i]; };
  double fro = 0.0;
  for (double x : A) fro += x * x;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i)
        if (i != j) off += a(i, j) * a(i, j);
    if (off <= 1e-30 * fro || fro == 0.0) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = a(p, q);
        if (apq == 0.0) continue;
        const double tau = (a(q, q) - a(p, p)) / (2.0 * apq);
        double t;
        if (std::fabs(tau) > 1e150) t = 0.5 / tau;
        else t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = t * c;
        for (int k = 0; k < m; ++k) {
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - sn * akq;
          a(k, q) = sn * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - sn * aqk;
          a(q, k) = sn * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double vkp = V[(size_t)p * m + k], vkq = V[(size_t)q * m + k];
          V[(size_t)p * m + k] = c * vkp - sn * vkq;
          V[(size_t)q * m + k] = sn * vkp + c * vkq;
        }
      }
  }
  w.resize(m);
  for (int i = 0; i < m; ++i) w[i] = a(i, i);
}

// Cholesky G = L L^T in place (lower triangle); false if not positive definite.
bool cholesky(int m, std::vector<double>& G) {
  for (int j = 0; j < m; ++j) {
    double d = G[(size_t)j * m + j];
    for (int k = 0; k < j; ++k) d -= G[(size_t)k * m + j] * G[(size_t)k * m + j];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    G[(size_t)j * m + j] = d;
    for (int i = j + 1; i < m; ++i) {
      double s = G[(size_t)j * m + i];
      for (int k = 0; k < j; ++k) s -= G[(size_t)k * m + i] * G[(size_t)k * m + j];
      G[(size_t)j * m + i] = s / d;
    }
  }
  return true;
}

// Orthonormal basis (m x c, column-major) of the columns of Y (m x c) by
// modified Gram–Schmidt run twice; the first column is y_0 / ||y_0||.
void orthonormalize(int m, int c, const std::vector<double>& Y, std::vector<double>& Qo) {
  Qo = Y;
  for (int j = 0; j < c; ++j) {
    double* qj = &Qo[(size_t)j * m];
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i < j; ++i) {
        const double* qi = &Qo[(size_t)i * m];
        double d = 0.0;
        for (int k = 0; k < m; ++k) d += qi[k] * qj[k];
        for (int k = 0; k < m; ++k) qj[k] -= d * qi[k];
      }
    double nr = 0.0;
    for (int k = 0; k < m; ++k) nr += qj[k] * qj[k];
    nr = std::sqrt(nr);
    for (int k = 0; k < m; ++k) qj[k] = nr > 0.0 ? qj[k] / nr : 0.0;
  }
}

// B = Q^T A Q for symmetric A (m x m) and Q (m x c)
std::vector<double> congruence(int m, int c, const std::vector<double>& A, const std::vector<double>& Q) {
  std::vector<double> AQ((size_t)m * c, 0.0), B((size_t)c * c, 0.0);
  for (int j = 0; j < c; ++j)
    for (int k = 0; k < m; ++k) {
      const double q = Q[(size_t)j * m + k];
      if (q == 0.0) continue;
      for (int i = 0; i < m; ++i) AQ[(size_t)j * m + i] += A[(size_t)k * m + i] * q;
    }
  for (int j = 0; j < c; ++j)
    for (int i = 0; i < c; ++i) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += Q[(size_t)i * m + k] * AQ[(size_t)j * m + k];
      B[(size_t)j * c + i] = s;
    }
  for (int j = 0; j < c; ++j)
    for (int i = j + 1; i < c; ++i) {
      const double v = 0.5 * (B[(size_t)j * c + i] + B[(size_t)i * c + j]);
      B[(size_t)j * c + i] = B[(size_t)i * c + j] = v;
    }
  return B;
}

}  // namespace hostla

// ------------------------------------------------------------ the solver ---
class JdSolver {
 public:
  JdSolver(anderson_s* h, ildl_s* pc, const jd_params& p, double sigma, int k, double tol, cudaStream_t s)
      : h_(h), pc_(pc), p_(p), sigma_(sigma), k_(k), tol_(tol), s_(s) {}
  ~JdSolver() { release(); }

  int run(double* evals, double* evecs, jd_stats* st);
  // shift-and-invert Lanczos (Section 4.1) over the same preconditioned
  // SQMR: the alternative to run()
  int lanczos(double* evals, double* evecs, jd_stats* st);

 private:
  anderson_s* h_;
  ildl_s* pc_;
  jd_params p_;
  double sigma_;
  int k_;
  double tol_;
  cudaStream_t s_;
  int64_t n_ = 0, ld_ = 0;
  int jmin_ = 0, jmax_ = 0;
  int kint_ = 0;  // pairs computed: k plus guard pairs
  double normA_ = 0.0;
  // binary64 buffers
  double *V_ = nullptr, *AV_ = nullptr, *Vt_ = nullptr, *AVt_ = nullptr, *Q_ = nullptr;
  double *t_ = nullptr, *u_ = nullptr, *Au_ = nullptr, *r_ = nullptr;
  double *H_ = nullptr, *theta_ = nullptr, *Y_ = nullptr, *dots_ = nullptr, *partial_ = nullptr, *scal_ = nullptr;
  double *Minv_ = nullptr, *gg_ = nullptr;
  int* flags_ = nullptr;  // [0] done, [1] breakdown
  unsigned long long* amax_ = nullptr;  // [0] max bits, [1] first index
  // inner-precision buffers (allocated as bytes)
  void *Qt_ = nullptr, *W_ = nullptr, *xb_ = nullptr, *rb_ = nullptr, *qb_ = nullptr, *db_ = nullptr,
       *tb_ = nullptr, *yb_ = nullptr, *ub_ = nullptr, *bb_ = nullptr;
  double* host_ = nullptr;  // pinned readback area
  int nb_ = 0;              // blocks of vector kernels
  // BF16 shadows of Q and V for the tensor-core first Gram-Schmidt pass:
  // columns [0, qb_ok_) of Q and [0, vb_ok_) of V are current
  bool gram_bf16_ = false;
  void *Xbq_ = nullptr, *Xbv_ = nullptr;
  int64_t ldb_ = 0;
  int qb_ok_ = 0, vb_ok_ = 0;
  int* gerr_ = nullptr;  // a tensor-core wait timed out
  std::vector<double> Mq_;  // cached Q^T W_Q block (host, kc x kc)
  int inner_total_ = 0;
  // CUDA events around the inner-loop preconditioner and stencil calls
  static constexpr int kEv = 16;
  cudaEvent_t evp_[2 * kEv] = {}, evs_[2 * kEv] = {};
  int nevp_ = 0, nevs_ = 0;
  int precond_calls_ = 0, stencil_calls_ = 0;
  double precond_ms_ = 0.0, stencil_ms_ = 0.0;
  int64_t launches0_ = 0;
  bool trace_ = std::getenv("AJD_JD_TRACE") != nullptr;
  void harvest_events();

  int alloc();
  void release();
  int dot_cols(Cols<double> X1, Cols<double> X2, const double* extra, const double* v, double* out);
  int cgs2(int kc, int m, double* t, double* nrm_host);
  int rr(int m);
  template <typename T, typename P>
  int correction(int kc, double theta_hat, double rel_tol, int* its);
  template <typename T, typename P>
  int sqmr_core(int c, double shift, const double* rhs, double sign, double rel_tol, int maxit, double* xout,
                int* its);
  // out = K^{-1} in with vectors in T and the preconditioner applied in P
  template <typename T, typename P>
  int apply_k(const T* in, T* out);
  template <typename T, typename P>
  int cache_lock_column(int kc);
  int finalize(int kc, double* lam, double* evals, double* evecs, jd_stats* st);
  int sync_read(const double* dev, int cnt, double* host);
  // wait for the work queued on s_ by blocking on an event: the waiting
  // thread yields its core (setup threads of a batch or a server share the
  // host cores with the solving threads)
  int wait_stream();
  cudaEvent_t sync_ev_ = nullptr;
};

int JdSolver::alloc() {
  n_ = h_->n;
  ld_ = (n_ + 31) & ~(int64_t)31;
  nb_ = vec_blocks(n_);
  const size_t vb = (size_t)ld_ * sizeof(double);
  // AJD_POISON_ALLOC set: fill every work buffer with 0xFF bytes (NaN in
  // binary32 and binary64), so that a read before the first write shows up
  // as a NaN in the tests instead of depending on what the memory held
  const bool poison = std::getenv("AJD_POISON_ALLOC") != nullptr;
  auto A = [&](void** p, size_t bytes) -> int {
    bytes = std::max<size_t>(bytes, 16);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess)
      return fail(e == cudaErrorMemoryAllocation ? JD_ENOMEM : JD_EDEVICE, "jd_solve: cudaMalloc: %s", cudaGetErrorString(e));
    if (poison) AJD_CUDA(cudaMemsetAsync(*p, 0xFF, bytes, s_));
    return JD_OK;
  };
  AJD_TRY(A((void**)&V_, vb * jmax_));
  AJD_TRY(A((void**)&AV_, vb * jmax_));
  AJD_TRY(A((void**)&Vt_, vb * jmax_));
  AJD_TRY(A((void**)&AVt_, vb * jmax_));
  AJD_TRY(A((void**)&Q_, vb * kint_));
  AJD_TRY(A((void**)&t_, vb));
  AJD_TRY(A((void**)&u_, vb));
  AJD_TRY(A((void**)&Au_, vb));
  AJD_TRY(A((void**)&r_, vb));
  AJD_TRY(A((void**)&H_, sizeof(double) * kMaxM * kMaxM));
  AJD_TRY(A((void**)&theta_, sizeof(double) * kMaxM));
  AJD_TRY(A((void**)&Y_, sizeof(double) * kMaxM * kMaxM));
  AJD_TRY(A((void**)&dots_, sizeof(double) * kMaxCols));
  AJD_TRY(A((void**)&partial_, sizeof(double) * (size_t)nb_ * kMaxCols));
  AJD_TRY(A((void**)&scal_, sizeof(double) * 64));
  AJD_TRY(A((void**)&Minv_, sizeof(double) * (kint_ + 1) * (kint_ + 1)));
  AJD_TRY(A((void**)&gg_, sizeof(double) * (kint_ + 1)));
  AJD_TRY(A((void**)&flags_, sizeof(int) * 4));
  AJD_TRY(A((void**)&amax_, 2 * sizeof(unsigned long long)));
  const size_t eb = p_.precision == JD_FP32 ? sizeof(float) : sizeof(double);

  const size_t pb = (size_t)ld_ * eb;
  AJD_TRY(A(&Qt_, pb * (kint_ + 1)));
  AJD_TRY(A(&W_, pb * (kint_ + 1)));
  for (void** b : {&xb_, &rb_, &qb_, &db_, &tb_, &yb_, &ub_, &bb_}) AJD_TRY(A(b, pb));
  gram_bf16_ = (p_.gram == 2 || (p_.gram == 0 && p_.precision != JD_FP64)) && kint_ + jmax_ <= gram_bf16_max_cols();
  if (gram_bf16_) {
    ldb_ = gram_bf16_ld(n_);
    AJD_TRY(A(&Xbq_, (size_t)ldb_ * 2 * kint_));
    AJD_TRY(A(&Xbv_, (size_t)ldb_ * 2 * jmax_));
    AJD_TRY(A((void**)&gerr_, sizeof(int)));
    AJD_CUDA(cudaMemsetAsync(gerr_, 0, sizeof(int), s_));
    qb_ok_ = vb_ok_ = 0;
  }
  AJD_CUDA(cudaMallocHost(&host_, sizeof(double) * (kMaxM * kMaxM + 256)));
  for (auto& e : evp_) AJD_CUDA(cudaEventCreate(&e));
  for (auto& e : evs_) AJD_CUDA(cudaEventCreate(&e));
  return JD_OK;
}

void JdSolver::harvest_events() {
  for (int i = 0; i < nevp_; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, evp_[2 * i], evp_[2 * i + 1]) == cudaSuccess) precond_ms_ += ms;
  }
  for (int i = 0; i < nevs_; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, evs_[2 * i], evs_[2 * i + 1]) == cudaSuccess) stencil_ms_ += ms;
  }
  precond_calls_ += nevp_;
  stencil_calls_ += nevs_;
  nevp_ = nevs_ = 0;
}

void JdSolver::release() {
  if (sync_ev_) cudaEventDestroy(sync_ev_);
  sync_ev_ = nullptr;
  for (auto& e : evp_) if (e) cudaEventDestroy(e);
  for (auto& e : evs_) if (e) cudaEventDestroy(e);
  for (void* p : {(void*)V_, (void*)AV_, (void*)Vt_, (void*)AVt_, (void*)Q_, (void*)t_, (void*)u_, (void*)Au_,
                  (void*)r_, (void*)H_, (void*)theta_, (void*)Y_, (void*)dots_, (void*)partial_, (void*)scal_,
                  (void*)Minv_, (void*)gg_, (void*)flags_, (void*)amax_, Qt_, W_, xb_, rb_, qb_, db_, tb_, yb_, ub_, bb_,
                  Xbq_, Xbv_, (void*)gerr_})
    if (p) cudaFree(p);
  if (host_) cudaFreeHost(host_);
  V_ = nullptr;
  host_ = nullptr;
}

int JdSolver::wait_stream() {
  if (!sync_ev_) AJD_CUDA(cudaEventCreateWithFlags(&sync_ev_, cudaEventDisableTiming | cudaEventBlockingSync));
  AJD_CUDA(cudaEventRecord(sync_ev_, s_));
  AJD_CUDA(cudaEventSynchronize(sync_ev_));
  return JD_OK;
}

int JdSolver::sync_read(const double* dev, int cnt, double* host) {
  AJD_CUDA(cudaMemcpyAsync(host_, dev, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s_));
  AJD_TRY(wait_stream());
  std::memcpy(host, host_, sizeof(double) * cnt);
  return JD_OK;
}

int JdSolver::dot_cols(Cols<double> X1, Cols<double> X2, const double* extra, const double* v, double* out) {
  const int nc = X1.c + X2.c + (extra ? 1 : 0);
  if (nc == 0) return JD_OK;
  multidot_kernel<double><<<nb_, kThreads, 0, s_>>>(X1, X2, extra, v, n_, partial_, nc, nullptr); count_launches();
  reduce_partials_kernel<<<1, kRedThreads, 0, s_>>>(partial_, nb_, nc, out, nullptr); count_launches();
  AJD_CHECK_LAUNCH();
  return JD_OK;
}

// t <- (I - [Q V][Q V]^T)^2 t; returns ||t|| (device scal[0] and host)
int JdSolver::cgs2(int kc, int m, double* t, double* nrm_host) {
  Cols<double> Xq{Q_, ld_, kc}, Xv{V_, ld_, m};
  if (gram_bf16_ && kc + m > 0) {
    // first pass: the projection c = X^T t on the tensor cores with the BF16
    // shadows (brought up to date column by column), the update t -= X c
    // with the binary64 columns -- so the BF16 error of c stays inside
    // span(X), where the binary64 second pass removes it, and nothing is
    // added to t's component outside span(X); if the second pass still
    // removes more than 3/4 of ||t||^2 (Daniel-Gragg-Kaufman-Stewart
    // criterion), one more binary64 pass
    if (qb_ok_ < kc) AJD_TRY(gram_bf16_convert(Q_, ld_, qb_ok_, kc, Xbq_, ldb_, n_, s_));
    if (vb_ok_ < m) AJD_TRY(gram_bf16_convert(V_, ld_, vb_ok_, m, Xbv_, ldb_, n_, s_));
    qb_ok_ = kc;
    vb_ok_ = m;
    AJD_TRY(gram_bf16_dots(Xbq_, kc, Xbv_, m, ldb_, t, n_, partial_, nb_, dots_, gerr_, s_));
    multiaxpy_kernel<double><<<nb_, kThreads, 0, s_>>>(Xq, Xv, dots_, t, n_); count_launches();
    AJD_TRY(dot_cols(Xq, Xv, t, t, dots_));  // projections and ||t||^2 before the pass
    multiaxpy_kernel<double><<<nb_, kThreads, 0, s_>>>(Xq, Xv, dots_, t, n_); count_launches();
    AJD_TRY(dot_cols(Cols<double>{t, ld_, 1}, Cols<double>{}, nullptr, t, scal_));
    double nb[2];
    AJD_CUDA(cudaMemcpyAsync(scal_ + 1, dots_ + kc + m, sizeof(double), cudaMemcpyDeviceToDevice, s_));
    AJD_TRY(sync_read(scal_, 2, nb));
    if (nb[0] < 0.25 * nb[1]) {
      AJD_TRY(dot_cols(Xq, Xv, nullptr, t, dots_));
      multiaxpy_kernel<double><<<nb_, kThreads, 0, s_>>>(Xq, Xv, dots_, t, n_); count_launches();
    } else {
      *nrm_host = std::sqrt(std::max(nb[0], 0.0));
      return JD_OK;
    }
  } else {
    for (int pass = 0; pass < 2; ++pass) {
      if (kc + m == 0) break;
      AJD_TRY(dot_cols(Xq, Xv, nullptr, t, dots_));
      multiaxpy_kernel<double><<<nb_, kThreads, 0, s_>>>(Xq, Xv, dots_, t, n_); count_launches();
    }
  }
  AJD_TRY(dot_cols(Cols<double>{t, ld_, 1}, Cols<double>{}, nullptr, t, scal_));
  double nn;
  AJD_TRY(sync_read(scal_, 1, &nn));
  *nrm_host = std::sqrt(std::max(nn, 0.0));
  return JD_OK;
}

int JdSolver::rr(int m) {
  const int mp = (m + 1) & ~1;
  const size_t sm = sizeof(double) * (2 * mp * mp + mp) + sizeof(int) * mp;
  static const cudaError_t attr = cudaFuncSetAttribute(  // once per process (thread-safe static init)
      rr_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)(sizeof(double) * (2 * kMaxM * kMaxM + kMaxM) + sizeof(int) * kMaxM));
  AJD_CUDA(attr);
  rr_eig_kernel<<<1, kThreads, sm, s_>>>(H_, kMaxM, m, sigma_, theta_, Y_, kMaxM); count_launches();
  AJD_CHECK_LAUNCH();
  return JD_OK;
}

template <typename T, typename P>
int JdSolver::apply_k(const T* in, T* out) {
  if constexpr (std::is_same<T, P>::value) {
    return ildl_apply_dev<T>(pc_, in, out, s_);
  } else {
    // binary32 factor, binary64 vectors and accumulation
    return ildl_apply_dev_mixed(pc_, in, out, s_);
  }
}

// Q~[:, kc] = u and W[:, kc] = K^{-1} u for a newly locked vector, and the
// new row/column of M = Q~^T W (host cache Mq_)
template <typename T, typename P>
int JdSolver::cache_lock_column(int kc) {
  const int c = kc + 1;
  T* Qt = static_cast<T*>(Qt_);
  T* W = static_cast<T*>(W_);
  convert_kernel<double, T><<<nb_, kThreads, 0, s_>>>(u_, Qt + (int64_t)kc * ld_, n_, 1.0); count_launches();
  AJD_TRY((apply_k<T, P>(Qt + (int64_t)kc * ld_, W + (int64_t)kc * ld_)));
  multidot_kernel<T><<<nb_, kThreads, 0, s_>>>(Cols<T>{Qt, ld_, c}, Cols<T>{}, nullptr, W + (int64_t)kc * ld_, n_,
                                               partial_, c, nullptr); count_launches();
  reduce_partials_kernel<<<1, kRedThreads, 0, s_>>>(partial_, nb_, c, dots_, nullptr); count_launches();
  std::vector<double> col(c);
  AJD_TRY(sync_read(dots_, c, col.data()));
  std::vector<double> Mn((size_t)c * c);
  for (int i = 0; i < kc; ++i)
    for (int j = 0; j < kc; ++j) Mn[(size_t)j * c + i] = Mq_[(size_t)j * kc + i];
  for (int i = 0; i < c; ++i) {
    Mn[(size_t)kc * c + i] = col[i];
    Mn[(size_t)i * c + kc] = col[i];
  }
  Mq_.swap(Mn);
  return JD_OK;
}

template <typename T, typename P>
int JdSolver::correction(int kc, double theta_hat, double rel_tol, int* its) {
  const int c = kc + 1;
  T* Qt = static_cast<T*>(Qt_);
  T* W = static_cast<T*>(W_);
  const int bl = nb_;
  // Qt[:, kc] = u, W[:, kc] = K^{-1} u  (Q columns and their W are cached)
  convert_kernel<double, T><<<bl, kThreads, 0, s_>>>(u_, Qt + (int64_t)kc * ld_, n_, 1.0); count_launches();
  AJD_TRY((apply_k<T, P>(Qt + (int64_t)kc * ld_, W + (int64_t)kc * ld_)));
  // M = Qt^T W (c x c): only row/column kc are new
  {
    multidot_kernel<T><<<bl, kThreads, 0, s_>>>(Cols<T>{Qt, ld_, c}, Cols<T>{}, nullptr, W + (int64_t)kc * ld_, n_,
                                                partial_, c, nullptr); count_launches();
    reduce_partials_kernel<<<1, kRedThreads, 0, s_>>>(partial_, bl, c, dots_, nullptr); count_launches();
    std::vector<double> col(c);
    AJD_TRY(sync_read(dots_, c, col.data()));
    // assemble M (host) from the cached Q block and the new column, invert
    std::vector<double> M((size_t)c * c), Mi((size_t)c * c, 0.0);
    for (int i = 0; i < kc; ++i)
      for (int j = 0; j < kc; ++j) M[(size_t)j * c + i] = Mq_[(size_t)j * kc + i];
    for (int i = 0; i < c; ++i) {
      M[(size_t)kc * c + i] = col[i];
      M[(size_t)i * c + kc] = col[i];
    }
    // Gauss–Jordan with partial pivoting (c <= 65)
    std::vector<double> A = M;
    for (int i = 0; i < c; ++i) Mi[(size_t)i * c + i] = 1.0;
    for (int cc = 0; cc < c; ++cc) {
      int pv = cc;
      for (int rr2 = cc + 1; rr2 < c; ++rr2)
        if (std::fabs(A[(size_t)cc * c + rr2]) > std::fabs(A[(size_t)cc * c + pv])) pv = rr2;
      if (A[(size_t)cc * c + pv] == 0.0) return fail(JD_EBREAKDOWN, "jd: Q~^T K^{-1} Q~ is singular");
      for (int j = 0; j < c; ++j) {
        std::swap(A[(size_t)j * c + cc], A[(size_t)j * c + pv]);
        std::swap(Mi[(size_t)j * c + cc], Mi[(size_t)j * c + pv]);
      }
      const double inv = 1.0 / A[(size_t)cc * c + cc];
      for (int j = 0; j < c; ++j) {
        A[(size_t)j * c + cc] *= inv;
        Mi[(size_t)j * c + cc] *= inv;
      }
      for (int rr2 = 0; rr2 < c; ++rr2) {
        if (rr2 == cc) continue;
        const double f = A[(size_t)cc * c + rr2];
        if (f == 0.0) continue;
        for (int j = 0; j < c; ++j) {
          A[(size_t)j * c + rr2] -= f * A[(size_t)j * c + cc];
          Mi[(size_t)j * c + rr2] -= f * Mi[(size_t)j * c + cc];
        }
      }
    }
    AJD_CUDA(cudaMemcpyAsync(Minv_, Mi.data(), sizeof(double) * c * c, cudaMemcpyHostToDevice, s_));
  }
  // rhs b = -r (binary64 residual, already orthogonal to Q and u); the
  // solution goes to t_ (binary64), which the caller orthogonalises
  return sqmr_core<T, P>(c, theta_hat, r_, -1.0, rel_tol, p_.max_inner, t_, its);
}

// Preconditioned SQMR for (P (A - shift I) P) x = P b with b = sign * rhs and
// P the projection against the first c columns of Q~ (the projected
// preconditioner K^{-1} - W M^{-1} W^T of the correction equation); c = 0
// is the plain preconditioned solve of (A - shift I) x = b.  Stops when the
// quasi-residual estimate falls below rel_tol ||b|| or after maxit
// iterations; x goes to xout (binary64).
template <typename T, typename P>
int JdSolver::sqmr_core(int c, double shift, const double* rhs, double sign, double rel_tol, int maxit, double* xout,
                        int* its) {
  T* Qt = static_cast<T*>(Qt_);
  T* W = static_cast<T*>(W_);
  T *x = static_cast<T*>(xb_), *r = static_cast<T*>(rb_), *q = static_cast<T*>(qb_), *d = static_cast<T*>(db_);
  T *t = static_cast<T*>(tb_), *y = static_cast<T*>(yb_), *u = static_cast<T*>(ub_), *b = static_cast<T*>(bb_);
  int* done = flags_;
  int* brk = flags_ + 1;
  const int bl = nb_;
  const double theta_hat = shift;
  convert_kernel<double, T><<<bl, kThreads, 0, s_>>>(rhs, b, n_, sign); count_launches();
  Cols<T> QtC{Qt, ld_, c}, WC{W, ld_, c};
  // init: r = b, x = d = 0, tau = ||b||; u = P b; q = u; rho = r^T u
  sqmr_init_kernel<T><<<bl, kThreads, 0, s_>>>(b, r, x, d, q, n_, partial_); count_launches();
  sqmr_scalar_init_kernel<<<1, 32, 0, s_>>>(partial_, bl, scal_, rel_tol, done, brk); count_launches();
  auto precond = [&]() -> int {
    const bool timed = nevp_ < kEv;
    if (timed) AJD_CUDA(cudaEventRecord(evp_[2 * nevp_], s_));
    AJD_TRY((apply_k<T, P>(r, y)));
    if (timed) AJD_CUDA(cudaEventRecord(evp_[2 * nevp_++ + 1], s_));
    multidot_kernel<T><<<bl, kThreads, 0, s_>>>(QtC, Cols<T>{}, nullptr, y, n_, partial_, c, done); count_launches();
    reduce_partials_kernel<<<1, kRedThreads, 0, s_>>>(partial_, bl, c, dots_, done); count_launches();
    small_matvec_kernel<<<1, 64, 0, s_>>>(Minv_, c, dots_, gg_, done); count_launches();
    sqmr_update_u_kernel<T><<<bl, kThreads, 0, s_>>>(WC, gg_, y, r, u, n_, partial_, done); count_launches();
    return JD_OK;
  };
  AJD_TRY(precond());
  sqmr_scalar_beta_kernel<<<1, 32, 0, s_>>>(partial_, bl, scal_, 1, done, brk); count_launches();
  sqmr_update_q_kernel<T><<<bl, kThreads, 0, s_>>>(u, q, n_, scal_, done); count_launches();  // q = u (beta = 0)
  int it = 0;
  const int chunk = 4;
  while (it < maxit) {
    const int nstep = std::min(chunk, maxit - it);
    for (int s = 0; s < nstep; ++s) {
      const bool timed = nevs_ < kEv;
      if (timed) AJD_CUDA(cudaEventRecord(evs_[2 * nevs_], s_));
      AJD_TRY(stencil_apply<T>(h_, (T)theta_hat, q, t, 1, s_));
      if (timed) AJD_CUDA(cudaEventRecord(evs_[2 * nevs_++ + 1], s_));
      multidot_kernel<T><<<bl, kThreads, 0, s_>>>(QtC, Cols<T>{}, q, t, n_, partial_, c + 1, done); count_launches();
      reduce_partials_kernel<<<1, kRedThreads, 0, s_>>>(partial_, bl, c + 1, dots_, done); count_launches();
      sqmr_update_r_kernel<T><<<bl, kThreads, 0, s_>>>(QtC, dots_, t, r, n_, scal_, partial_, done); count_launches();
      sqmr_scalar_theta_kernel<<<1, 32, 0, s_>>>(partial_, bl, dots_, c, scal_, done, brk); count_launches();
      sqmr_update_dx_kernel<T><<<bl, kThreads, 0, s_>>>(d, x, q, n_, scal_, done); count_launches();
      sqmr_mark_done_kernel<<<1, 1, 0, s_>>>(done); count_launches();
      AJD_TRY(precond());
      sqmr_scalar_beta_kernel<<<1, 32, 0, s_>>>(partial_, bl, scal_, 0, done, brk); count_launches();
      sqmr_update_q_kernel<T><<<bl, kThreads, 0, s_>>>(u, q, n_, scal_, done); count_launches();
    }
    AJD_CHECK_LAUNCH();
    it += nstep;
    double sc[S_NSCAL];
    int fl[2];
    AJD_CUDA(cudaMemcpyAsync(host_, scal_, sizeof(double) * S_NSCAL, cudaMemcpyDeviceToHost, s_));
    AJD_CUDA(cudaMemcpyAsync(host_ + S_NSCAL, flags_, sizeof(int) * 2, cudaMemcpyDeviceToHost, s_));
    AJD_TRY(wait_stream());
    std::memcpy(sc, host_, sizeof(sc));
    std::memcpy(fl, host_ + S_NSCAL, sizeof(fl));
    harvest_events();
    if (fl[0]) {
      it = (int)sc[S_IT];
      break;
    }
  }
  *its = it;
  AJD_TRY(ildl_check_device_error(pc_, s_));
  convert_kernel<T, double><<<bl, kThreads, 0, s_>>>(x, xout, n_, 1.0); count_launches();
  AJD_CHECK_LAUNCH();
  return JD_OK;
}

int JdSolver::run(double* evals, double* evecs, jd_stats* st) {
  using Clock = std::chrono::steady_clock;
  const auto t0 = Clock::now();
  normA_ = h_->norm_bound();
  const int64_t n = h_->n;
  const int guard = p_.guard < 0 ? 0 : (p_.guard == 0 ? 2 : p_.guard);
  kint_ = (int)std::min<int64_t>(k_ + guard, n / 2 > k_ ? n / 2 : k_);
  jmin_ = p_.jmin > 0 ? p_.jmin : std::max(2 * kint_, 10);
  jmax_ = p_.jmax > 0 ? p_.jmax : jmin_ + 15;
  jmax_ = (int)std::min<int64_t>(std::min<int64_t>(jmax_, kMaxM), n - kint_);
  jmin_ = std::min(jmin_, jmax_ - 1);
  if (jmax_ < 2 || jmin_ < 1) return fail(JD_EINVAL, "jd_solve: lattice too small for k = %d", k_);
  if (kint_ + 2 * jmax_ + 2 > kMaxCols) return fail(JD_EINVAL, "jd_solve: k + jmax too large");
  AJD_TRY(alloc());
  launches0_ = launch_counter();
  Mq_.clear();
  const uint64_t seed = p_.seed ? p_.seed : (h_->seed ^ 0xD1B54A32D192ED03ull);
  random_kernel<<<nb_, kThreads, 0, s_>>>(t_, n, seed); count_launches();
  int m = 0, kc = 0, outer = 0, restarts = 0, steps_on_pair = 0;
  std::vector<double> lam;
  double theta0 = sigma_, rnorm = 0.0, gap = 0.0;
  int status = JD_OK;
  uint64_t reseed = seed;
  std::vector<double> Yc, th;
  // host copies of H = V^T A V and G = (AV - sigma V)^T (AV - sigma V) for
  // the current basis
  std::vector<double> Hh((size_t)kMaxM * kMaxM, 0.0), Gh((size_t)kMaxM * kMaxM, 0.0);
  auto hget = [&](std::vector<double>& X, int i, int j) -> double& { return X[(size_t)j * kMaxM + i]; };
  auto compact = [&](const std::vector<double>& X, int m) {
    std::vector<double> c((size_t)m * m);
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i) c[(size_t)j * m + i] = X[(size_t)j * kMaxM + i];
    return c;
  };
  auto expand_h = [&](std::vector<double>& X, const std::vector<double>& c, int m) {
    std::fill(X.begin(), X.end(), 0.0);
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i) X[(size_t)j * kMaxM + i] = c[(size_t)j * m + i];
  };
  // apply the coefficient basis Qy (m x c) to V and AV on the device and to
  // H, M2 on the host
  auto transform = [&](int m, int c, const std::vector<double>& Qy) -> int {
    std::vector<double> up((size_t)kMaxM * c, 0.0);
    for (int j = 0; j < c; ++j)
      for (int i = 0; i < m; ++i) up[(size_t)j * kMaxM + i] = Qy[(size_t)j * m + i];
    AJD_CUDA(cudaMemcpyAsync(Y_, up.data(), sizeof(double) * kMaxM * c, cudaMemcpyHostToDevice, s_));
    lincomb_kernel<<<nb_, kThreads, 0, s_>>>(V_, ld_, m, Y_, kMaxM, c, Vt_, ld_, n); count_launches();
    lincomb_kernel<<<nb_, kThreads, 0, s_>>>(AV_, ld_, m, Y_, kMaxM, c, AVt_, ld_, n); count_launches();
    std::swap(V_, Vt_);
    std::swap(AV_, AVt_);
    vb_ok_ = 0;  // every column of V changed
    expand_h(Hh, hostla::congruence(m, c, compact(Hh, m), Qy), c);
    expand_h(Gh, hostla::congruence(m, c, compact(Gh, m), Qy), c);
    AJD_TRY(wait_stream());  // Y_ is reused by the next upload
    return JD_OK;
  };
  // Ritz extraction on the current basis: coefficient vectors Yc (m x m,
  // unit columns, best target first) and Rayleigh quotients th.
  // Harmonic (default): (H - sigma I) y = mu G y with
  // G = (AV - sigma V)^T (AV - sigma V), largest |mu| first -- the harmonic
  // Ritz values nearest sigma; the reported value is the Rayleigh quotient
  // y^T H y.  Standard: eigenpairs of H nearest sigma.
  auto extract = [&](int m, std::vector<double>& Yc, std::vector<double>& th) {
    std::vector<double> H = compact(Hh, m);
    std::vector<double> w, Z;
    std::vector<int> order(m);
    for (int i = 0; i < m; ++i) order[i] = i;
    bool harmonic = p_.extraction == 0;
    std::vector<double> Lc;
    if (harmonic) {
      Lc = compact(Gh, m);
      for (int j = 0; j < m; ++j)
        for (int i = j + 1; i < m; ++i) {
          const double v = 0.5 * (Lc[(size_t)j * m + i] + Lc[(size_t)i * m + j]);
          Lc[(size_t)j * m + i] = Lc[(size_t)i * m + j] = v;
        }
      harmonic = hostla::cholesky(m, Lc);
    }
    Yc.assign((size_t)m * m, 0.0);
    th.assign(m, 0.0);
    if (harmonic) {
      // C = L^{-1} (H - sigma I) L^{-T}
      std::vector<double> X = H;
      for (int i = 0; i < m; ++i) X[(size_t)i * m + i] -= sigma_;
      auto fwd = [&](std::vector<double>& B) {  // B <- L^{-1} B (columns)
        for (int j = 0; j < m; ++j)
          for (int i = 0; i < m; ++i) {
            double v = B[(size_t)j * m + i];
            for (int k = 0; k < i; ++k) v -= Lc[(size_t)k * m + i] * B[(size_t)j * m + k];
            B[(size_t)j * m + i] = v / Lc[(size_t)i * m + i];
          }
      };
      fwd(X);
      std::vector<double> Xt((size_t)m * m);
      for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) Xt[(size_t)j * m + i] = X[(size_t)i * m + j];
      fwd(Xt);  // = L^{-1} (L^{-1} (H - sigma I))^T = C
      hostla::jacobi_eig(m, Xt, w, Z);
      std::sort(order.begin(), order.end(), [&](int a, int b) { return std::fabs(w[a]) > std::fabs(w[b]); });
      for (int jj = 0; jj < m; ++jj) {
        const int j = order[jj];
        // y = L^{-T} z
        std::vector<double> y(m);
        for (int i = m - 1; i >= 0; --i) {
          double v = Z[(size_t)j * m + i];
          for (int k = i + 1; k < m; ++k) v -= Lc[(size_t)i * m + k] * y[k];
          y[i] = v / Lc[(size_t)i * m + i];
        }
        double nr = 0.0;
        for (double v : y) nr += v * v;
        nr = std::sqrt(nr);
        double rq = 0.0;
        for (int i = 0; i < m; ++i) {
          y[i] /= nr;
          Yc[(size_t)jj * m + i] = y[i];
        }
        for (int a = 0; a < m; ++a)
          for (int b = 0; b < m; ++b) rq += y[a] * H[(size_t)b * m + a] * y[b];
        th[jj] = rq;
      }
    } else {
      hostla::jacobi_eig(m, H, w, Z);
      std::sort(order.begin(), order.end(), [&](int a, int b) {
        const double da = std::fabs(w[a] - sigma_), db = std::fabs(w[b] - sigma_);
        return da != db ? da < db : w[a] < w[b];
      });
      for (int jj = 0; jj < m; ++jj) {
        th[jj] = w[order[jj]];
        for (int i = 0; i < m; ++i) Yc[(size_t)jj * m + i] = Z[(size_t)order[jj] * m + i];
      }
    }
  };

  // append t (orthogonalised against [Q V]) to V, A t to AV and the new
  // columns of H and G
  auto expand = [&]() -> int {
    double nrm = 0.0;
    AJD_TRY(cgs2(kc, m, t_, &nrm));
    int tries = 0;
    while (!(nrm > 1e-10) && tries < 3) {  // t in span: take a fresh random direction
      random_kernel<<<nb_, kThreads, 0, s_>>>(t_, n, ++reseed); count_launches();
      AJD_TRY(cgs2(kc, m, t_, &nrm));
      ++tries;
    }
    if (!(nrm > 0.0)) return fail(JD_EBREAKDOWN, "jd_solve: cannot expand the search space");
    scale_copy_kernel<<<nb_, kThreads, 0, s_>>>(t_, V_ + (int64_t)m * ld_, n, scal_, 0, 1); count_launches();
    vb_ok_ = std::min(vb_ok_, m);
    AJD_TRY(stencil_apply<double>(h_, 0.0, V_ + (int64_t)m * ld_, AV_ + (int64_t)m * ld_, 1, s_));
    AJD_TRY(dot_cols(Cols<double>{V_, ld_, m + 1}, Cols<double>{}, nullptr, AV_ + (int64_t)m * ld_, dots_));
    shifted_dots_kernel<<<nb_, kThreads, 0, s_>>>(V_, AV_, ld_, m + 1, sigma_, n, partial_); count_launches();
    reduce_partials_kernel<<<1, kRedThreads, 0, s_>>>(partial_, nb_, m + 1, dots_ + (m + 1), nullptr); count_launches();
    double d[2 * kMaxM + 2];
    AJD_TRY(sync_read(dots_, 2 * (m + 1), d));
    for (int i = 0; i <= m; ++i) {
      hget(Hh, i, m) = hget(Hh, m, i) = d[i];
      hget(Gh, i, m) = hget(Gh, m, i) = d[m + 1 + i];
    }
    ++m;
    return JD_OK;
  };
  while (true) {
    AJD_TRY(expand());
    ++outer;
    // --- Ritz extraction, selection, locking
    bool finished = false;
    while (true) {
      extract(m, Yc, th);
      theta0 = th[0];
      gap = std::numeric_limits<double>::infinity();
      for (int i = 1; i < m; ++i) gap = std::min(gap, std::fabs(th[i] - theta0));
      // u = V y1, Au = AV y1, r = Au - theta u, r -= Q Q^T r
      {
        std::vector<double> up(kMaxM, 0.0);
        for (int i = 0; i < m; ++i) up[i] = Yc[i];
        AJD_CUDA(cudaMemcpyAsync(Y_, up.data(), sizeof(double) * kMaxM, cudaMemcpyHostToDevice, s_));
        AJD_CUDA(cudaMemcpyAsync(theta_, &theta0, sizeof(double), cudaMemcpyHostToDevice, s_));
      }
      lincomb_kernel<<<nb_, kThreads, 0, s_>>>(V_, ld_, m, Y_, kMaxM, 1, u_, ld_, n); count_launches();
      lincomb_kernel<<<nb_, kThreads, 0, s_>>>(AV_, ld_, m, Y_, kMaxM, 1, Au_, ld_, n); count_launches();
      residual_kernel<<<nb_, kThreads, 0, s_>>>(Au_, u_, theta_, r_, n); count_launches();
      AJD_TRY(dot_cols(Cols<double>{r_, ld_, 1}, Cols<double>{}, nullptr, r_, scal_ + 1));
      double rr2;
      AJD_TRY(sync_read(scal_ + 1, 1, &rr2));
      rnorm = std::sqrt(std::max(rr2, 0.0));
      if (kc > 0) {
        Cols<double> Xq{Q_, ld_, kc};
        AJD_TRY(dot_cols(Xq, Cols<double>{}, nullptr, r_, dots_));
        multiaxpy_kernel<double><<<nb_, kThreads, 0, s_>>>(Xq, Cols<double>{}, dots_, r_, n); count_launches();
      }
      if (rnorm <= tol_ * normA_) {
        // lock u
        AJD_CUDA(cudaMemcpyAsync(Q_ + (int64_t)kc * ld_, u_, sizeof(double) * n, cudaMemcpyDeviceToDevice, s_));
        qb_ok_ = std::min(qb_ok_, kc);
        lam.push_back(theta0);
        if (trace_) std::fprintf(stderr, "jd LOCK %d theta=%.15g res=%.3e at outer %d\n", kc, theta0, rnorm / normA_, outer);
        // cache W = K^{-1} q and the Q^T W block for the projected preconditioner
        if (p_.precision == JD_FP32) AJD_TRY((cache_lock_column<float, float>(kc)));
        else if (p_.precision == JD_MIXED) AJD_TRY((cache_lock_column<double, float>(kc)));
        else AJD_TRY((cache_lock_column<double, double>(kc)));
        ++kc;
        steps_on_pair = 0;
        if (kc == kint_) {
          finished = true;
          break;
        }
        // deflate: keep span(V) minus u, orthonormal
        if (m > 1) {
          std::vector<double> Qy;
          hostla::orthonormalize(m, m, Yc, Qy);
          std::vector<double> rest(Qy.begin() + m, Qy.end());
          AJD_TRY(transform(m, m - 1, rest));
          --m;
        } else {
          m = 0;
          std::fill(Hh.begin(), Hh.end(), 0.0);
          std::fill(Gh.begin(), Gh.end(), 0.0);
        }
        // inject a fresh random direction: JD's correction cannot see other
        // eigenvectors of a (nearly) repeated eigenvalue once they have left
        // the search space
        if (m + 1 < jmax_) {
          random_kernel<<<nb_, kThreads, 0, s_>>>(t_, n, ++reseed); count_launches();
          AJD_TRY(expand());
        }
        continue;
      }
      break;
    }
    if (finished) break;
    if (kc >= k_ && steps_on_pair >= 30) break;  // guard pair stalled: k pairs are in hand
    if (outer >= p_.max_outer) {
      status = kc >= k_ ? JD_OK
                        : fail(JD_ENOCONV, "jd_solve: %d of %d eigenpairs after %d outer steps (residual %.3e)", kc,
                               k_, outer, rnorm / normA_);
      break;
    }
    // --- restart: keep the jmin best Ritz vectors (orthonormalised)
    if (m >= jmax_) {
      std::vector<double> keep(Yc.begin(), Yc.begin() + (size_t)m * jmin_), Qy;
      hostla::orthonormalize(m, jmin_, keep, Qy);
      AJD_TRY(transform(m, jmin_, Qy));
      m = jmin_;
      ++restarts;
    }
    // --- correction equation
    // correction shift: sigma until the target is resolved (residual below
    // switch_tol ||A|| and below half the distance to the next Ritz value)
    const bool resolved = rnorm <= p_.switch_tol * normA_ && rnorm <= 0.5 * gap;
    const double theta_hat = resolved ? theta0 : sigma_;
    if (trace_)
      std::fprintf(stderr, "jd outer %d m=%d kc=%d theta=%.15g res=%.3e gap=%.2e shift=%s\n", outer, m, kc, theta0,
                   rnorm / normA_, gap, resolved ? "theta" : "sigma");
    const double floor =
        p_.inner_floor > 0.0 ? p_.inner_floor : (p_.precision == JD_FP32 ? 1e-5 : p_.precision == JD_MIXED ? 1e-6 : 1e-8);
    const double rel = std::max(std::pow(p_.inner_decay, steps_on_pair + 1), floor);
    int its = 0;
    if (p_.precision == JD_FP32) AJD_TRY((correction<float, float>(kc, theta_hat, rel, &its)));
    else if (p_.precision == JD_MIXED) AJD_TRY((correction<double, float>(kc, theta_hat, rel, &its)));
    else AJD_TRY((correction<double, double>(kc, theta_hat, rel, &its)));
    inner_total_ += its;
    ++steps_on_pair;
    if (trace_) std::fprintf(stderr, "   inner its %d (rel tol %.2e)\n", its, rel);
  }
  // orthonormality of the final search-space basis, max |V^T V - I| (the
  // Gram-Schmidt of every expansion, its BF16 first pass included)
  {
    double borth = 0.0;
    for (int j = 0; j < m; ++j) {
      AJD_TRY(dot_cols(Cols<double>{V_, ld_, m}, Cols<double>{}, nullptr, V_ + (int64_t)j * ld_, dots_));
      double g[kMaxM];
      AJD_TRY(sync_read(dots_, m, g));
      for (int i = 0; i < m; ++i) borth = std::max(borth, std::fabs(g[i] - (i == j ? 1.0 : 0.0)));
    }
    if (st) st->basis_orth_error = borth;
  }
  if (gerr_) {
    int ge = 0;
    AJD_CUDA(cudaMemcpyAsync(&ge, gerr_, sizeof(int), cudaMemcpyDeviceToHost, s_));
    AJD_TRY(wait_stream());
    if (ge) return fail(JD_EDEVICE, "jd_solve: a tensor-core wait of the Gram-Schmidt timed out");
  }
  if (st) {
    st->outer_its = outer;
    st->inner_its = inner_total_;
    st->restarts = restarts;
  }
  const int rc = finalize(kc, lam.data(), evals, evecs, st);
  if (st) {
    st->solve_ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    st->kernel_launches = launch_counter() - launches0_;
    st->precond_calls = precond_calls_;
    st->precond_ms = precond_ms_;
    st->stencil_calls = stencil_calls_;
    st->stencil_ms = stencil_ms_;
  }
  if (rc != JD_OK) return rc;
  return status;
}

// Shift-and-invert Lanczos (Section 4.1, Eq. (4.2)): Lanczos vectors of
// (A - sigma I)^{-1}, each product a preconditioned SQMR solve (the same
// ILDL^T and kernels as the correction equation, no projection) to
// relative residual inner_floor (default 1e-10, the paper's stopping rule
// for this mode).  Full reorthogonalisation (CGS2) instead of implicit
// restarts: at most jmax (<= 64) Lanczos vectors.  The Ritz values nu of the
// tridiagonal T give lambda = sigma + 1/nu; the k + guard largest |nu| are
// taken when their residual estimates ||A - sigma I|| beta |z_last| / |nu|
// fall below tol ||A||, their Ritz vectors go through the same final
// Rayleigh-Ritz, residual check and ordering as run().
int JdSolver::lanczos(double* evals, double* evecs, jd_stats* st) {
  using Clock = std::chrono::steady_clock;
  const auto t0 = Clock::now();
  normA_ = h_->norm_bound();
  const int64_t n = h_->n;
  const int guard = p_.guard < 0 ? 0 : (p_.guard == 0 ? 2 : p_.guard);
  kint_ = (int)std::min<int64_t>(k_ + guard, n - 1);
  jmax_ = (int)std::min<int64_t>(p_.jmax > 0 ? std::min(p_.jmax, kMaxM) : kMaxM, n);
  if (jmax_ < kint_ + 1) jmax_ = std::min<int64_t>(kint_ + 1, n);
  jmin_ = 1;
  if (kint_ < 1 || jmax_ < kint_) return fail(JD_EINVAL, "jd_lanczos_solve: lattice too small for k = %d", k_);
  AJD_TRY(alloc());
  launches0_ = launch_counter();
  const uint64_t seed = p_.seed ? p_.seed : (h_->seed ^ 0xD1B54A32D192ED03ull);
  random_kernel<<<nb_, kThreads, 0, s_>>>(t_, n, seed); count_launches();
  double nrm = 0.0;
  AJD_TRY(cgs2(0, 0, t_, &nrm));
  if (!(nrm > 0.0)) return fail(JD_EBREAKDOWN, "jd_lanczos_solve: zero start vector");
  scale_copy_kernel<<<nb_, kThreads, 0, s_>>>(t_, V_, n, scal_, 0, 1); count_launches();
  vb_ok_ = 0;
  // the paper's 1e-10; a binary32 inner solve cannot get below ~1e-6 (its
  // Lanczos operator is then only that accurate)
  const double inner_tol = p_.inner_floor > 0.0 ? p_.inner_floor : (p_.precision == JD_FP32 ? 1e-6 : 1e-10);
  const int maxit = std::max(p_.max_inner, 2000);
  const double op_norm = normA_ + std::fabs(sigma_);  // bound on ||A - sigma I||
  std::vector<double> alpha, beta, w, Z;
  std::vector<int> order;
  int m = 0, steps = 0;
  bool converged = false;
  double worst = 0.0;
  for (int j = 0; j < jmax_; ++j) {
    int its = 0;
    double* vj = V_ + (int64_t)j * ld_;
    if (p_.precision == JD_FP32) AJD_TRY((sqmr_core<float, float>(0, sigma_, vj, 1.0, inner_tol, maxit, t_, &its)));
    else if (p_.precision == JD_MIXED) AJD_TRY((sqmr_core<double, float>(0, sigma_, vj, 1.0, inner_tol, maxit, t_, &its)));
    else AJD_TRY((sqmr_core<double, double>(0, sigma_, vj, 1.0, inner_tol, maxit, t_, &its)));
    inner_total_ += its;
    ++steps;
    // alpha_j = v_j^T w, then w orthogonalised against v_0..v_j (twice)
    AJD_TRY(dot_cols(Cols<double>{vj, ld_, 1}, Cols<double>{}, nullptr, t_, scal_ + 2));
    double aj;
    AJD_TRY(sync_read(scal_ + 2, 1, &aj));
    AJD_TRY(cgs2(0, j + 1, t_, &nrm));
    alpha.push_back(aj);
    m = j + 1;
    // Ritz values of T_m
    std::vector<double> T((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) {
      T[(size_t)i * m + i] = alpha[i];
      if (i + 1 < m) T[(size_t)i * m + i + 1] = T[(size_t)(i + 1) * m + i] = beta[i];
    }
    hostla::jacobi_eig(m, T, w, Z);
    order.resize(m);
    for (int i = 0; i < m; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return std::fabs(w[a]) > std::fabs(w[b]); });
    if (m >= kint_) {
      worst = 0.0;
      for (int q = 0; q < kint_; ++q) {
        const int i = order[q];
        const double est = op_norm * nrm * std::fabs(Z[(size_t)i * m + (m - 1)]) / std::max(std::fabs(w[i]), 1e-300);
        worst = std::max(worst, est);
      }
      if (trace_) std::fprintf(stderr, "lanczos step %d: beta %.3e worst estimate %.3e (inner its %d)\n", j, nrm,
                               worst / normA_, its);
      if (worst <= tol_ * normA_) {
        converged = true;
        break;
      }
    }
    if (!(nrm > 1e-14 * std::fabs(aj)) || m == jmax_) break;  // invariant subspace, or no room
    beta.push_back(nrm);
    scale_copy_kernel<<<nb_, kThreads, 0, s_>>>(t_, V_ + (int64_t)(j + 1) * ld_, n, scal_, 0, 1); count_launches();
    vb_ok_ = std::min(vb_ok_, j + 1);
  }
  // Ritz vectors of the kint largest |nu| into Q
  const int kc = std::min(kint_, m);
  {
    std::vector<double> up((size_t)kMaxM * kc, 0.0);
    for (int q = 0; q < kc; ++q)
      for (int i = 0; i < m; ++i) up[(size_t)q * kMaxM + i] = Z[(size_t)order[q] * m + i];
    AJD_CUDA(cudaMemcpyAsync(Y_, up.data(), sizeof(double) * kMaxM * kc, cudaMemcpyHostToDevice, s_));
    lincomb_kernel<<<nb_, kThreads, 0, s_>>>(V_, ld_, m, Y_, kMaxM, kc, Q_, ld_, n); count_launches();
    qb_ok_ = 0;
    AJD_TRY(wait_stream());
  }
  if (st) {
    st->outer_its = steps;
    st->inner_its = inner_total_;
    st->restarts = 0;
  }
  const int rc = finalize(kc, nullptr, evals, evecs, st);
  if (st) {
    st->solve_ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    st->kernel_launches = launch_counter() - launches0_;
    st->precond_calls = precond_calls_;
    st->precond_ms = precond_ms_;
    st->stencil_calls = stencil_calls_;
    st->stencil_ms = stencil_ms_;
  }
  if (rc != JD_OK) return rc;
  if (!converged)
    return fail(JD_ENOCONV, "jd_lanczos_solve: Ritz estimates %.3e after %d Lanczos steps (tol %.1e)", worst / normA_,
                steps, tol_);
  return JD_OK;
}

// Final Rayleigh–Ritz on the locked vectors, residuals, ordering, signs,
// copy-out.
int JdSolver::finalize(int kc, double* lam, double* evals, double* evecs, jd_stats* st) {
  (void)lam;
  const int kout = std::min(kc, k_);  // the k nearest of the locked pairs
  if (st) st->nconv = kout;
  if (kc == 0) return JD_OK;
  const int64_t n = n_;
  // A Q into AV_ (columns 0..kc), H = Q^T A Q
  for (int j = 0; j < kc; ++j)
    AJD_TRY(stencil_apply<double>(h_, 0.0, Q_ + (int64_t)j * ld_, AV_ + (int64_t)j * ld_, 1, s_));
  for (int j = 0; j < kc; ++j) {
    AJD_TRY(dot_cols(Cols<double>{Q_, ld_, j + 1}, Cols<double>{}, nullptr, AV_ + (int64_t)j * ld_, dots_));
    set_h_column_kernel<<<1, 128, 0, s_>>>(H_, kMaxM, j, dots_); count_launches();
  }
  AJD_TRY(rr(kc));  // eigenpairs of Q^T A Q ordered by |theta - sigma|
  lincomb_kernel<<<nb_, kThreads, 0, s_>>>(Q_, ld_, kc, Y_, kMaxM, kout, Vt_, ld_, n); count_launches();
  lincomb_kernel<<<nb_, kThreads, 0, s_>>>(AV_, ld_, kc, Y_, kMaxM, kout, AVt_, ld_, n); count_launches();
  double max_res = 0.0;
  std::vector<double> signs(kout);
  for (int j = 0; j < kout; ++j) {
    double* x = Vt_ + (int64_t)j * ld_;
    double* ax = AVt_ + (int64_t)j * ld_;
    AJD_TRY(dot_cols(Cols<double>{x, ld_, 1}, Cols<double>{}, nullptr, x, dots_));
    residual_kernel<<<nb_, kThreads, 0, s_>>>(ax, x, theta_ + j, r_, n); count_launches();
    AJD_TRY(dot_cols(Cols<double>{r_, ld_, 1}, Cols<double>{}, nullptr, r_, dots_ + 1));
    AJD_CUDA(cudaMemsetAsync(amax_, 0, sizeof(unsigned long long), s_));
    AJD_CUDA(cudaMemsetAsync(amax_ + 1, 0xFF, sizeof(unsigned long long), s_));
    max_abs_bits_kernel<<<nb_, kThreads, 0, s_>>>(x, n, amax_); count_launches();
    first_index_kernel<<<nb_, kThreads, 0, s_>>>(x, n, amax_, amax_ + 1); count_launches();
    double nn[2];
    AJD_TRY(sync_read(dots_, 2, nn));
    // readbacks on the solver's stream (never the legacy default stream,
    // which would serialise the device against concurrent solves)
    unsigned long long key = 0;
    AJD_CUDA(cudaMemcpyAsync(host_, amax_ + 1, sizeof(key), cudaMemcpyDeviceToHost, s_));
    AJD_TRY(wait_stream());
    std::memcpy(&key, host_, sizeof(key));
    const int64_t imax = (int64_t)key;
    double xv = 0.0;
    AJD_TRY(sync_read(x + imax, 1, &xv));
    const double nrm = std::sqrt(nn[0]);
    max_res = std::max(max_res, std::sqrt(std::max(nn[1], 0.0)) / nrm / normA_);
    signs[j] = (xv < 0 ? -1.0 : 1.0) / nrm;
  }
  AJD_CUDA(cudaMemcpyAsync(evals, theta_, sizeof(double) * kout, cudaMemcpyDefault, s_));
  for (int j = 0; j < kout; ++j) {
    double* x = Vt_ + (int64_t)j * ld_;
    AJD_CUDA(cudaMemcpyAsync(scal_ + 8, &signs[j], sizeof(double), cudaMemcpyHostToDevice, s_));
    scale_copy_kernel<<<nb_, kThreads, 0, s_>>>(x, x, n, scal_, 8, 0); count_launches();
    AJD_TRY(wait_stream());
  }
  double orth = 0.0;
  for (int j = 0; j < kout; ++j) {
    AJD_TRY(dot_cols(Cols<double>{Vt_, ld_, kout}, Cols<double>{}, nullptr, Vt_ + (int64_t)j * ld_, dots_));
    double g[kMaxM];
    AJD_TRY(sync_read(dots_, kout, g));
    for (int i = 0; i < kout; ++i) orth = std::max(orth, std::fabs(g[i] - (i == j ? 1.0 : 0.0)));
  }
  if (evecs) {
    for (int j = 0; j < kout; ++j)
      AJD_CUDA(cudaMemcpyAsync(evecs + (int64_t)j * n, Vt_ + (int64_t)j * ld_, sizeof(double) * n, cudaMemcpyDefault, s_));
  }
  AJD_TRY(wait_stream());
  if (st) {
    st->max_residual = max_res;
    st->orth_error = orth;
  }
  return JD_OK;
}

int normalize_jd_params(const jd_params* p, jd_params& prm);

int solve_problem(anderson_s* h, ildl_s* pc, const jd_params& prm, double sigma, int k, double tol, double* evals,
                  double* evecs, jd_stats* st, cudaStream_t s) {
  JdSolver solver(h, pc, prm, sigma, k, tol, s);
  return solver.run(evals, evecs, st);
}

}  // namespace ajd

using namespace ajd;

extern "C" int jd_params_default(jd_params* p) {
  if (!p) return fail(JD_EINVAL, "jd_params_default: NULL");
  std::memset(p, 0, sizeof(*p));
  p->max_outer = 3000;
  p->max_inner = 60;
  p->inner_decay = 0.7;
  p->inner_floor = 0.0;
  p->extraction = 0;
  p->guard = 0;
  p->switch_tol = 1e-3;
  p->precision = JD_FP64;
  ildl_params_default(&p->ildl);
  return JD_OK;
}

static int normalize_params(const jd_params* p, jd_params& prm);
int ajd::normalize_jd_params(const jd_params* p, jd_params& prm) { return normalize_params(p, prm); }

extern "C" int jd_solve(anderson_t h, double sigma, int k, double tol, const jd_params* p, double* evals,
                        double* evecs, jd_stats* st, void* stream) {
  if (!h || !evals) return fail(JD_EINVAL, "jd_solve: NULL handle or evals");
  if (!std::isfinite(sigma)) return fail(JD_EINVAL, "jd_solve: sigma must be finite");
  if (k < 1 || k > 64 || (int64_t)k >= h->n) return fail(JD_EINVAL, "jd_solve: need 1 <= k <= 64 and k < n");
  if (!(tol > 0.0)) return fail(JD_EINVAL, "jd_solve: tol must be > 0");
  jd_params prm;
  AJD_TRY(normalize_params(p, prm));
  if (st) std::memset(st, 0, sizeof(*st));
  using Clock = std::chrono::steady_clock;
  const auto t0 = Clock::now();
  ildl_t pc = prm.precond;
  bool own = false;
  if (!pc) {
    AJD_TRY(ildl_create_on_stream(h, sigma, &prm.ildl, &pc, reinterpret_cast<cudaStream_t>(stream),
                                  copy_for_precision(prm.precision)));
    own = true;
  }
  if (st) {
    st->setup_ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    ildl_info(pc, &st->ildl);
  }
  int rc;
  {
    JdSolver solver(h, pc, prm, sigma, k, tol, reinterpret_cast<cudaStream_t>(stream));
    rc = solver.run(evals, evecs, st);
  }
  if (own) ildl_destroy(pc);
  return rc;
}

extern "C" int jd_lanczos_solve(anderson_t h, double sigma, int k, double tol, const jd_params* p, double* evals,
                                double* evecs, jd_stats* st, void* stream) {
  if (!h || !evals) return fail(JD_EINVAL, "jd_lanczos_solve: NULL handle or evals");
  if (!std::isfinite(sigma)) return fail(JD_EINVAL, "jd_lanczos_solve: sigma must be finite");
  if (k < 1 || k > 60 || (int64_t)k >= h->n) return fail(JD_EINVAL, "jd_lanczos_solve: need 1 <= k <= 60 and k < n");
  if (!(tol > 0.0)) return fail(JD_EINVAL, "jd_lanczos_solve: tol must be > 0");
  jd_params prm;
  AJD_TRY(normalize_params(p, prm));
  if (st) std::memset(st, 0, sizeof(*st));
  using Clock = std::chrono::steady_clock;
  const auto t0 = Clock::now();
  ildl_t pc = prm.precond;
  bool own = false;
  if (!pc) {
    AJD_TRY(ildl_create_on_stream(h, sigma, &prm.ildl, &pc, reinterpret_cast<cudaStream_t>(stream),
                                  copy_for_precision(prm.precision)));
    own = true;
  }
  if (st) {
    st->setup_ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    ildl_info(pc, &st->ildl);
  }
  int rc;
  {
    JdSolver solver(h, pc, prm, sigma, k, tol, reinterpret_cast<cudaStream_t>(stream));
    rc = solver.lanczos(evals, evecs, st);
  }
  if (own) ildl_destroy(pc);
  return rc;
}

static int normalize_params(const jd_params* p, jd_params& prm) {
  jd_params_default(&prm);
  if (p) {
    prm = *p;
    jd_params d;
    jd_params_default(&d);
    if (prm.max_outer <= 0) prm.max_outer = d.max_outer;
    if (prm.max_inner <= 0) prm.max_inner = d.max_inner;
    if (!(prm.inner_decay > 0.0 && prm.inner_decay < 1.0)) prm.inner_decay = d.inner_decay;
    if (!(prm.inner_floor >= 0.0)) prm.inner_floor = d.inner_floor;
    if (prm.extraction != 0 && prm.extraction != 1) prm.extraction = d.extraction;
    if (!(prm.switch_tol > 0.0)) prm.switch_tol = d.switch_tol;
    if (prm.ildl.kappa == 0.0 && prm.ildl.max_levels == 0 && prm.ildl.n_dense == 0) {
      const double aggressive = prm.ildl.aggressive;  // the one field whose default is 0
      prm.ildl = d.ildl;
      prm.ildl.aggressive = aggressive;
    }
  }
  if (prm.precision != JD_FP64 && prm.precision != JD_FP32 && prm.precision != JD_MIXED)
    return fail(JD_EINVAL, "jd_solve: unknown precision");
  return JD_OK;
}

// ------------------------------------------------------------ batches ---
// Independent problems, pipelined: `setup_threads` host threads build the
// preconditioners of problems i+1, i+2, ... (host C++ with OpenMP, device
// upload on their own streams) while the calling thread solves problem i
// on `stream`.  At most setup_threads + 1 factors are alive at any time.
extern "C" int jd_solve_batch(const anderson_t* hs, int nprob, const double* sigma, const int* k, double tol,
                              const jd_params* p, double* const* evals, double* const* evecs, jd_stats* stats,
                              int setup_threads, void* stream) {
  if (nprob < 0 || (nprob > 0 && (!hs || !sigma || !k || !evals)))
    return fail(JD_EINVAL, "jd_solve_batch: bad arguments");
  if (!(tol > 0.0)) return fail(JD_EINVAL, "jd_solve_batch: tol must be > 0");
  for (int i = 0; i < nprob; ++i) {
    if (!hs[i] || !evals[i] || !std::isfinite(sigma[i]) || k[i] < 1 || k[i] > 64 || (int64_t)k[i] >= hs[i]->n)
      return fail(JD_EINVAL, "jd_solve_batch: bad problem %d", i);
  }
  if (nprob == 0) return JD_OK;
  jd_params prm;
  AJD_TRY(normalize_params(p, prm));
  if (prm.precond) return fail(JD_EINVAL, "jd_solve_batch: a prebuilt preconditioner is per problem; pass NULL");
  if (stats) std::memset(stats, 0, sizeof(jd_stats) * nprob);
  const int nthr = std::max(1, std::min(setup_threads > 0 ? setup_threads : 2, nprob));
  const int omp_total = std::max(1, omp_get_max_threads());
  // the host cores are shared by the setups: the solving thread waits on
  // the device in blocking synchronisation and needs almost no CPU
  const int omp_each = std::max(1, omp_total / nthr);
  int dev = 0;
  AJD_CUDA(cudaGetDevice(&dev));

  std::vector<ildl_t> pcs(nprob, nullptr);
  std::vector<int> setup_rc(nprob, JD_OK);
  std::vector<std::string> setup_msg(nprob);
  std::vector<double> setup_ms(nprob, 0.0);
  std::vector<char> ready(nprob, 0);
  std::mutex mu;
  std::condition_variable cv;
  std::atomic<int> next{0};
  int solved = 0;  // guarded by mu
  bool abort_all = false;

  auto worker = [&]() {
    cudaSetDevice(dev);
    omp_set_num_threads(omp_each);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= nprob) break;
      {
        std::unique_lock<std::mutex> lk(mu);  // bound the factors alive
        cv.wait(lk, [&] { return abort_all || i <= solved + nthr; });
        if (abort_all) break;
      }
      const auto t0 = std::chrono::steady_clock::now();
      ildl_t pc = nullptr;
      const int rc = ildl_create_on_stream(hs[i], sigma[i], &prm.ildl, &pc, st, copy_for_precision(prm.precision));
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      std::lock_guard<std::mutex> lk(mu);
      pcs[i] = pc;
      setup_rc[i] = rc;
      if (rc != JD_OK) setup_msg[i] = jd_last_error();
      setup_ms[i] = ms;
      ready[i] = 1;
      cv.notify_all();
    }
    if (st) cudaStreamDestroy(st);
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nthr; ++t) pool.emplace_back(worker);

  int status = JD_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // this thread's applies join the chain that the setup threads' autotuning
  // applies join too, so no two cooperative applies run at once
  const bool serialized = apply_serialization();
  set_apply_serialization(true);
  struct Restore {
    bool v;
    ~Restore() { set_apply_serialization(v); }
  } restore{serialized};
  for (int i = 0; i < nprob; ++i) {
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return ready[i] != 0; });
    }
    jd_stats* st = stats ? &stats[i] : nullptr;
    int rc = setup_rc[i];
    if (rc == JD_OK) {
      if (st) {
        st->setup_ms = setup_ms[i];
        ildl_info(pcs[i], &st->ildl);
      }
      JdSolver solver(hs[i], pcs[i], prm, sigma[i], k[i], tol, s);
      rc = solver.run(evals[i], evecs ? evecs[i] : nullptr, st);
      ildl_destroy(pcs[i]);
      pcs[i] = nullptr;
    } else {
      set_error_msg("%s", setup_msg[i].c_str());
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      ++solved;
      if (rc != JD_OK && rc != JD_ENOCONV) abort_all = true;
      cv.notify_all();
    }
    if (rc != JD_OK && status == JD_OK) status = rc;
    if (rc != JD_OK && rc != JD_ENOCONV) {
      // fatal: stop the pipeline; release what the workers built
      for (auto& t : pool) t.join();
      for (auto& pc : pcs) ildl_destroy(pc);
      return fail(rc, "jd_solve_batch: problem %d: %s", i, jd_last_error());
    }
  }
  for (auto& t : pool) t.join();
  return status;
}
