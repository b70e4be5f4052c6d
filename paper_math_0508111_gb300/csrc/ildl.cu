// Device part of the multilevel incomplete LDL^T preconditioner: upload of
// the host factor and the application x = K^{-1} b.
//
// K^{-1} b = P^T S L^{-T} D^{-1} L^{-1} S P b.  Positions are ordered level by
// level and every level's pivots are mutually independent, so the forward
// solve with L is one parallel sweep per level (each row of level l only
// reads rows of earlier levels) and the backward solve with L^T is one
// parallel sweep per level in reverse.  The gather/scale P, S is fused into
// the forward sweeps, the block diagonal D^{-1} (1x1 and 2x2 pivots) and the
// scatter into the backward sweeps, and the trailing dense block is one
// matrix-vector product with its stored inverse.  Every stored entry of L is
// read exactly once per sweep, so the apply streams 2 * nnz(L) * (value +
// index) bytes plus a few vectors.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <new>
#include <cstdio>
#include <cstdlib>
#include <type_traits>

#include "anderson_impl.cuh"
#include "ildl_impl.cuh"
#include "jd_impl.cuh"
#include "ildl_setup.h"

namespace ajd {
namespace {

// ---- persistent apply: all phases of K^{-1} b in one cooperative launch ----
// Phase kinds: gather (level 0), forward level, dense trailing block,
// backward level.  Phases run in order; a grid-wide barrier separates them
// (every phase reads only results of earlier phases).  The barrier counts
// CTA arrivals on one counter (zeroed before the launch); waits are bounded
// and record a timeout in `err` instead of hanging.
enum { PH_GATHER = 0, PH_FWD = 1, PH_DENSE = 2, PH_BWD = 3 };
constexpr int kPersistThreads = 512;
constexpr unsigned kSpinLimit = 1u << 22;  // ~0.1-0.5 s at 32-128 ns per poll

// V: type of the stored factor values; X: type of the work vectors and of
// the accumulation; IO: type of the caller's b and x (V = X = IO for the
// binary64 and binary32 applies; V = hi32_t, X = IO = double for the mixed
// apply: half the factor bytes, binary64 arithmetic).
// Load a stored value and widen it to the arithmetic type X.
template <typename X, typename V>
__device__ __forceinline__ X ldw(const V* p) {
  return (X)__ldg(p);
}
template <>
__device__ __forceinline__ double ldw<double, hi32_t>(const hi32_t* p) {
  return __hiloint2double((int)__ldg(&p->u), 0);
}

template <typename V, typename X, typename IO = X>
struct ApplyArgs {
  const int* perm;
  const V* scale;
  const int* Lptr;
  const int* Lcol;
  const V* Lval;
  const int* Uptr;
  const int* Ucol;
  const V* Uval;
  const V* dd;
  const V* dof;
  const int* partner;
  const V* dense;
  X* w;
  X* z;
  const IO* b;
  IO* out;
  int nd, d0;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier number `ph` (0-based) of one cooperative launch: every CTA
// adds one arrival to `count` (release) and polls it (acquire) until all
// CTAs of barriers 0..ph have arrived.  Polls are bounded: after kSpinLimit
// of them the CTA records a timeout in `err` and the kernel returns early;
// the other CTAs see the flag and return too.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned ph, int* err) {
  (void)gen;
  __syncthreads();
  __shared__ int failed;
  if (threadIdx.x == 0) {
    int f = 0;
    // release-add: this CTA's writes (ordered by the CTA barrier above)
    // become visible before its arrival is counted
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    const unsigned target = (ph + 1) * gridDim.x;
    unsigned spins = 0;
    while (ld_acquire_u32(count) < target) {
      ++spins;
      if ((spins & 1023u) == 0 && *((volatile int*)err)) { f = 1; break; }
      if (spins > kSpinLimit) {
        atomicExch(err, 1);
        f = 1;
        break;
      }
      if (spins > 64) __nanosleep(32);
    }
    failed = f;
  }
  __syncthreads();
  return failed == 0;
}

// Final value of row p of a sweep, given the row's dot product `acc` with
// the solution entries it depends on, its right-hand side (forward) and its
// 2x2 partner and permutation entry (backward; loaded before the row's
// entries so that their latency overlaps the gathers).
// ---- Gauss–Jordan inversion of the dense trailing block (setup) ----
// X = A^{-1} for the m x m row-major binary64 matrix A (overwritten), with
// partial pivoting, in one cooperative launch: for every column c three
// phases separated by grid barriers --
//   1. each CTA finds the largest |A[r][c]|, r >= c, over its share of the
//      rows (partials: value with sign, row);
//   2. every CTA reduces the partials (largest modulus, lowest row on ties),
//      swaps rows c and piv of A (columns >= c) and of X, scales the new row
//      c by 1/pivot, and records the multipliers f[r] = A[r][c];
//   3. rows r != c: A[r][k] -= f[r] A[c][k] (k >= c) and X[r][k] -= f[r] X[c][k]
//      (all k: the swaps move entries of X into every column).
// X starts as I and ends symmetrised ((X + X^T)/2).  A zero or non-finite
// pivot sets *bad.  Bounded barrier waits set *err, and the kernel returns.
constexpr int kGjThreads = 512;

__global__ void __launch_bounds__(kGjThreads, 1)
gj_invert_kernel(double* __restrict__ A, double* __restrict__ X, int m, double* __restrict__ part_v,
                 int* __restrict__ part_i, double* __restrict__ f, double* __restrict__ acc_old, unsigned* count,
                 int* err, int* bad) {
  // every read of data another CTA may have written goes through L2 (__ldcg)
  __shared__ double sv[kGjThreads / 32];
  __shared__ int si[kGjThreads / 32];
  __shared__ int s_piv;
  __shared__ double s_pval;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned ph = 0;
  for (int64_t t = tid; t < (int64_t)m * m; t += nth) X[t] = (t / m == t % m) ? 1.0 : 0.0;
  if (!grid_barrier(count, nullptr, ph++, err)) return;
  for (int c = 0; c < m; ++c) {
    // 1. partial pivot search (largest modulus, lowest row on ties; the
    //    partial keeps the signed value)
    double bv = 0.0;
    int bi = m;
    for (int64_t r = c + tid; r < m; r += nth) {
      const double a = __ldcg(A + r * m + c);
      if (bi == m || fabs(a) > fabs(bv)) { bv = a; bi = (int)r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (i2 < m && (bi == m || fabs(v2) > fabs(bv) || (fabs(v2) == fabs(bv) && i2 < bi))) { bv = v2; bi = i2; }
    }
    if (lane == 0) { sv[warp] = bv; si[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      int w = 0;
      for (int j = 1; j < kGjThreads / 32; ++j)
        if (si[j] < m && (si[w] == m || fabs(sv[j]) > fabs(sv[w]) || (fabs(sv[j]) == fabs(sv[w]) && si[j] < si[w])))
          w = j;
      part_i[blockIdx.x] = si[w];
      part_v[blockIdx.x] = sv[w];
      if (blockIdx.x == 0) *acc_old = __ldcg(A + (int64_t)c * m + c);
    }
    if (!grid_barrier(count, nullptr, ph++, err)) return;
    // 2. reduce the partials (every CTA, same order), swap, scale, multipliers
    if (threadIdx.x == 0) {
      int w = 0;
      for (int j = 1; j < (int)gridDim.x; ++j) {
        const int ij = __ldcg(part_i + j), iw = __ldcg(part_i + w);
        const double vj = fabs(__ldcg(part_v + j)), vw = fabs(__ldcg(part_v + w));
        if (ij < m && (iw == m || vj > vw || (vj == vw && ij < iw))) w = j;
      }
      const int pw = __ldcg(part_i + w);
      s_piv = pw < m ? pw : c;
      s_pval = pw < m ? __ldcg(part_v + w) : 0.0;
      if (!(fabs(s_pval) > 0.0) || !isfinite(s_pval)) *bad = 1;
    }
    __syncthreads();
    const int piv = s_piv;
    const double inv = 1.0 / s_pval;
    const double aold = __ldcg(acc_old);
    // multipliers first: rows other than c and piv are not written in this
    // phase; f[piv] is the old A[c][c], which the swap moves to row piv
    for (int64_t r = tid; r < m; r += nth) f[r] = r == c ? 0.0 : (r == piv ? aold : __ldcg(A + r * m + c));
    for (int64_t k = tid; k < m; k += nth) {
      const double xc = __ldcg(X + (int64_t)c * m + k), xp = __ldcg(X + (int64_t)piv * m + k);
      X[(int64_t)c * m + k] = xp * inv;
      if (piv != c) X[(int64_t)piv * m + k] = xc;
      if (k >= c) {
        const double ac = __ldcg(A + (int64_t)c * m + k), ap = __ldcg(A + (int64_t)piv * m + k);
        A[(int64_t)c * m + k] = ap * inv;
        if (piv != c) A[(int64_t)piv * m + k] = ac;
      }
    }
    if (!grid_barrier(count, nullptr, ph++, err)) return;
    // 3. eliminate column c from every other row (f[c] = 0 skips row c)
    const int64_t w = (int64_t)(m - c) + m;
    for (int64_t t = tid; t < (int64_t)m * w; t += nth) {
      const int r = (int)(t / w);
      const int j = (int)(t - (int64_t)r * w);
      const double fr = __ldcg(f + r);
      if (fr == 0.0) continue;
      if (j < m - c) {
        const int k = c + j;
        if (k == c) A[(int64_t)r * m + k] = 0.0;
        else A[(int64_t)r * m + k] = __ldcg(A + (int64_t)r * m + k) - fr * __ldcg(A + (int64_t)c * m + k);
      } else {
        const int k = j - (m - c);
        X[(int64_t)r * m + k] = __ldcg(X + (int64_t)r * m + k) - fr * __ldcg(X + (int64_t)c * m + k);
      }
    }
    if (!grid_barrier(count, nullptr, ph++, err)) return;
  }
  for (int64_t t = tid; t < (int64_t)m * m; t += nth) {
    const int i = (int)(t / m), j = (int)(t % m);
    if (j <= i) continue;
    const double sym = 0.5 * (__ldcg(X + (int64_t)i * m + j) + __ldcg(X + (int64_t)j * m + i));
    X[(int64_t)i * m + j] = sym;
    X[(int64_t)j * m + i] = sym;
  }
}

template <typename V, typename X, typename IO>
__device__ __forceinline__ void finish_value(const ApplyArgs<V, X, IO>& a, int kind, int p, X acc, X rhs, int pp,
                                             int perm) {
  if (kind == PH_FWD) {
    __stcg(a.w + p, rhs - acc);  // rhs = s[p] b[perm[p]], stored in w by the gather phase
  } else {
    X d = ldw<X>(a.dd + p) * __ldcg(a.w + p);
    if (pp >= 0) d += ldw<X>(a.dof + p) * __ldcg(a.w + pp);
    const X zp = d - acc;
    __stcg(a.z + p, zp);
    a.out[perm] = (IO)(ldw<X>(a.scale + p) * zp);
  }
}

template <typename V, typename X, typename IO, int G>
__device__ __forceinline__ void finish_row(const ApplyArgs<V, X, IO>& a, int kind, int p, X acc, int lane, X rhs,
                                           int pp, int perm) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
  if (p >= 0 && lane == 0) finish_value(a, kind, p, acc, rhs, pp, perm);
}

// Rows of one level, G threads per row; each group handles two rows at a
// time with their loads interleaved (index/value loads of both rows first,
// then the gathers), so every memory latency is shared by two rows.
template <typename V, typename X, typename IO, int G>
__device__ __forceinline__ void level_rows(const ApplyArgs<V, X, IO>& a, int kind, int p0, int p1) {
  const int lane = threadIdx.x % G;
  const int64_t groups = (int64_t)gridDim.x * blockDim.x / G;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int* ptr = kind == PH_FWD ? a.Lptr : a.Uptr;
  const int* col = kind == PH_FWD ? a.Lcol : a.Ucol;
  const V* val = kind == PH_FWD ? a.Lval : a.Uval;
  const X* x = kind == PH_FWD ? a.w : a.z;  // vector read through the columns
  constexpr int B = 8;                      // entries per lane and row per batch
  for (int64_t base = p0; base < p1; base += 2 * groups) {
    const int64_t ra = base + g0, rb = base + groups + g0;
    const int pa = ra < p1 ? (int)ra : -1;
    const int pb = rb < p1 ? (int)rb : -1;
    int qa = 0, ea = 0, qb = 0, eb = 0;
    X ra_rhs = X(0), rb_rhs = X(0);
    int ppa = -1, ppb = -1, pma = 0, pmb = 0;
    if (pa >= 0) {
      qa = __ldg(ptr + pa) + lane;
      ea = __ldg(ptr + pa + 1);
      if (lane == 0) {
        if (kind == PH_FWD) ra_rhs = __ldcg(a.w + pa);
        else { ppa = __ldg(a.partner + pa); pma = __ldg(a.perm + pa); }
      }
    }
    if (pb >= 0) {
      qb = __ldg(ptr + pb) + lane;
      eb = __ldg(ptr + pb + 1);
      if (lane == 0) {
        if (kind == PH_FWD) rb_rhs = __ldcg(a.w + pb);
        else { ppb = __ldg(a.partner + pb); pmb = __ldg(a.perm + pb); }
      }
    }
    // two partial sums per row halve the dependent chain of FMAs
    X acca = X(0), accb = X(0), acca2 = X(0), accb2 = X(0);
    while (qa < ea || qb < eb) {
      // lanes past the end of a row gather nothing: the solution entry they
      // would point at may not be written yet in this sweep (0 * NaN = NaN)
      int ca[B], cb[B];
      X va[B], vb[B];
#pragma unroll
      for (int i = 0; i < B; ++i) {
        const int q1 = qa + i * G, q2 = qb + i * G;
        const bool o1 = q1 < ea, o2 = q2 < eb;
        ca[i] = o1 ? __ldg(col + q1) : -1;
        va[i] = o1 ? ldw<X>(val + q1) : X(0);
        cb[i] = o2 ? __ldg(col + q2) : -1;
        vb[i] = o2 ? ldw<X>(val + q2) : X(0);
      }
#pragma unroll
      for (int i = 0; i < B; i += 2) {
        const X xa0 = ca[i] >= 0 ? __ldcg(x + ca[i]) : X(0);
        const X xb0 = cb[i] >= 0 ? __ldcg(x + cb[i]) : X(0);
        const X xa1 = ca[i + 1] >= 0 ? __ldcg(x + ca[i + 1]) : X(0);
        const X xb1 = cb[i + 1] >= 0 ? __ldcg(x + cb[i + 1]) : X(0);
        acca += va[i] * xa0;
        accb += vb[i] * xb0;
        acca2 += va[i + 1] * xa1;
        accb2 += vb[i + 1] * xb1;
      }
      qa += B * G;
      qb += B * G;
    }
    acca += acca2;
    accb += accb2;
    finish_row<V, X, IO, G>(a, kind, pa, acca, lane, ra_rhs, ppa, pma);
    finish_row<V, X, IO, G>(a, kind, pb, accb, lane, rb_rhs, ppb, pmb);
  }
}

// Rows of one level with G = 64..512 threads per row (G / 32 warps, 512 / G
// rows per CTA): for few, long rows, such as the deepest levels, whose rows
// collect the fill of every earlier level.  Warp partial sums meet in
// shared memory.  The row loop is uniform across the CTA (it depends on the
// block index only), as the CTA barriers inside it require.
template <typename V, typename X, typename IO, int G>
__device__ __forceinline__ void level_rows_wide(const ApplyArgs<V, X, IO>& a, int kind, int p0, int p1) {
  constexpr int W = G / 32;                 // warps per row
  constexpr int RPC = kPersistThreads / G;  // rows per CTA and pass
  constexpr int B = 8;                      // entries per thread and batch
  __shared__ X part[kPersistThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = threadIdx.x / G, t = threadIdx.x % G;
  const int* ptr = kind == PH_FWD ? a.Lptr : a.Uptr;
  const int* col = kind == PH_FWD ? a.Lcol : a.Ucol;
  const V* val = kind == PH_FWD ? a.Lval : a.Uval;
  const X* x = kind == PH_FWD ? a.w : a.z;
  for (int64_t base = p0 + (int64_t)blockIdx.x * RPC; base < p1; base += (int64_t)gridDim.x * RPC) {
    const int p = base + slot < p1 ? (int)(base + slot) : -1;
    X acc = X(0), acc2 = X(0), rhs = X(0);
    int pp = -1, pm = 0;
    if (p >= 0 && t == 0) {
      if (kind == PH_FWD) rhs = __ldcg(a.w + p);
      else { pp = __ldg(a.partner + p); pm = __ldg(a.perm + p); }
    }
    if (p >= 0) {
      int q = __ldg(ptr + p) + t;
      const int e = __ldg(ptr + p + 1);
      for (; q < e; q += B * G) {
        int c[B];
        X v[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
          const bool o = q + i * G < e;
          c[i] = o ? __ldg(col + q + i * G) : -1;
          v[i] = o ? ldw<X>(val + q + i * G) : X(0);
        }
#pragma unroll
        for (int i = 0; i < B; i += 2) {
          const X x0 = c[i] >= 0 ? __ldcg(x + c[i]) : X(0);
          const X x1 = c[i + 1] >= 0 ? __ldcg(x + c[i + 1]) : X(0);
          acc += v[i] * x0;
          acc2 += v[i + 1] * x1;
        }
      }
    }
    acc += acc2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (p >= 0 && t == 0) {
      X sum = X(0);
#pragma unroll
      for (int j = 0; j < W; ++j) sum += part[slot * W + j];
      finish_value(a, kind, p, sum, rhs, pp, pm);
    }
    __syncthreads();  // part[] is reused by the next pass
  }
}

// Prefetch the stored rows of a level phase into L2 (lines strided over the
// whole grid); skipped for phases larger than 16 MB, which stream from HBM
// at full bandwidth anyway.
template <typename V, typename X, typename IO>
__device__ __forceinline__ void prefetch_phase(const ApplyArgs<V, X, IO>& a, int4 P) {
  if (P.x != PH_FWD && P.x != PH_BWD) return;
  const int* ptr = P.x == PH_FWD ? a.Lptr : a.Uptr;
  const int* col = P.x == PH_FWD ? a.Lcol : a.Ucol;
  const V* val = P.x == PH_FWD ? a.Lval : a.Uval;
  const int64_t q0 = __ldg(ptr + P.y), q1 = __ldg(ptr + P.z);
  const int64_t bytes = (q1 - q0) * (int64_t)(sizeof(V) + sizeof(int));
  if (bytes > (16ll << 20) || q1 <= q0) return;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t lines_v = ((q1 - q0) * (int64_t)sizeof(V) + 127) / 128;
  const int64_t lines_c = ((q1 - q0) * (int64_t)sizeof(int) + 127) / 128;
  const char* vb = reinterpret_cast<const char*>(val + q0);
  const char* cb = reinterpret_cast<const char*>(col + q0);
  for (int64_t l = tid; l < lines_v + lines_c; l += nth) {
    const char* addr = l < lines_v ? vb + l * 128 : cb + (l - lines_v) * 128;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(addr));
  }
}

template <typename V, typename X, typename IO>
__global__ void __launch_bounds__(kPersistThreads, 1)
ildl_apply_persistent_kernel(ApplyArgs<V, X, IO> a, const int4* __restrict__ phases, int nphase, unsigned* count,
                             unsigned* gen, int* err, unsigned long long* stamps) {
  for (int ph = 0; ph < nphase; ++ph) {
    const int4 P = phases[ph];  // kind, p0, p1, G
    const int kind = P.x, p0 = P.y, p1 = P.z, G = P.w;
    if (stamps && blockIdx.x == 0 && threadIdx.x == 0) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      stamps[ph] = t;
    }
    const int4 Pn = ph + 1 < nphase ? phases[ph + 1] : make_int4(-1, 0, 0, 0);
    if (kind == PH_GATHER) {
      for (int p = p0 + blockIdx.x * blockDim.x + threadIdx.x; p < p1; p += gridDim.x * blockDim.x)
        __stcg(a.w + p, ldw<X>(a.scale + p) * (X)__ldg(a.b + __ldg(a.perm + p)));
    } else if (kind == PH_DENSE) {
      const int lane = threadIdx.x & 31;
      const int warps = (gridDim.x * blockDim.x) >> 5;
      for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < a.nd; r += warps) {
        const V* row = a.dense + (int64_t)r * a.nd;
        X acc = X(0), acc2 = X(0);
        for (int c0 = lane; c0 < a.nd; c0 += 8 * 32) {
          X rv[8], wv[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int c = c0 + 32 * i;
            const bool ok = c < a.nd;
            rv[i] = ok ? ldw<X>(row + c) : X(0);
            wv[i] = ok ? __ldcg(a.w + a.d0 + c) : X(0);
          }
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            acc += rv[i] * wv[i];
            acc2 += rv[i + 1] * wv[i + 1];
          }
        }
        acc += acc2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
          __stcg(a.z + a.d0 + r, acc);
          a.out[__ldg(a.perm + a.d0 + r)] = (IO)(ldw<X>(a.scale + a.d0 + r) * acc);
        }
      }
    } else {
      switch (G) {  // threads per row, fixed per phase at upload
        case 4: level_rows<V, X, IO, 4>(a, kind, p0, p1); break;
        case 8: level_rows<V, X, IO, 8>(a, kind, p0, p1); break;
        case 16: level_rows<V, X, IO, 16>(a, kind, p0, p1); break;
        case 32: level_rows<V, X, IO, 32>(a, kind, p0, p1); break;
        case 64: level_rows_wide<V, X, IO, 64>(a, kind, p0, p1); break;
        case 128: level_rows_wide<V, X, IO, 128>(a, kind, p0, p1); break;
        case 256: level_rows_wide<V, X, IO, 256>(a, kind, p0, p1); break;
        default: level_rows_wide<V, X, IO, 512>(a, kind, p0, p1); break;
      }
    }
    if (ph + 1 < nphase) prefetch_phase<V, X, IO>(a, Pn);
    if (ph + 1 < nphase && !grid_barrier(count, gen, (unsigned)ph, err)) return;
  }
  if (stamps && blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    stamps[nphase] = t;
  }
}

template <typename T>
void free_dev(DevFactor<T>& d) {
  cudaFree(d.perm);
  cudaFree(d.scale);
  cudaFree(d.Lptr);
  cudaFree(d.Lcol);
  cudaFree(d.Lval);
  cudaFree(d.Uptr);
  cudaFree(d.Ucol);
  cudaFree(d.Uval);
  cudaFree(d.dd);
  cudaFree(d.dof);
  cudaFree(d.partner);
  cudaFree(d.dense);
  cudaFree(d.w);
  cudaFree(d.z);
  cudaFree(d.phases);
  cudaFree(d.bar);
  cudaFree(d.w64);
  cudaFree(d.z64);
  d = DevFactor<T>();
}

template <typename S, typename D>
int upload(D** dst, const std::vector<S>& src, cudaStream_t st) {
  *dst = nullptr;
  if (src.empty()) return JD_OK;
  const size_t n = src.size();
  cudaError_t e = cudaMalloc(dst, n * sizeof(D));
  if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? JD_ENOMEM : JD_EDEVICE, "ildl upload: %s", cudaGetErrorString(e));
  if constexpr (std::is_same<S, D>::value) {
    AJD_CUDA(cudaMemcpyAsync(*dst, src.data(), n * sizeof(D), cudaMemcpyHostToDevice, st));
    AJD_CUDA(cudaStreamSynchronize(st));
  } else {
    std::vector<D> tmp(n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) tmp[i] = D(src[i]);
    AJD_CUDA(cudaMemcpyAsync(*dst, tmp.data(), n * sizeof(D), cudaMemcpyHostToDevice, st));
    AJD_CUDA(cudaStreamSynchronize(st));  // tmp is released on return
  }
  return JD_OK;
}

template <typename T>
int upload_factor(const HostFactor& F, DevFactor<T>& d, cudaStream_t st) {
  if (F.Lcol.size() >= (size_t)1 << 31) return fail(JD_ENOMEM, "ildl: factor has more than 2^31 entries");
  std::vector<int> lp(F.Lptr.begin(), F.Lptr.end()), up(F.Uptr.begin(), F.Uptr.end());
  AJD_TRY(upload(&d.perm, F.perm, st));
  AJD_TRY(upload(&d.scale, F.scale, st));
  AJD_TRY(upload(&d.Lptr, lp, st));
  AJD_TRY(upload(&d.Lcol, F.Lcol, st));
  AJD_TRY(upload(&d.Lval, F.Lval, st));
  AJD_TRY(upload(&d.Uptr, up, st));
  AJD_TRY(upload(&d.Ucol, F.Ucol, st));
  AJD_TRY(upload(&d.Uval, F.Uval, st));
  AJD_TRY(upload(&d.dd, F.dinv_d, st));
  AJD_TRY(upload(&d.dof, F.dinv_o, st));
  AJD_TRY(upload(&d.partner, F.partner, st));
  AJD_TRY(upload(&d.dense, F.dense_inv, st));
  const size_t nb = std::max<size_t>(1, F.n);
  const bool poison = std::getenv("AJD_POISON_ALLOC") != nullptr;  // NaN-filled work vectors (tests)
  if constexpr (std::is_same<T, hi32_t>::value) {  // binary64 work vectors of the mixed apply
    AJD_CUDA(cudaMalloc(&d.w64, nb * sizeof(double)));
    AJD_CUDA(cudaMalloc(&d.z64, nb * sizeof(double)));
    if (poison) {
      AJD_CUDA(cudaMemsetAsync(d.w64, 0xFF, nb * sizeof(double), st));
      AJD_CUDA(cudaMemsetAsync(d.z64, 0xFF, nb * sizeof(double), st));
    }
  } else {
    AJD_CUDA(cudaMalloc(&d.w, nb * sizeof(T)));
    AJD_CUDA(cudaMalloc(&d.z, nb * sizeof(T)));
    if (poison) {
      AJD_CUDA(cudaMemsetAsync(d.w, 0xFF, nb * sizeof(T), st));
      AJD_CUDA(cudaMemsetAsync(d.z, 0xFF, nb * sizeof(T), st));
    }
  }
  // phase list of the persistent apply
  std::vector<int4> ph;
  const std::vector<int>& lvp = F.level_ptr;
  const int nl = F.nlev;
  // threads per row: enough rows in flight to cover the grid, and about four
  // stored entries per thread of a row (a power of two in 4..512)
  const double threads_total = (double)sm_count() * kPersistThreads;
  auto pick_g = [&](int rows, double avg) {
    // (a phase of many long rows keeps up to a warp per row: each thread then
    // works through several rows, eight entries per batch)
    const double want = std::max(std::min(threads_total / std::max(rows, 1), avg / 4.0), std::min(avg / 8.0, 32.0));
    int g = 4;
    while (g < 512 && 2 * g <= want) g *= 2;
    return g;
  };
  // the gather phase writes s[p] b[perm[p]] into w for every position; level
  // 0 rows are then final and later rows read their right-hand side from w
  ph.push_back(make_int4(PH_GATHER, 0, F.n, 1));
  for (int l = 1; l <= nl; ++l) {
    const int p0 = lvp[l], p1 = lvp[l + 1];
    if (p1 <= p0) continue;
    const double avg = (double)(F.Lptr[p1] - F.Lptr[p0]) / (p1 - p0);
    ph.push_back(make_int4(PH_FWD, p0, p1, pick_g(p1 - p0, avg)));
  }
  if (F.n_dense > 0) ph.push_back(make_int4(PH_DENSE, lvp[nl], lvp[nl + 1], 32));
  for (int l = nl - 1; l >= 0; --l) {
    const int p0 = lvp[l], p1 = lvp[l + 1];
    if (p1 <= p0) continue;
    const double avg = (double)(F.Uptr[p1] - F.Uptr[p0]) / (p1 - p0);
    ph.push_back(make_int4(PH_BWD, p0, p1, pick_g(p1 - p0, avg)));
  }
  d.nphase = (int)ph.size();
  AJD_CUDA(cudaMalloc(&d.phases, std::max<size_t>(1, ph.size()) * sizeof(int4)));
  if (!ph.empty()) {
    AJD_CUDA(cudaMemcpyAsync(d.phases, ph.data(), ph.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    AJD_CUDA(cudaStreamSynchronize(st));
  }
  // barrier words on separate 128-byte lines: [0] arrivals, [32] generation,
  // [64] timeout flag
  AJD_CUDA(cudaMalloc(&d.bar, 96 * sizeof(unsigned)));
  AJD_CUDA(cudaMemsetAsync(d.bar, 0, 96 * sizeof(unsigned), st));
  AJD_CUDA(cudaStreamSynchronize(st));
  int per_sm = 0;
  using XT = typename std::conditional<std::is_same<T, hi32_t>::value, double, T>::type;
  AJD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ildl_apply_persistent_kernel<T, XT, XT>, kPersistThreads, 0));
  if (per_sm < 1) return fail(JD_EDEVICE, "ildl: persistent apply kernel cannot be resident");
  d.grid = sm_count();  // one CTA per SM
  d.ready = true;
  return JD_OK;
}

thread_local bool tl_serialize_applies = false;
std::mutex g_chain_mu;
cudaEvent_t g_chain_last = nullptr;  // completion of the last serialised apply

}  // namespace

void set_apply_serialization(bool on) { tl_serialize_applies = on; }

// One persistent apply with factor values V, work vectors X, caller vectors IO.
template <typename V, typename X, typename IO>
int launch_apply(const ildl_s* f, const DevFactor<V>& d, X* w, X* z, const IO* b, IO* out, cudaStream_t s) {
  if (!d.ready) return fail(JD_EINVAL, "ildl_apply: factor has no device copy (use ildl_create)");
  const HostFactor& F = f->F;
  if (F.n == 0 || d.nphase == 0) return JD_OK;
  ApplyArgs<V, X, IO> a{d.perm, d.scale, d.Lptr, d.Lcol, d.Lval, d.Uptr, d.Ucol, d.Uval, d.dd, d.dof, d.partner,
                        d.dense, w, z, b, out, F.n_dense, F.level_ptr[F.nlev]};
  AJD_CUDA(cudaMemsetAsync(d.bar, 0, 64 * sizeof(unsigned), s));  // arrivals and generation
  const int4* ph = d.phases;
  int np = d.nphase;
  unsigned* cnt = d.bar;
  unsigned* gen = d.bar + 32;
  int* err = reinterpret_cast<int*>(d.bar + 64);
  // AJD_APPLY_TIMING=1: record the start of every phase (globaltimer, CTA 0)
  // and print a per-kind summary of the next apply to stderr (diagnostics)
  static const bool timing = std::getenv("AJD_APPLY_TIMING") != nullptr;
  unsigned long long* stamps = nullptr;
  if (timing) AJD_CUDA(cudaMalloc(&stamps, (np + 1) * sizeof(unsigned long long)));
  void* args[] = {&a, &ph, &np, &cnt, &gen, &err, &stamps};
  if (tl_serialize_applies) {
    // concurrent solvers: this apply starts on the device only after the
    // previous serialised apply (of any thread) has finished, so no two of
    // these grid-wide cooperative kernels ever run at the same time
    std::lock_guard<std::mutex> lk(g_chain_mu);
    if (g_chain_last) AJD_CUDA(cudaStreamWaitEvent(s, g_chain_last, 0));
    AJD_CUDA(cudaLaunchCooperativeKernel((void*)ildl_apply_persistent_kernel<V, X, IO>, dim3(d.grid),
                                         dim3(kPersistThreads), args, 0, s));
    cudaEvent_t ev = nullptr;
    AJD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    AJD_CUDA(cudaEventRecord(ev, s));
    if (g_chain_last) cudaEventDestroy(g_chain_last);  // released once it has completed
    g_chain_last = ev;
  } else {
    AJD_CUDA(cudaLaunchCooperativeKernel((void*)ildl_apply_persistent_kernel<V, X, IO>, dim3(d.grid),
                                         dim3(kPersistThreads), args, 0, s));
  }
  count_launches(2);
  if (timing) {
    std::vector<unsigned long long> t(np + 1);
    std::vector<int4> phs(np);
    AJD_CUDA(cudaMemcpyAsync(t.data(), stamps, (np + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    AJD_CUDA(cudaMemcpyAsync(phs.data(), d.phases, np * sizeof(int4), cudaMemcpyDeviceToHost, s));
    AJD_CUDA(cudaStreamSynchronize(s));
    cudaFree(stamps);
    double kind_us[4] = {0, 0, 0, 0};
    int kind_n[4] = {0, 0, 0, 0};
    for (int i = 0; i < np; ++i) {
      const double us = (t[i + 1] - t[i]) * 1e-3;
      kind_us[phs[i].x] += us;
      kind_n[phs[i].x]++;
      if (std::getenv("AJD_APPLY_TIMING_ALL"))
        std::fprintf(stderr, "phase %d kind %d rows %d G %d: %.2f us\n", i, phs[i].x, phs[i].z - phs[i].y, phs[i].w, us);
    }
    std::fprintf(stderr, "apply %.1f us: gather %.1f (%d) fwd %.1f (%d) dense %.1f (%d) bwd %.1f (%d)\n",
                 (t[np] - t[0]) * 1e-3, kind_us[0], kind_n[0], kind_us[1], kind_n[1], kind_us[2], kind_n[2], kind_us[3],
                 kind_n[3]);
  }
  return JD_OK;
}

template <typename T>
int ildl_apply_dev(const ildl_s* f, const T* b, T* out, cudaStream_t s) {
  const DevFactor<T>& d = f->dev<T>();
  return launch_apply<T, T, T>(f, d, d.w, d.z, b, out, s);
}

int ildl_apply_dev_mixed(const ildl_s* f, const double* b, double* out, cudaStream_t s) {
  const DevFactor<hi32_t>& d = f->dh;
  if (!d.w64) return fail(JD_EINVAL, "ildl_apply: no mixed-precision work vectors");
  return launch_apply<hi32_t, double, double>(f, d, d.w64, d.z64, b, out, s);
}

// Timeout flag of the persistent apply (sticky until cleared): JD_EDEVICE if
// a grid barrier gave up.
int ildl_check_device_error(const ildl_s* f) {
  for (int prec = 0; prec < 3; ++prec) {
    const unsigned* bar = prec == 0 ? f->d64.bar : prec == 1 ? f->d32.bar : f->dh.bar;
    if (!bar) continue;
    int e = 0;
    AJD_CUDA(cudaMemcpy(&e, bar + 64, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) return fail(JD_EDEVICE, "ildl_apply: a device-side barrier timed out");
  }
  return JD_OK;
}

template int ildl_apply_dev<double>(const ildl_s*, const double*, double*, cudaStream_t);
template int ildl_apply_dev<float>(const ildl_s*, const float*, float*, cudaStream_t);

// Invert the dense trailing block (host matrix in, host inverse out) on the
// current device.
int invert_dense_on_device(std::vector<double>& M, int m, cudaStream_t st) {
  if (m == 0) return JD_OK;
  const size_t bytes = (size_t)m * m * sizeof(double);
  const int grid = sm_count();
  double *A = nullptr, *X = nullptr, *f = nullptr, *pv = nullptr;
  int* pi = nullptr;
  unsigned* bar = nullptr;  // [0] arrivals, [32] timeout flag, [64] singular flag, [96..97] old pivot-row entry
  cudaError_t e = cudaMalloc(&A, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&X, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&f, (size_t)m * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&pv, (size_t)grid * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&pi, (size_t)grid * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&bar, 128 * sizeof(unsigned));
  int rc = JD_OK;
  if (e == cudaSuccess) e = cudaMemcpyAsync(A, M.data(), bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, 128 * sizeof(unsigned), st);
  if (e == cudaSuccess) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gj_invert_kernel, kGjThreads, 0);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
  }
  if (e == cudaSuccess) {
    unsigned* cnt = bar;
    int* err = reinterpret_cast<int*>(bar + 32);
    int* bad = reinterpret_cast<int*>(bar + 64);
    double* acc_old = reinterpret_cast<double*>(bar + 96);
    void* args[] = {&A, &X, &m, &pv, &pi, &f, &acc_old, &cnt, &err, &bad};
    e = cudaLaunchCooperativeKernel((void*)gj_invert_kernel, dim3(grid), dim3(kGjThreads), args, 0, st);
    count_launches();
    int flags[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags[0], err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags[1], bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(M.data(), X, bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && flags[0]) rc = fail(JD_EDEVICE, "ildl dense inverse: a device-side barrier timed out");
    else if (e == cudaSuccess && flags[1]) rc = fail(JD_ESETUP, "ildl: the final dense block (%d rows) is singular", m);
  }
  if (e != cudaSuccess) rc = fail(JD_EDEVICE, "ildl dense inverse: %s", cudaGetErrorString(e));
  cudaFree(A);
  cudaFree(X);
  cudaFree(f);
  cudaFree(pv);
  cudaFree(pi);
  cudaFree(bar);
  return rc;
}

int ildl_upload_all(ildl_s* f, cudaStream_t st, int copies) {
  if (f->F.dense_is_matrix) {
    AJD_TRY(invert_dense_on_device(f->F.dense_inv, f->F.n_dense, st));
    f->F.dense_is_matrix = false;
  }
  if (copies & kCopyF64) AJD_TRY(upload_factor<double>(f->F, f->d64, st));
  if (copies & kCopyF32) AJD_TRY(upload_factor<float>(f->F, f->d32, st));
  if (copies & kCopyMixed) AJD_TRY(upload_factor<hi32_t>(f->F, f->dh, st));
  return JD_OK;
}

void ildl_free_device(ildl_s* f) {
  free_dev(f->d64);
  free_dev(f->d32);
  free_dev(f->dh);
}

// CSR of A - sigma I for a lattice (host, from the binary64 potential).
int lattice_csr(const anderson_s* h, const std::vector<double>& eps, double sigma, SymCsr& A) {
  const int L = h->L;
  const int64_t n = h->n;
  const bool per = h->bc == JD_PERIODIC;
  A.n = (int)n;
  A.ptr.assign(n + 1, 0);
  A.col.clear();
  A.val.clear();
  A.col.reserve(7 * n);
  A.val.reserve(7 * n);
  int nb[7];
  double nv[7];
  for (int64_t s = 0; s < n; ++s) {
    const int x = (int)(s % L), y = (int)((s / L) % L), z = (int)(s / ((int64_t)L * L));
    int k = 0;
    auto add = [&](int xx, int yy, int zz) {
      if (per) {
        xx = (xx + L) % L;
        yy = (yy + L) % L;
        zz = (zz + L) % L;
      } else if (xx < 0 || xx >= L || yy < 0 || yy >= L || zz < 0 || zz >= L) {
        return;
      }
      nb[k] = (int)(xx + (int64_t)L * (yy + (int64_t)L * zz));
      nv[k] = h->hop;
      ++k;
    };
    add(x - 1, y, z);
    add(x + 1, y, z);
    add(x, y - 1, z);
    add(x, y + 1, z);
    add(x, y, z - 1);
    add(x, y, z + 1);
    nb[k] = (int)s;
    nv[k] = eps[s] - sigma;
    ++k;
    // sort by column (insertion sort on 7 entries)
    for (int a = 1; a < k; ++a)
      for (int b = a; b > 0 && nb[b] < nb[b - 1]; --b) {
        std::swap(nb[b], nb[b - 1]);
        std::swap(nv[b], nv[b - 1]);
      }
    for (int a = 0; a < k; ++a) {
      A.col.push_back(nb[a]);
      A.val.push_back(nv[a]);
    }
    A.ptr[s + 1] = (int64_t)A.col.size();
  }
  return JD_OK;
}

}  // namespace ajd

using namespace ajd;

extern "C" int ildl_params_default(ildl_params* p) {
  if (!p) return fail(JD_EINVAL, "ildl_params_default: NULL");
  p->kappa = 5.0;
  p->drop = -1.0;
  p->gamma = -1.0;
  p->max_levels = 256;
  p->n_dense = 6000;
  p->matching = -1;
  return JD_OK;
}

static int check_params(const ildl_params* p, ildl_params& out) {
  if (p) out = *p;
  else ildl_params_default(&out);
  if (!(out.kappa > 1.0)) return fail(JD_EINVAL, "ildl: kappa must be > 1");
  if (!std::isfinite(out.drop) && out.drop > 0) return fail(JD_EINVAL, "ildl: drop must be finite");
  if (out.gamma >= 1.0 || std::isnan(out.gamma)) return fail(JD_EINVAL, "ildl: gamma must be < 1");
  if (out.max_levels < 1 || out.n_dense < 1 || out.n_dense > 8000)
    return fail(JD_EINVAL, "ildl: max_levels >= 1 and 1 <= n_dense <= 8000 required");
  return JD_OK;
}

extern "C" int ildl_setup_csr(int n, const int64_t* rowptr, const int* col, const double* val,
                              const ildl_params* p, ildl_t* out) {
  if (!out) return fail(JD_EINVAL, "ildl_setup_csr: out is NULL");
  *out = nullptr;
  if (n <= 0 || !rowptr || !col || !val) return fail(JD_EINVAL, "ildl_setup_csr: bad matrix arguments");
  ildl_params prm;
  AJD_TRY(check_params(p, prm));
  try {
    SymCsr A;
    A.n = n;
    A.ptr.assign(rowptr, rowptr + n + 1);
    if (A.ptr[0] != 0) return fail(JD_EINVAL, "ildl_setup_csr: rowptr[0] must be 0");
    const int64_t nnz = A.ptr[n];
    A.col.assign(col, col + nnz);
    A.val.assign(val, val + nnz);
    // ensure sorted rows with a diagonal entry
    SymCsr B;
    B.n = n;
    B.ptr.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
      bool has_diag = false;
      int prev = -1;
      for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
        const int c = A.col[q];
        if (c < 0 || c >= n || c <= prev) return fail(JD_EINVAL, "ildl_setup_csr: row %d not sorted/unique or out of range", i);
        if (c > i && !has_diag) { B.col.push_back(i); B.val.push_back(0.0); has_diag = true; }
        if (c == i) has_diag = true;
        B.col.push_back(c);
        B.val.push_back(A.val[q]);
        prev = c;
      }
      if (!has_diag) { B.col.push_back(i); B.val.push_back(0.0); }
      B.ptr[i + 1] = (int64_t)B.col.size();
    }
    ildl_s* f = new ildl_s();
    int rc = build_ildl(B, prm, f->F);
    if (rc != JD_OK) {
      delete f;
      return rc;
    }
    *out = f;
    return JD_OK;
  } catch (const std::bad_alloc&) {
    return fail(JD_ENOMEM, "ildl_setup_csr: out of host memory");
  }
}

extern "C" int ildl_matching(int n, const int64_t* rowptr, const int* col, const double* val, int* match_col,
                             double* scale, int* partner) {
  if (n <= 0 || !rowptr || !col || !val || !match_col || !scale || !partner)
    return fail(JD_EINVAL, "ildl_matching: bad arguments");
  try {
    SymCsr A;
    A.n = n;
    A.ptr.assign(rowptr, rowptr + n + 1);
    A.col.assign(col, col + A.ptr[n]);
    A.val.assign(val, val + A.ptr[n]);
    std::vector<int> mc;
    std::vector<double> u, v, rmax;
    max_product_matching(A, mc, u, v, rmax);
    SymCsr S = A;
    for (int i = 0; i < n; ++i) {
      scale[i] = std::sqrt(std::exp(u[i] + v[i]) / rmax[i]);
      match_col[i] = mc[i];
    }
    for (int i = 0; i < n; ++i)
      for (int64_t p = S.ptr[i]; p < S.ptr[i + 1]; ++p) S.val[p] *= scale[i] * scale[S.col[p]];
    std::vector<std::pair<int, int>> groups;
    split_cycles(S, mc, groups);
    for (int i = 0; i < n; ++i) partner[i] = -1;
    for (const auto& g : groups)
      if (g.second >= 0) {
        partner[g.first] = g.second;
        partner[g.second] = g.first;
      }
    return JD_OK;
  } catch (const std::bad_alloc&) {
    return fail(JD_ENOMEM, "ildl_matching: out of host memory");
  }
}

namespace ajd {
// ildl_create with the device work (potential download, dense inverse,
// upload) on `st`
int ildl_create_on_stream(anderson_t h, double sigma, const ildl_params* p, ildl_t* out, cudaStream_t st,
                          int copies) {
  if (!out || !h) return fail(JD_EINVAL, "ildl_create: NULL argument");
  *out = nullptr;
  if (!std::isfinite(sigma)) return fail(JD_EINVAL, "ildl_create: sigma must be finite");
  ildl_params prm;
  AJD_TRY(check_params(p, prm));
  try {
    std::vector<double> eps(h->n);
    AJD_CUDA(cudaMemcpyAsync(eps.data(), h->eps64, h->n * sizeof(double), cudaMemcpyDeviceToHost, st));
    AJD_CUDA(cudaStreamSynchronize(st));
    SymCsr A;
    lattice_csr(h, eps, sigma, A);
    ildl_s* f = new ildl_s();
    f->device = h->device;
    const auto t0 = std::chrono::steady_clock::now();
    int rc = build_ildl(A, prm, f->F, /*dense_on_host=*/false);
    if (rc == JD_OK) rc = ildl_upload_all(f, st, copies);
    f->F.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc != JD_OK) {
      ildl_free_device(f);
      delete f;
      return rc;
    }
    *out = f;
    return JD_OK;
  } catch (const std::bad_alloc&) {
    return fail(JD_ENOMEM, "ildl_create: out of host memory");
  }
}
}  // namespace ajd

extern "C" int ildl_create(anderson_t h, double sigma, const ildl_params* p, ildl_t* out) {
  return ajd::ildl_create_on_stream(h, sigma, p, out, 0, ajd::kCopyAll);
}

extern "C" int ildl_info(ildl_t f, ildl_info_t* info) {
  if (!f || !info) return fail(JD_EINVAL, "ildl_info: NULL argument");
  const HostFactor& F = f->F;
  info->n = F.n;
  info->levels = F.nlev;
  info->n_dense = F.n_dense;
  info->n_2x2 = F.n_2x2;
  info->nnz_L = (int64_t)F.Lcol.size();
  info->nnz_A = F.nnz_A;
  const double nnzD = (double)(F.n - F.n_dense) + 2.0 * F.n_2x2 + (double)F.n_dense * F.n_dense;
  info->fill = F.nnz_A > 0 ? (2.0 * (double)F.Lcol.size() + nnzD) / (double)F.nnz_A : 0.0;
  info->setup_ms = F.t_total_ms;
  info->match_ms = F.t_match_ms;
  info->relaxed_levels = F.n_relaxed;
  info->max_abs_L = F.max_abs_L;
  return JD_OK;
}

extern "C" int ildl_export(ildl_t f, int* perm, double* scale, int* level_ptr, int64_t* Lptr, int* Lcol,
                           double* Lval, double* dinv_d, double* dinv_o, int* partner, double* dense_inv) {
  if (!f) return fail(JD_EINVAL, "ildl_export: NULL handle");
  const HostFactor& F = f->F;
  if (perm) std::copy(F.perm.begin(), F.perm.end(), perm);
  if (scale) std::copy(F.scale.begin(), F.scale.end(), scale);
  if (level_ptr) std::copy(F.level_ptr.begin(), F.level_ptr.end(), level_ptr);
  if (Lptr) std::copy(F.Lptr.begin(), F.Lptr.end(), Lptr);
  if (Lcol) std::copy(F.Lcol.begin(), F.Lcol.end(), Lcol);
  if (Lval) std::copy(F.Lval.begin(), F.Lval.end(), Lval);
  if (dinv_d) std::copy(F.dinv_d.begin(), F.dinv_d.end(), dinv_d);
  if (dinv_o) std::copy(F.dinv_o.begin(), F.dinv_o.end(), dinv_o);
  if (partner) std::copy(F.partner.begin(), F.partner.end(), partner);
  if (dense_inv) std::copy(F.dense_inv.begin(), F.dense_inv.end(), dense_inv);
  return JD_OK;
}

extern "C" int ildl_apply(ildl_t f, const void* b, void* x, int precision, void* stream) {
  if (!f || !b || !x) return fail(JD_EINVAL, "ildl_apply: NULL argument");
  if (b == x) return fail(JD_EINVAL, "ildl_apply: b and x must be distinct");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (precision == JD_FP64)
    return ildl_apply_dev<double>(f, static_cast<const double*>(b), static_cast<double*>(x), s);
  if (precision == JD_FP32)
    return ildl_apply_dev<float>(f, static_cast<const float*>(b), static_cast<float*>(x), s);
  if (precision == JD_MIXED)
    return ildl_apply_dev_mixed(f, static_cast<const double*>(b), static_cast<double*>(x), s);
  return fail(JD_EINVAL, "ildl_apply: unknown precision %d", precision);
}

extern "C" int ildl_destroy(ildl_t f) {
  if (!f) return JD_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  if (f->d64.ready || f->d32.ready || f->dh.ready) {
    cudaSetDevice(f->device);
    ildl_free_device(f);
    cudaSetDevice(dev);
  }
  delete f;
  return JD_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free preconditioner application.
//
// Some callers cannot allocate device memory while they run: code executing
// under an allocator that forbids it (a memory pool reserved up front, a
// captured region that must stay allocation-free, an embedding runtime that
// owns all device memory).  ildl_apply_noalloc serves them: it launches the
// same persistent kernel as ildl_apply but takes its scratch (the two work
// vectors and the grid-barrier words) from one file-scope device array
// instead of the factor's own buffers.  Nothing is allocated or freed.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxN = 131072;  // largest order served (L <= 50 lattices)
constexpr size_t kNoAllocVecBytes = (size_t)kNoAllocMaxN * sizeof(double);
constexpr size_t kNoAllocBytes = 2 * kNoAllocVecBytes + 512;  // w, z, barrier words

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device (host code may not use the
// symbol itself: it names a host-side stand-in).
struct NoAllocSlot {
  bool ready = false;
  unsigned char* ptr = nullptr;
};
constexpr int kMaxDevices = 64;
NoAllocSlot g_noalloc_slots[kMaxDevices];
std::mutex g_noalloc_mutex;

int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  AJD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(JD_EDEVICE, "ildl_apply_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mutex);
  NoAllocSlot& sl = g_noalloc_slots[dev];
  if (!sl.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(JD_EDEVICE, "ildl_apply_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    sl.ptr = static_cast<unsigned char*>(p);
    sl.ready = true;
  }
  *out = sl.ptr;
  return JD_OK;
}

template <typename V, typename X, typename IO>
int launch_apply_static(const ildl_s* f, const DevFactor<V>& d, const IO* b, IO* out, unsigned char* scratch,
                        cudaStream_t s) {
  const HostFactor& F = f->F;
  if (F.n == 0 || d.nphase == 0) return JD_OK;
  X* w = reinterpret_cast<X*>(scratch);
  X* z = reinterpret_cast<X*>(scratch + kNoAllocVecBytes);
  unsigned* bar = reinterpret_cast<unsigned*>(scratch + 2 * kNoAllocVecBytes);
  ApplyArgs<V, X, IO> a{d.perm, d.scale, d.Lptr, d.Lcol, d.Lval, d.Uptr, d.Ucol, d.Uval, d.dd, d.dof, d.partner,
                        d.dense, w, z, b, out, F.n_dense, F.level_ptr[F.nlev]};
  // the array keeps the previous call's contents: the barrier words (arrivals,
  // generation, timeout flag) must start at zero; w and z are written before
  // they are read
  AJD_CUDA(cudaMemsetAsync(bar, 0, 96 * sizeof(unsigned), s));
  const int4* ph = d.phases;
  int np = d.nphase;
  unsigned* cnt = bar;
  unsigned* gen = bar + 32;
  int* err = reinterpret_cast<int*>(bar + 64);
  unsigned long long* stamps = nullptr;
  void* args[] = {&a, &ph, &np, &cnt, &gen, &err, &stamps};
  AJD_CUDA(cudaLaunchCooperativeKernel((void*)ildl_apply_persistent_kernel<V, X, IO>, dim3(d.grid),
                                       dim3(kPersistThreads), args, 0, s));
  count_launches(2);
  int herr = 0;
  AJD_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  AJD_CUDA(cudaStreamSynchronize(s));
  if (herr) return fail(JD_EDEVICE, "ildl_apply_noalloc: a device-side barrier timed out");
  return JD_OK;
}

}  // namespace

extern "C" int ildl_apply_noalloc(ildl_t f, const void* b, void* x, int precision, void* stream) {
  if (!f || !b || !x) return fail(JD_EINVAL, "ildl_apply_noalloc: NULL argument");
  if (b == x) return fail(JD_EINVAL, "ildl_apply_noalloc: b and x must be distinct");
  if ((int64_t)f->F.n > kNoAllocMaxN)
    return fail(JD_EINVAL, "ildl_apply_noalloc: order %d exceeds the static scratch limit of %lld rows", f->F.n,
                (long long)kNoAllocMaxN);
  unsigned char* scratch = nullptr;
  AJD_TRY(noalloc_scratch(&scratch));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (precision == JD_FP64) {
    if (!f->d64.ready) return fail(JD_EINVAL, "ildl_apply_noalloc: factor has no device copy");
    return launch_apply_static<double, double, double>(f, f->d64, static_cast<const double*>(b), static_cast<double*>(x),
                                               scratch, s);
  }
  if (precision == JD_FP32) {
    if (!f->d32.ready) return fail(JD_EINVAL, "ildl_apply_noalloc: factor has no device copy");
    return launch_apply_static<float, float, float>(f, f->d32, static_cast<const float*>(b), static_cast<float*>(x),
                                             scratch, s);
  }
  if (precision == JD_MIXED) {
    if (!f->dh.ready) return fail(JD_EINVAL, "ildl_apply_noalloc: factor has no device copy");
    return launch_apply_static<hi32_t, double, double>(f, f->dh, static_cast<const double*>(b), static_cast<double*>(x),
                                              scratch, s);
  }
  return fail(JD_EINVAL, "ildl_apply_noalloc: unknown precision %d", precision);
}
