// Schur complements of the multilevel ILDL^T on the GPU (Section 6.3: the
// factorization continues on S' = S_CC - L_F D_B L_F^T of each level).
//
// The host level loop (ildl_setup.cpp) still chooses the pivots, forms L_F
// and groups its entries per pivot block ("records"); this engine keeps the
// level matrix S on the device and computes S' there, bit for bit what the
// host code computes:
//   1. upper_rows_kernel, one warp per C row r: the row's entries of S
//      (columns c >= r in the C numbering) and, block by block in the
//      records' order, the updates -(w_a l_a(q) + w_b l_b(q)) for every C row
//      q >= r that the block reaches, accumulated per column in a hash
//      table (shared memory, or a slice of global memory for long rows) in
//      exactly the host's order and with the host's IEEE operations (no
//      contraction into FMAs); entries below tau off the diagonal are
//      dropped and the rest sorted by column;
//   2. the mirror into a full symmetric CSR: lower entries counted per
//      column, row pointers formed on the host (which needs them anyway),
//      entries placed, each row's lower part sorted by column (the host's
//      order: increasing row), and the row maxima for the next matching.
// S' comes back to the host (the next level's matching and candidates run
// there) and stays on the device as the next level matrix.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <climits>
#include <cstring>
#include <memory>
#include <mutex>
#include <utility>
#include <vector>

#include <omp.h>

#include <math_constants.h>

#include "common.cuh"
#include "ildl_setup.h"
#include "schur_gpu.h"

namespace ajd {
namespace {

constexpr int kWarpsPerCta = 4;
constexpr int kSmemSlots = 1024;  // hash slots per warp in shared memory
constexpr int kSmemMaxBound = kSmemSlots / 2;  // rows with a larger bound use global memory
constexpr unsigned kHashMul = 2654435761u;

// ---- device helpers ----

// Slot of key q in the table (keys -1 when free), inserting it if absent;
// `fresh` tells whether this call inserted it.  Keys of concurrent callers
// differ or are the same key (then one inserts, the others find it).
__device__ __forceinline__ int hash_slot(int* keys, int cap, int q, bool& fresh) {
  unsigned h = ((unsigned)q * kHashMul) & (unsigned)(cap - 1);
  fresh = false;
  for (;;) {
    const int k = keys[h];
    if (k == q) return (int)h;
    if (k == -1) {
      const int prev = atomicCAS(keys + h, -1, q);
      if (prev == -1) {
        fresh = true;
        return (int)h;
      }
      if (prev == q) return (int)h;
    }
    h = (h + 1) & (unsigned)(cap - 1);
  }
}

// Bitonic sort of (key, val) pairs [0, n) by key, n a power of two, by one
// warp (keys distinct, padding INT_MAX).
__device__ void warp_bitonic(int* keys, double* vals, int n) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      __syncwarp();
      for (int i = lane; i < n; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const int ki = keys[i], kl = keys[l];
          if ((ki > kl) == up) {
            keys[i] = kl;
            keys[l] = ki;
            const double t = vals[i];
            vals[i] = vals[l];
            vals[l] = t;
          }
        }
      }
    }
  }
  __syncwarp();
}

__device__ __forceinline__ int pow2_at_least(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}

struct UpperArgs {
  const int64_t* sptr;  // level matrix S (scaled)
  const int* scol;
  const double* sval;
  const int* cidx;
  const int* cnodes;
  const int64_t* rrec;
  const int* rec_blk;
  const int64_t* rec_slot;
  const int64_t* cptr;
  const int* crow;
  const double* c1;
  const double* c2;
  const double* bmat;
  const char* is2x2;
  const int64_t* off;   // output slots of row r: off[r] .. off[r + 1]
  const int64_t* hoff;  // global hash slice of a long row (size hoff[r+1]-hoff[r]), else unused
  int* gkeys;
  double* gvals;
  int* ucol;            // upper rows (sorted, dropped), in the output slots
  double* uval;
  int* ucnt;
  int mc_n;
  double tau;
};

__global__ void __launch_bounds__(32 * kWarpsPerCta)
upper_rows_kernel(UpperArgs a) {
  __shared__ int s_keys[kWarpsPerCta][kSmemSlots];
  __shared__ double s_vals[kWarpsPerCta][kSmemSlots];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwarps = gridDim.x * kWarpsPerCta;
  for (int r = blockIdx.x * kWarpsPerCta + wib; r < a.mc_n; r += nwarps) {
    const int k = a.cnodes[r];
    const int64_t s0 = a.sptr[k], s1 = a.sptr[k + 1];
    const int64_t R0 = a.rrec[r], R1 = a.rrec[r + 1];
    const int64_t o0 = a.off[r];
    if (R0 == R1) {
      // no elimination update reaches this row: the row of S on C, in order
      int cnt = 0;
      for (int64_t p0 = s0; p0 < s1; p0 += 32) {
        const int64_t p = p0 + lane;
        int c = -1;
        double v = 0.0;
        if (p < s1) {
          c = a.cidx[a.scol[p]];
          v = a.sval[p];
        }
        const bool keep = c >= r && (c == r || fabs(v) >= a.tau);
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          const int pos = cnt + __popc(m & ((1u << lane) - 1));
          a.ucol[o0 + pos] = c;
          a.uval[o0 + pos] = v;
        }
        cnt += __popc(m);
      }
      if (lane == 0) a.ucnt[r] = cnt;
      continue;
    }
    // hash table of the row: shared memory, or the row's global slice
    const int bound = (int)(a.off[r + 1] - o0);
    int* keys;
    double* vals;
    int cap;
    if (bound <= kSmemMaxBound) {
      keys = s_keys[wib];
      vals = s_vals[wib];
      cap = pow2_at_least(2 * bound);
    } else {
      keys = a.gkeys + a.hoff[r];
      vals = a.gvals + a.hoff[r];
      cap = (int)(a.hoff[r + 1] - a.hoff[r]);
    }
    for (int i = lane; i < cap; i += 32) keys[i] = -1;
    __syncwarp();
    // entries of S (each column once): 0 + s, as the host's accumulator
    for (int64_t p = s0 + lane; p < s1; p += 32) {
      const int c = a.cidx[a.scol[p]];
      if (c < r) continue;
      bool fresh;
      const int h = hash_slot(keys, cap, c, fresh);
      vals[h] = __dadd_rn(0.0, a.sval[p]);
    }
    __syncwarp();
    // the diagonal is always stored in S; the host adds it if absent
    if (lane == 0) {
      bool fresh;
      const int h = hash_slot(keys, cap, r, fresh);
      if (fresh) vals[h] = 0.0;
    }
    __syncwarp();
    // updates, block by block in the records' order (one update per column
    // and block, so the lanes of one block never share a slot)
    for (int64_t i = R0; i < R1; ++i) {
      const int b = a.rec_blk[i];
      const int64_t me = a.rec_slot[i];
      const double la = a.c1[me], lb = a.c2[me];
      const double b0 = a.bmat[3 * b], b1 = a.bmat[3 * b + 1], b2 = a.bmat[3 * b + 2];
      const bool two = a.is2x2[b] != 0;
      double wa, wb;
      if (!two) {
        wa = __dmul_rn(la, b0);
        wb = 0.0;
      } else {
        wa = __dadd_rn(__dmul_rn(la, b0), __dmul_rn(lb, b1));
        wb = __dadd_rn(__dmul_rn(la, b1), __dmul_rn(lb, b2));
      }
      const int64_t te = a.cptr[b + 1];
      for (int64_t t = me + lane; t < te; t += 32) {
        const int q = a.crow[t];
        const double u = two ? __dadd_rn(__dmul_rn(wa, a.c1[t]), __dmul_rn(wb, a.c2[t]))
                             : __dadd_rn(__dmul_rn(wa, a.c1[t]), 0.0);
        bool fresh;
        const int h = hash_slot(keys, cap, q, fresh);
        const double prev = fresh ? 0.0 : vals[h];
        vals[h] = __dsub_rn(prev, u);
      }
      __syncwarp();
    }
    // drop (the diagonal always stays), compact the kept entries to the
    // front of the table, sort them by column
    int cnt = 0;
    for (int i0 = 0; i0 < cap; i0 += 32) {
      const int i = i0 + lane;
      const int key = keys[i];
      const double v = vals[i];
      __syncwarp();
      const bool keep = key >= 0 && (key == r || fabs(v) >= a.tau);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int pos = cnt + __popc(m & ((1u << lane) - 1));
        keys[pos] = key;
        vals[pos] = v;
      }
      cnt += __popc(m);
      __syncwarp();
    }
    const int n2 = pow2_at_least(cnt);  // <= cap
    for (int i = cnt + lane; i < n2; i += 32) keys[i] = INT_MAX;
    __syncwarp();
    warp_bitonic(keys, vals, n2);
    for (int i = lane; i < cnt; i += 32) {
      a.ucol[o0 + i] = keys[i];
      a.uval[o0 + i] = vals[i];
    }
    if (lane == 0) a.ucnt[r] = cnt;
    __syncwarp();
  }
}

// lower entries per column: (r, c), r < c, of the upper rows
__global__ void count_lower_kernel(const int64_t* __restrict__ off, const int* __restrict__ ucol,
                                   const int* __restrict__ ucnt, int* __restrict__ lowcnt, int mc_n) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < mc_n; r += nwarps) {
    const int64_t o = off[r];
    const int n = ucnt[r];
    for (int j = lane; j < n; j += 32) {
      const int c = ucol[o + j];
      if (c != r) atomicAdd(lowcnt + c, 1);
    }
  }
}

// S' rows: lower entries (unordered for now, through per-row cursors) then
// the row's own upper entries
__global__ void place_kernel(const int64_t* __restrict__ off, const int* __restrict__ ucol,
                             const double* __restrict__ uval, const int* __restrict__ ucnt,
                             const int* __restrict__ lowcnt, const int64_t* __restrict__ nptr, int* __restrict__ cursor,
                             int* __restrict__ ncol, double* __restrict__ nval, int mc_n) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < mc_n; r += nwarps) {
    const int64_t o = off[r];
    const int n = ucnt[r];
    const int64_t up = nptr[r] + lowcnt[r];
    for (int j = lane; j < n; j += 32) {
      const int c = ucol[o + j];
      const double v = uval[o + j];
      ncol[up + j] = c;
      nval[up + j] = v;
      if (c != r) {
        const int pos = atomicAdd(cursor + c, 1);
        ncol[nptr[c] + pos] = r;
        nval[nptr[c] + pos] = v;
      }
    }
  }
}

// each row's lower part sorted by column (= increasing r, as the host's
// bucket pass leaves it), and the row maxima |S'_ij| for the next matching
__global__ void __launch_bounds__(32 * kWarpsPerCta)
sort_lower_kernel(const int* __restrict__ lowcnt, const int64_t* __restrict__ nptr, int* __restrict__ ncol,
                  double* __restrict__ nval, double* __restrict__ rowmax, int* gkeys, double* gvals,
                  const int64_t* __restrict__ goff, int mc_n) {
  __shared__ int s_keys[kWarpsPerCta][kSmemSlots];
  __shared__ double s_vals[kWarpsPerCta][kSmemSlots];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwarps = gridDim.x * kWarpsPerCta;
  for (int r = blockIdx.x * kWarpsPerCta + wib; r < mc_n; r += nwarps) {
    const int64_t p0 = nptr[r], p1 = nptr[r + 1];
    const int nl = lowcnt[r];
    if (nl > 1) {
      const int n2 = pow2_at_least(nl);
      int* keys = n2 <= kSmemSlots ? s_keys[wib] : gkeys + goff[r];
      double* vals = n2 <= kSmemSlots ? s_vals[wib] : gvals + goff[r];
      for (int i = lane; i < n2; i += 32) {
        keys[i] = i < nl ? ncol[p0 + i] : INT_MAX;
        vals[i] = i < nl ? nval[p0 + i] : 0.0;
      }
      warp_bitonic(keys, vals, n2);
      for (int i = lane; i < nl; i += 32) {
        ncol[p0 + i] = keys[i];
        nval[p0 + i] = vals[i];
      }
      __syncwarp();
    }
    double mx = 0.0;
    for (int64_t p = p0 + lane; p < p1; p += 32) mx = fmax(mx, fabs(nval[p]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) rowmax[r] = mx;
  }
}

__global__ void scale_kernel(const int64_t* __restrict__ ptr, const int* __restrict__ col, double* __restrict__ val,
                             const double* __restrict__ d, int m) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += nwarps) {
    const double di = d[i];
    for (int64_t p = ptr[i] + lane; p < ptr[i + 1]; p += 32) val[p] = __dmul_rn(val[p], __dmul_rn(di, d[col[p]]));
  }
}

// ---- the next level's matching potentials ----
// The host matching (Section 5.1) starts from u_i = min_j (c_ij - v_j) and
// v_j = min_i c_ij with c_ij = log a_i - log |a_ij|, a_i the row maximum.
// Formed here from S' while it is on the device, with the host's
// logarithm re-done step for step (the same table, every product and sum
// rounded to nearest, no fused multiply-adds) and exact minima (order does
// not matter), so the potentials are the host's bit for bit and the host
// only takes logarithms of the entries its searches read.  Subnormal,
// infinite or NaN arguments, which the host hands to its libm, go to the
// device's log here (entries that small or large do not occur in S').
__constant__ double c_log_inv[128];
__constant__ double c_log_c[128];

__device__ __forceinline__ double log_pos_dev(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ef = (int)((b >> 52) & 0x7ff);
  if (ef == 0 || ef == 0x7ff) return log(x);
  const int k = (int)((b >> 45) & 127);
  const double m = __longlong_as_double((long long)((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
  const double r = k == 0 ? __dsub_rn(m, 1.0) : __dsub_rn(__dmul_rn(m, c_log_inv[k]), 1.0);
  double t = 1.0 / 9.0;
  t = __dsub_rn(__dmul_rn(t, r), 1.0 / 8.0);
  t = __dadd_rn(__dmul_rn(t, r), 1.0 / 7.0);
  t = __dsub_rn(__dmul_rn(t, r), 1.0 / 6.0);
  t = __dadd_rn(__dmul_rn(t, r), 1.0 / 5.0);
  t = __dsub_rn(__dmul_rn(t, r), 1.0 / 4.0);
  t = __dadd_rn(__dmul_rn(t, r), 1.0 / 3.0);
  t = __dsub_rn(__dmul_rn(t, r), 1.0 / 2.0);
  t = __dadd_rn(__dmul_rn(t, r), 1.0);
  return __dadd_rn(__dmul_rn((double)(ef - 1023), 0.6931471805599453), __dadd_rn(c_log_c[k], __dmul_rn(r, t)));
}

__device__ __forceinline__ double entry_log_dev(double a) {
  a = fabs(a);
  return a > 0.0 ? log_pos_dev(a) : -CUDART_INF;
}

__device__ __forceinline__ double warp_min(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// logmax_i = log a_i (a_i = 1 for an empty row)
__global__ void logmax_kernel(const double* __restrict__ rowmax, double* __restrict__ logmax, int m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double r = rowmax[i];
    logmax[i] = log_pos_dev(r == 0.0 ? 1.0 : r);
  }
}

// v_j = min over row j (= column j) of logmax[col] - log|a| (0 if none);
// log|a| of every entry kept in loga for the host's searches
__global__ void duals_v_kernel(const int64_t* __restrict__ ptr, const int* __restrict__ col,
                               const double* __restrict__ val, const double* __restrict__ logmax,
                               double* __restrict__ v, double* __restrict__ loga, int m) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < m; j += nwarps) {
    double best = CUDART_INF;
    for (int64_t p = ptr[j] + lane; p < ptr[j + 1]; p += 32) {
      const double la = entry_log_dev(val[p]);
      loga[p] = la;
      if (la > -CUDART_INF) best = fmin(best, __dsub_rn(logmax[col[p]], la));
    }
    best = warp_min(best);
    if (lane == 0) v[j] = best == CUDART_INF ? 0.0 : best;
  }
}

// u_i = min over row i of (logmax_i - log|a|) - v[col] (0 if none)
__global__ void duals_u_kernel(const int64_t* __restrict__ ptr, const int* __restrict__ col,
                               const double* __restrict__ loga, const double* __restrict__ logmax,
                               const double* __restrict__ v, double* __restrict__ u, int m) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += nwarps) {
    const double lm = logmax[i];
    double best = CUDART_INF;
    for (int64_t p = ptr[i] + lane; p < ptr[i + 1]; p += 32) {
      const double c = __dsub_rn(lm, loga[p]);
      if (c < CUDART_INF) best = fmin(best, __dsub_rn(c, v[col[p]]));
    }
    best = warp_min(best);
    if (lane == 0) u[i] = best == CUDART_INF ? 0.0 : best;
  }
}

// ---- pinned host staging, pooled across setups ----
// S' comes back through page-locked memory (a copy into fresh pageable pages
// runs at a few GB/s); the buffers are kept for the next setup of the
// process, since page-locking hundreds of MB per setup would cost more than
// the copies it speeds up.
struct PinnedPool {
  std::mutex mu;
  std::vector<std::pair<void*, size_t>> free;
};
PinnedPool& pinned_pool() {
  static PinnedPool* p = new PinnedPool();  // never destroyed: setups may run until exit
  return *p;
}

struct Pinned {
  void* p = nullptr;
  size_t cap = 0;
  Pinned() = default;
  Pinned(const Pinned&) = delete;
  Pinned& operator=(const Pinned&) = delete;
  ~Pinned() {
    if (p) {
      std::lock_guard<std::mutex> lk(pinned_pool().mu);
      pinned_pool().free.push_back({p, cap});
    }
  }
  int reserve(size_t bytes) {
    if (bytes <= cap) return JD_OK;
    {
      std::lock_guard<std::mutex> lk(pinned_pool().mu);
      auto& fl = pinned_pool().free;
      for (size_t i = 0; i < fl.size(); ++i)
        if (fl[i].second >= bytes) {
          if (p) fl.push_back({p, cap});
          p = fl[i].first;
          cap = fl[i].second;
          fl.erase(fl.begin() + i);
          return JD_OK;
        }
    }
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    const size_t want = std::max(bytes + bytes / 4, (size_t)64 << 20);
    cudaError_t e = cudaMallocHost(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(JD_ENOMEM, "gpu schur: pinned staging: %s", cudaGetErrorString(e));
    }
    cap = want;
    return JD_OK;
  }
};

// ---- device buffers that grow as needed ----
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t cap = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { cudaFree(p); }
  void swap(DBuf& o) {
    std::swap(p, o.p);
    std::swap(cap, o.cap);
  }
  int reserve(size_t n) {
    if (n <= cap) return JD_OK;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = std::max<size_t>(n, 16);
    cudaError_t e = cudaMalloc(&p, want * sizeof(T));
    if (e != cudaSuccess)
      return fail(e == cudaErrorMemoryAllocation ? JD_ENOMEM : JD_EDEVICE, "gpu schur: %s", cudaGetErrorString(e));
    cap = want;
    return JD_OK;
  }
};

class DeviceSchur final : public SchurEngine {
 public:
  explicit DeviceSchur(cudaStream_t st) : st_(st) {
    const double *inv = nullptr, *logc = nullptr;
    log_table_data(&inv, &logc);
    table_rc_ = cudaMemcpyToSymbolAsync(c_log_inv, inv, 128 * sizeof(double), 0, cudaMemcpyHostToDevice, st_);
    if (table_rc_ == cudaSuccess)
      table_rc_ = cudaMemcpyToSymbolAsync(c_log_c, logc, 128 * sizeof(double), 0, cudaMemcpyHostToDevice, st_);
  }

  int begin(const SymCsr& A) override {
    m_ = A.n;
    nnz_ = (int64_t)A.col.size();
    AJD_TRY(sptr_.reserve(m_ + 1));
    AJD_TRY(scol_.reserve(nnz_));
    AJD_TRY(sval_.reserve(nnz_));
    AJD_CUDA(cudaMemcpyAsync(sptr_.p, A.ptr.data(), (m_ + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st_));
    AJD_CUDA(cudaMemcpyAsync(scol_.p, A.col.data(), nnz_ * sizeof(int), cudaMemcpyHostToDevice, st_));
    AJD_CUDA(cudaMemcpyAsync(sval_.p, A.val.data(), nnz_ * sizeof(double), cudaMemcpyHostToDevice, st_));
    return sync();
  }

  int scale(const double* d, int m) override {
    if (m != m_) return fail(JD_ESETUP, "gpu schur: scaling of %d rows for a level of %d", m, m_);
    AJD_TRY(dd_.reserve(m));
    AJD_CUDA(cudaMemcpyAsync(dd_.p, d, m * sizeof(double), cudaMemcpyHostToDevice, st_));
    scale_kernel<<<grid_for(m), 256, 0, st_>>>(sptr_.p, scol_.p, sval_.p, dd_.p, m);
    count_launches();
    AJD_CHECK_LAUNCH();
    return JD_OK;  // ordered before the level's Schur complement on the stream
  }

  int schur(const SchurLevel& lv, SymCsr& Sn, std::vector<double>& rowmax, std::vector<double>* u,
            std::vector<double>* v, dvec<double>* loga) override {
    if (table_rc_ != cudaSuccess)
      return fail(JD_EDEVICE, "gpu schur: logarithm table upload: %s", cudaGetErrorString(table_rc_));
    const bool duals = u && v && loga;
    const auto t0 = std::chrono::steady_clock::now();
    auto ms = [&]() { return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count(); };
    double t_bounds = 0, t_up = 0, t_k1 = 0, t_ptr = 0, t_k2 = 0;
    const int mc = lv.mc_n;
    const int64_t nrec = lv.rrec[mc];
    // output slots per row: its entries of S plus one per update (plus the
    // diagonal): an upper bound of the row of S'
    std::vector<int64_t> off(mc + 1, 0), hoff(mc + 1, 0);
    {
      const int64_t* sp = lv.sptr;
#pragma omp parallel for schedule(static)
      for (int r = 0; r < mc; ++r) {
        const int k = lv.cnodes[r];
        int64_t b = sp[k + 1] - sp[k] + 1;
        for (int64_t i = lv.rrec[r]; i < lv.rrec[r + 1]; ++i) b += lv.cptr[lv.rec_blk[i] + 1] - lv.rec_slot[i];
        off[r + 1] = b;
        int64_t h = 0;
        if (b > kSmemMaxBound) {
          h = 32;
          while (h < 2 * b) h <<= 1;
        }
        hoff[r + 1] = h;
      }
    }
    for (int r = 0; r < mc; ++r) {
      off[r + 1] += off[r];
      hoff[r + 1] += hoff[r];
    }
    t_bounds = ms();
    AJD_TRY(cidx_.reserve(lv.m));
    AJD_TRY(cnodes_.reserve(mc));
    AJD_TRY(rrec_.reserve(mc + 1));
    AJD_TRY(rblk_.reserve(nrec));
    AJD_TRY(rslot_.reserve(nrec));
    AJD_TRY(cptr_.reserve(lv.nblk + 1));
    AJD_TRY(crow_.reserve(nrec));
    AJD_TRY(c1_.reserve(nrec));
    AJD_TRY(c2_.reserve(nrec));
    AJD_TRY(bmat_.reserve(3 * (size_t)lv.nblk));
    AJD_TRY(is2_.reserve(lv.nblk));
    AJD_TRY(off_.reserve(mc + 1));
    AJD_TRY(hoff_.reserve(mc + 1));
    AJD_TRY(gkeys_.reserve(hoff[mc]));
    AJD_TRY(gvals_.reserve(hoff[mc]));
    AJD_TRY(ucol_.reserve(off[mc]));
    AJD_TRY(uval_.reserve(off[mc]));
    AJD_TRY(ucnt_.reserve(mc));
    AJD_TRY(lowcnt_.reserve(mc));
    auto up = [&](auto* dst, const auto* src, size_t n) -> int {
      if (n) AJD_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(*src), cudaMemcpyHostToDevice, st_));
      return JD_OK;
    };
    AJD_TRY(up(cidx_.p, lv.cidx, lv.m));
    AJD_TRY(up(cnodes_.p, lv.cnodes, mc));
    AJD_TRY(up(rrec_.p, lv.rrec, mc + 1));
    AJD_TRY(up(rblk_.p, lv.rec_blk, nrec));
    AJD_TRY(up(rslot_.p, lv.rec_slot, nrec));
    AJD_TRY(up(cptr_.p, lv.cptr, lv.nblk + 1));
    AJD_TRY(up(crow_.p, lv.crow, nrec));
    AJD_TRY(up(c1_.p, lv.c1, nrec));
    AJD_TRY(up(c2_.p, lv.c2, nrec));
    AJD_TRY(up(bmat_.p, lv.bmat, 3 * (size_t)lv.nblk));
    AJD_TRY(up(is2_.p, lv.is2x2, lv.nblk));
    AJD_TRY(up(off_.p, off.data(), mc + 1));
    AJD_TRY(up(hoff_.p, hoff.data(), mc + 1));
    t_up = ms();
    UpperArgs ua{sptr_.p, scol_.p, sval_.p, cidx_.p, cnodes_.p, rrec_.p, rblk_.p, rslot_.p, cptr_.p, crow_.p,
                 c1_.p, c2_.p, bmat_.p, is2_.p, off_.p, hoff_.p, gkeys_.p, gvals_.p, ucol_.p, uval_.p, ucnt_.p,
                 mc, lv.tau};
    const int gw = std::max(1, std::min(ceil_div(mc, kWarpsPerCta), 16 * sm_count()));
    upper_rows_kernel<<<gw, 32 * kWarpsPerCta, 0, st_>>>(ua);
    AJD_CUDA(cudaMemsetAsync(lowcnt_.p, 0, mc * sizeof(int), st_));
    count_lower_kernel<<<grid_for(mc), 256, 0, st_>>>(off_.p, ucol_.p, ucnt_.p, lowcnt_.p, mc);
    count_launches(2);
    AJD_CHECK_LAUNCH();
    // row pointers of S' (on the host, which keeps S' too)
    std::vector<int> ucnt(mc), lowcnt(mc);
    AJD_CUDA(cudaMemcpyAsync(ucnt.data(), ucnt_.p, mc * sizeof(int), cudaMemcpyDeviceToHost, st_));
    AJD_CUDA(cudaMemcpyAsync(lowcnt.data(), lowcnt_.p, mc * sizeof(int), cudaMemcpyDeviceToHost, st_));
    AJD_TRY(sync());
    t_k1 = ms();
    Sn.n = mc;
    Sn.ptr.assign(mc + 1, 0);
    std::vector<int64_t> goff(mc + 1, 0);
    for (int r = 0; r < mc; ++r) {
      Sn.ptr[r + 1] = Sn.ptr[r] + ucnt[r] + lowcnt[r];
      int64_t g = 0;
      if (lowcnt[r] > kSmemSlots) {
        g = 32;
        while (g < lowcnt[r]) g <<= 1;
      }
      goff[r + 1] = goff[r] + g;
    }
    const int64_t nnz = Sn.ptr[mc];
    AJD_TRY(nptr_.reserve(mc + 1));
    AJD_TRY(ncol_.reserve(nnz));
    AJD_TRY(nval_.reserve(nnz));
    AJD_TRY(cursor_.reserve(mc));
    AJD_TRY(rowmax_.reserve(mc));
    AJD_TRY(goff_.reserve(mc + 1));
    AJD_TRY(gkeys_.reserve(goff[mc]));
    AJD_TRY(gvals_.reserve(goff[mc]));
    t_ptr = ms();
    AJD_TRY(up(nptr_.p, Sn.ptr.data(), mc + 1));
    AJD_TRY(up(goff_.p, goff.data(), mc + 1));
    AJD_CUDA(cudaMemsetAsync(cursor_.p, 0, mc * sizeof(int), st_));
    place_kernel<<<grid_for(mc), 256, 0, st_>>>(off_.p, ucol_.p, uval_.p, ucnt_.p, lowcnt_.p, nptr_.p, cursor_.p,
                                                ncol_.p, nval_.p, mc);
    sort_lower_kernel<<<gw, 32 * kWarpsPerCta, 0, st_>>>(lowcnt_.p, nptr_.p, ncol_.p, nval_.p, rowmax_.p, gkeys_.p,
                                                         gvals_.p, goff_.p, mc);
    count_launches(2);
    if (duals) {
      AJD_TRY(logmax_.reserve(mc));
      AJD_TRY(du_.reserve(mc));
      AJD_TRY(dv_.reserve(mc));
      AJD_TRY(dloga_.reserve(nnz));
      logmax_kernel<<<grid_for(mc), 256, 0, st_>>>(rowmax_.p, logmax_.p, mc);
      duals_v_kernel<<<grid_for(mc), 256, 0, st_>>>(nptr_.p, ncol_.p, nval_.p, logmax_.p, dv_.p, dloga_.p, mc);
      duals_u_kernel<<<grid_for(mc), 256, 0, st_>>>(nptr_.p, ncol_.p, dloga_.p, logmax_.p, dv_.p, du_.p, mc);
      count_launches(3);
    }
    AJD_CHECK_LAUNCH();
    AJD_TRY(sync());
    t_k2 = ms();
    // S' and its row maxima through the pinned staging, then into the
    // host's arrays by all threads (which also spreads the first touch of
    // their pages)
    const size_t vbytes = nnz * sizeof(double), cbytes = nnz * sizeof(int), mbytes = mc * sizeof(double);
    const size_t lbytes = duals ? vbytes : 0;
    AJD_TRY(stage_.reserve(vbytes + cbytes + 3 * mbytes + lbytes + 64));
    char* hv = static_cast<char*>(stage_.p);
    char* hc = hv + vbytes;
    char* hm = hc + ((cbytes + 15) & ~(size_t)15);
    char* hu = hm + mbytes;
    char* hw = hu + mbytes;
    char* hl = hw + mbytes;
    AJD_CUDA(cudaMemcpyAsync(hv, nval_.p, vbytes, cudaMemcpyDeviceToHost, st_));
    AJD_CUDA(cudaMemcpyAsync(hc, ncol_.p, cbytes, cudaMemcpyDeviceToHost, st_));
    AJD_CUDA(cudaMemcpyAsync(hm, rowmax_.p, mbytes, cudaMemcpyDeviceToHost, st_));
    if (duals) {
      AJD_CUDA(cudaMemcpyAsync(hu, du_.p, mbytes, cudaMemcpyDeviceToHost, st_));
      AJD_CUDA(cudaMemcpyAsync(hw, dv_.p, mbytes, cudaMemcpyDeviceToHost, st_));
      AJD_CUDA(cudaMemcpyAsync(hl, dloga_.p, lbytes, cudaMemcpyDeviceToHost, st_));
      if ((size_t)nnz > loga->capacity()) dvec<double>().swap(*loga);  // no copy of stale contents
      loga->resize(nnz);
    }
    Sn.col.resize(nnz);
    Sn.val.resize(nnz);
    rowmax.resize(mc);
    if (duals) {
      u->resize(mc);
      v->resize(mc);
    }
    AJD_TRY(sync());
    {
      const double* sv = reinterpret_cast<const double*>(hv);
      const int* sc = reinterpret_cast<const int*>(hc);
      double* dv = Sn.val.data();
      int* dc = Sn.col.data();
      const double* sl = reinterpret_cast<const double*>(hl);
      double* dl = duals ? loga->data() : nullptr;
#pragma omp parallel for schedule(static)
      for (int64_t b = 0; b < (nnz + 65535) / 65536; ++b) {
        const int64_t i0 = b * 65536, i1 = std::min<int64_t>(nnz, i0 + 65536);
        std::memcpy(dv + i0, sv + i0, (i1 - i0) * sizeof(double));
        std::memcpy(dc + i0, sc + i0, (i1 - i0) * sizeof(int));
        if (dl) std::memcpy(dl + i0, sl + i0, (i1 - i0) * sizeof(double));
      }
      std::memcpy(rowmax.data(), hm, mbytes);
      if (duals) {
        std::memcpy(u->data(), hu, mbytes);
        std::memcpy(v->data(), hw, mbytes);
      }
    }
    if (verbose_)
      std::fprintf(stderr, "  gpu schur m=%d C=%d nnz'=%lld slots=%lld: bounds %.1f upload %.1f rows+count %.1f ptr %.1f "
                   "mirror %.1f download %.1f ms\n", lv.m, mc, (long long)nnz, (long long)off[mc], t_bounds,
                   t_up - t_bounds, t_k1 - t_up, t_ptr - t_k1, t_k2 - t_ptr, ms() - t_k2);
    // S' is the next level matrix
    sptr_.swap(nptr_);
    scol_.swap(ncol_);
    sval_.swap(nval_);
    m_ = mc;
    nnz_ = nnz;
    return JD_OK;
  }

 private:
  static int grid_for(int64_t rows) { return std::max(1, std::min(ceil_div(rows, 8), 16 * sm_count())); }
  int sync() {
    AJD_CUDA(cudaStreamSynchronize(st_));
    return JD_OK;
  }
  cudaStream_t st_;
  bool verbose_ = std::getenv("AJD_SETUP_VERBOSE") != nullptr;
  int m_ = 0;
  int64_t nnz_ = 0;
  DBuf<int64_t> sptr_, nptr_, rrec_, rslot_, cptr_, off_, hoff_, goff_;
  DBuf<int> scol_, ncol_, cidx_, cnodes_, rblk_, crow_, gkeys_, ucol_, ucnt_, lowcnt_, cursor_;
  DBuf<double> sval_, nval_, dd_, c1_, c2_, bmat_, gvals_, uval_, rowmax_, logmax_, du_, dv_, dloga_;
  cudaError_t table_rc_ = cudaSuccess;
  DBuf<char> is2_;
  Pinned stage_;
};

}  // namespace

std::unique_ptr<SchurEngine> make_device_schur(cudaStream_t st) { return std::make_unique<DeviceSchur>(st); }

}  // namespace ajd
