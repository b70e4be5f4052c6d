// The persistent preconditioner apply kernel (device code only): all phases
// of x = K^{-1} b in one cooperative launch.  Included by ildl.cu; kept in
// its own file so that measurements of this kernel can be tied to its
// source (bench.py keys recorded DRAM counters to this file's hash).
#pragma once
#include "ildl_impl.cuh"

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

}  // namespace
}  // namespace ajd
