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
// the sums; IO: type of the caller's b and x.  binary64 apply: V = X = IO =
// double; binary32: all float; mixed: V = float, X = df64, IO = double --
// binary32 factor values, work vectors and sums carried as unevaluated
// float pairs (about 48 significant bits) in FP32-pipe arithmetic, binary64
// only at the gather and the final scaling.

// hi + lo with |lo| <= ulp(hi)/2: a float-float number.
struct __align__(8) df64 {
  float hi, lo;
};

// Register type of a factor value in the products: the value type itself,
// float for the float-float sums.
template <typename V, typename X>
struct ValueReg {
  using type = X;
};
template <>
struct ValueReg<float, df64> {
  using type = float;
};

template <typename W, typename V>
__device__ __forceinline__ W ldw(const V* p) {
  return (W)__ldg(p);
}

// ---- arithmetic of the sweeps, per work type ----
// zero, acc += v * x (mac), a + b, a - b, v * x, shuffles, L2 loads/stores,
// conversions from and to the caller's type.  The float-float forms use the
// error-free transformations of Dekker and Knuth (TwoSum, FMA-based
// TwoProduct): the product v * x.hi is split into its rounded value and
// exact error, and every addition carries its rounding error into lo.
template <typename X>
__device__ __forceinline__ X zero() {
  return X(0);
}
template <>
__device__ __forceinline__ df64 zero<df64>() {
  return df64{0.f, 0.f};
}

template <typename X, typename W>
__device__ __forceinline__ void mac(X& acc, W v, X x) {
  acc = fma((X)v, x, acc);
}
__device__ __forceinline__ void mac(df64& acc, float v, df64 x) {
  const float p = v * x.hi;
  float e = fmaf(v, x.hi, -p);
  e = fmaf(v, x.lo, e);
  const float t = acc.hi + p;  // TwoSum(acc.hi, p)
  const float bp = t - acc.hi;
  const float err = (acc.hi - (t - bp)) + (p - bp);
  acc.hi = t;
  acc.lo += err + e;
}

__device__ __forceinline__ df64 quick_two_sum(float a, float b) {
  const float s = a + b;
  return df64{s, b - (s - a)};
}

template <typename X>
__device__ __forceinline__ X add(X a, X b) {
  return a + b;
}
__device__ __forceinline__ df64 add(df64 a, df64 b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  return quick_two_sum(s, e + a.lo + b.lo);
}
template <typename X>
__device__ __forceinline__ X sub(X a, X b) {
  return a - b;
}
__device__ __forceinline__ df64 sub(df64 a, df64 b) {
  return add(a, df64{-b.hi, -b.lo});
}
template <typename X, typename W>
__device__ __forceinline__ X mul(W v, X x) {
  return (X)v * x;
}
__device__ __forceinline__ df64 mul(float v, df64 x) {
  const float p = v * x.hi;
  float e = fmaf(v, x.hi, -p);
  e = fmaf(v, x.lo, e);
  return quick_two_sum(p, e);
}
template <typename X>
__device__ __forceinline__ X norm(X a) {
  return a;
}
__device__ __forceinline__ df64 norm(df64 a) {
  return quick_two_sum(a.hi, a.lo);
}

template <typename X>
__device__ __forceinline__ X shfl_xor(X v, int o, int w) {
  return __shfl_xor_sync(0xffffffffu, v, o, w);
}
__device__ __forceinline__ df64 shfl_xor(df64 v, int o, int w) {
  return df64{__shfl_xor_sync(0xffffffffu, v.hi, o, w), __shfl_xor_sync(0xffffffffu, v.lo, o, w)};
}

template <typename X>
__device__ __forceinline__ X ldx(const X* p) {
  return __ldcg(p);
}
__device__ __forceinline__ df64 ldx(const df64* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return df64{v.x, v.y};
}
template <typename X>
__device__ __forceinline__ void stx(X* p, X v) {
  __stcg(p, v);
}
__device__ __forceinline__ void stx(df64* p, df64 v) {
  __stcg(reinterpret_cast<float2*>(p), make_float2(v.hi, v.lo));
}

template <typename X, typename IO>
__device__ __forceinline__ X from_io(IO v) {
  return (X)v;
}
template <>
__device__ __forceinline__ df64 from_io<df64, double>(double v) {
  const float hi = __double2float_rn(v);
  return df64{hi, __double2float_rn(v - (double)hi)};
}
template <typename IO, typename X>
__device__ __forceinline__ IO to_io(X v) {
  return (IO)v;
}
template <>
__device__ __forceinline__ double to_io<double, df64>(df64 v) {
  return (double)v.hi + (double)v.lo;
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
  using W = typename ValueReg<V, X>::type;
  if (kind == PH_FWD) {
    stx(a.w + p, sub(rhs, acc));  // rhs = s[p] b[perm[p]], stored in w by the gather phase
  } else {
    X d = mul(ldw<W>(a.dd + p), ldx(a.w + p));
    if (pp >= 0) d = add(d, mul(ldw<W>(a.dof + p), ldx(a.w + pp)));
    const X zp = sub(d, acc);
    stx(a.z + p, zp);
    a.out[perm] = to_io<IO>(mul(ldw<W>(a.scale + p), zp));
  }
}

template <typename V, typename X, typename IO, int G>
__device__ __forceinline__ void finish_row(const ApplyArgs<V, X, IO>& a, int kind, int p, X acc, int lane, X rhs,
                                           int pp, int perm) {
  acc = norm(acc);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc = add(acc, shfl_xor(acc, o, G));
  if (p >= 0 && lane == 0) finish_value(a, kind, p, acc, rhs, pp, perm);
}

// Rows of one level, G threads per row; each group handles two rows at a
// time with their loads interleaved (index/value loads of both rows first,
// then the gathers), so every memory latency is shared by two rows.
template <typename V, typename X, typename IO, int G>
__device__ __forceinline__ void level_rows(const ApplyArgs<V, X, IO>& a, int kind, int p0, int p1) {
  using W = typename ValueReg<V, X>::type;
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
    X ra_rhs = zero<X>(), rb_rhs = zero<X>();
    int ppa = -1, ppb = -1, pma = 0, pmb = 0;
    if (pa >= 0) {
      qa = __ldg(ptr + pa) + lane;
      ea = __ldg(ptr + pa + 1);
      if (lane == 0) {
        if (kind == PH_FWD) ra_rhs = ldx(a.w + pa);
        else { ppa = __ldg(a.partner + pa); pma = __ldg(a.perm + pa); }
      }
    }
    if (pb >= 0) {
      qb = __ldg(ptr + pb) + lane;
      eb = __ldg(ptr + pb + 1);
      if (lane == 0) {
        if (kind == PH_FWD) rb_rhs = ldx(a.w + pb);
        else { ppb = __ldg(a.partner + pb); pmb = __ldg(a.perm + pb); }
      }
    }
    // two partial sums per row halve the dependent chain of FMAs
    X acca = zero<X>(), accb = zero<X>(), acca2 = zero<X>(), accb2 = zero<X>();
    while (qa < ea || qb < eb) {
      // lanes past the end of a row gather nothing: the solution entry they
      // would point at may not be written yet in this sweep (0 * NaN = NaN)
      int ca[B], cb[B];
      W va[B], vb[B];
#pragma unroll
      for (int i = 0; i < B; ++i) {
        const int q1 = qa + i * G, q2 = qb + i * G;
        const bool o1 = q1 < ea, o2 = q2 < eb;
        ca[i] = o1 ? __ldg(col + q1) : -1;
        va[i] = o1 ? ldw<W>(val + q1) : W(0);
        cb[i] = o2 ? __ldg(col + q2) : -1;
        vb[i] = o2 ? ldw<W>(val + q2) : W(0);
      }
#pragma unroll
      for (int i = 0; i < B; i += 2) {
        const X xa0 = ca[i] >= 0 ? ldx(x + ca[i]) : zero<X>();
        const X xb0 = cb[i] >= 0 ? ldx(x + cb[i]) : zero<X>();
        const X xa1 = ca[i + 1] >= 0 ? ldx(x + ca[i + 1]) : zero<X>();
        const X xb1 = cb[i + 1] >= 0 ? ldx(x + cb[i + 1]) : zero<X>();
        mac(acca, va[i], xa0);
        mac(accb, vb[i], xb0);
        mac(acca2, va[i + 1], xa1);
        mac(accb2, vb[i + 1], xb1);
      }
      qa += B * G;
      qb += B * G;
    }
    acca = add(norm(acca), norm(acca2));
    accb = add(norm(accb), norm(accb2));
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
  using VR = typename ValueReg<V, X>::type;
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
    X acc = zero<X>(), acc2 = zero<X>(), rhs = zero<X>();
    int pp = -1, pm = 0;
    if (p >= 0 && t == 0) {
      if (kind == PH_FWD) rhs = ldx(a.w + p);
      else { pp = __ldg(a.partner + p); pm = __ldg(a.perm + p); }
    }
    if (p >= 0) {
      int q = __ldg(ptr + p) + t;
      const int e = __ldg(ptr + p + 1);
      for (; q < e; q += B * G) {
        int c[B];
        VR v[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
          const bool o = q + i * G < e;
          c[i] = o ? __ldg(col + q + i * G) : -1;
          v[i] = o ? ldw<VR>(val + q + i * G) : VR(0);
        }
#pragma unroll
        for (int i = 0; i < B; i += 2) {
          const X x0 = c[i] >= 0 ? ldx(x + c[i]) : zero<X>();
          const X x1 = c[i + 1] >= 0 ? ldx(x + c[i + 1]) : zero<X>();
          mac(acc, v[i], x0);
          mac(acc2, v[i + 1], x1);
        }
      }
    }
    acc = add(norm(acc), norm(acc2));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = add(acc, shfl_xor(acc, o, 32));
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (p >= 0 && t == 0) {
      X sum = zero<X>();
#pragma unroll
      for (int j = 0; j < W; ++j) sum = add(sum, part[slot * W + j]);
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
    using W = typename ValueReg<V, X>::type;
    if (kind == PH_GATHER) {
      for (int p = p0 + blockIdx.x * blockDim.x + threadIdx.x; p < p1; p += gridDim.x * blockDim.x)
        stx(a.w + p, mul(ldw<W>(a.scale + p), from_io<X>(__ldg(a.b + __ldg(a.perm + p)))));
    } else if (kind == PH_DENSE) {
      const int lane = threadIdx.x & 31;
      const int warps = (gridDim.x * blockDim.x) >> 5;
      for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < a.nd; r += warps) {
        const V* row = a.dense + (int64_t)r * a.nd;
        X acc = zero<X>(), acc2 = zero<X>();
        for (int c0 = lane; c0 < a.nd; c0 += 8 * 32) {
          W rv[8];
          X wv[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int c = c0 + 32 * i;
            const bool ok = c < a.nd;
            rv[i] = ok ? ldw<W>(row + c) : W(0);
            wv[i] = ok ? ldx(a.w + a.d0 + c) : zero<X>();
          }
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            mac(acc, rv[i], wv[i]);
            mac(acc2, rv[i + 1], wv[i + 1]);
          }
        }
        acc = add(norm(acc), norm(acc2));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = add(acc, shfl_xor(acc, o, 32));
        if (lane == 0) {
          stx(a.z + a.d0 + r, acc);
          a.out[__ldg(a.perm + a.d0 + r)] = to_io<IO>(mul(ldw<W>(a.scale + a.d0 + r), acc));
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
