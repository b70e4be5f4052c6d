// The persistent preconditioner apply kernel (device code only): all of
// x = K^{-1} b in one cooperative launch.  Included by ildl.cu; kept in its
// own file so that measurements of this kernel can be tied to its source
// (bench.py keys recorded DRAM counters to this file's hash).
//
// Synchronisation-free level scheduling.  The positions are ordered level by
// level; a row of the forward sweep reads only solution entries of earlier
// levels, a row of the backward sweep only entries of later levels.  Instead
// of a grid-wide barrier between levels, every solution entry of w (forward)
// and z (backward) starts as a sentinel bit pattern (all ones: a NaN no
// arithmetic produces), written by the host before the launch, and each
// row's final value is published with one single-copy-atomic relaxed store.
// A row that needs an entry loads it with a relaxed (L2-coherent) load and
// polls while it still reads the sentinel.  So a row waits only for the rows
// it actually depends on, the index and value loads of a level are issued
// before its dependencies are ready, and consecutive levels overlap.  Every
// thread walks the levels in order and all CTAs are resident (cooperative
// launch, one CTA per SM), so every wait ends: the rows of level 0 depend on
// nothing, and a row of level l waits only on rows of levels < l, whose
// threads never wait on level l.  The waits are bounded anyway: after
// kSpinLimit polls a thread records a timeout in `err`, stops waiting and
// the apply returns garbage that the host reports as JD_EDEVICE.
#pragma once
#include "ildl_impl.cuh"

namespace ajd {
namespace {

// Phase kinds: level 0 (no dependencies), forward level, dense trailing
// block, backward level.  Threads walk the phase list in order.
enum { PH_GATHER = 0, PH_FWD = 1, PH_DENSE = 2, PH_BWD = 3 };
constexpr int kPersistThreads = 512;
constexpr unsigned kSpinLimit = 1u << 20;  // polls per thread and apply (~0.5-1 s)

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
// zero, acc += v * x (mac), a + b, a - b, v * x, shuffles, conversions from
// and to the caller's type.  The float-float forms use the error-free
// transformations of Dekker and Knuth (TwoSum, FMA-based TwoProduct): the
// product v * x.hi is split into its rounded value and exact error, and
// every addition carries its rounding error into lo.
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

// ---- publication and polling of solution entries ----
// Bits of one work-vector entry (8 bytes for binary64 and float-float,
// 4 for binary32); the sentinel is all ones.  Stores and loads are relaxed
// at GPU scope and of the entry's full width, so a reader sees either the
// sentinel or the final value, never a mix, and never a stale L1 copy.
template <typename X>
struct Bits {
  using type = unsigned long long;
};
template <>
struct Bits<float> {
  using type = unsigned;
};

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename X>
__device__ __forceinline__ typename Bits<X>::type to_bits(X v) {
  typename Bits<X>::type b;
  memcpy(&b, &v, sizeof(b));
  return b;
}
template <typename X>
__device__ __forceinline__ X from_bits(typename Bits<X>::type b) {
  X v;
  memcpy(&v, &b, sizeof(b));
  return v;
}
template <typename B>
__device__ __forceinline__ bool is_sentinel(B b) {
  return b == ~B(0);
}

// Per-thread wait state: polls spent so far in this apply, and whether a
// wait has given up (then no further wait is attempted).
struct Waiter {
  unsigned spins;
  bool dead;
  int* err;
};

// Poll entry p until it holds a published value (bounded).
template <typename X>
__device__ __noinline__ typename Bits<X>::type wait_bits(const X* p, Waiter& wt) {
  using B = typename Bits<X>::type;
  const B* q = reinterpret_cast<const B*>(p);
  B b = ld_relaxed(q);
  while (is_sentinel(b) && !wt.dead) {
    ++wt.spins;
    if ((wt.spins & 255u) == 0 && *((volatile int*)wt.err)) {
      wt.dead = true;
      break;
    }
    if (wt.spins > kSpinLimit) {
      atomicExch(wt.err, 1);
      wt.dead = true;
      break;
    }
    __nanosleep(20);
    b = ld_relaxed(q);
  }
  return is_sentinel(b) ? B(0) : b;
}

// Load entry p of a work vector: one relaxed load, polling only while the
// entry is not yet published.
template <typename X>
__device__ __forceinline__ X take(const X* p, Waiter& wt) {
  using B = typename Bits<X>::type;
  B b = ld_relaxed(reinterpret_cast<const B*>(p));
  if (is_sentinel(b)) b = wait_bits(p, wt);
  return from_bits<X>(b);
}

// Gathers of N entries x[c[i]] (c[i] < 0: none, value 0): all N loads are
// issued before the first is inspected, so their latencies overlap; only
// entries still unpublished are then polled.
template <typename X, int N>
__device__ __forceinline__ void gather(const X* x, const int (&c)[N], X (&out)[N], Waiter& wt) {
  using B = typename Bits<X>::type;
  B r[N];
#pragma unroll
  for (int i = 0; i < N; ++i) r[i] = c[i] >= 0 ? ld_relaxed(reinterpret_cast<const B*>(x + c[i])) : B(0);
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (is_sentinel(r[i])) r[i] = wait_bits(x + c[i], wt);
#pragma unroll
  for (int i = 0; i < N; ++i) out[i] = from_bits<X>(r[i]);
}

template <typename X>
__device__ __forceinline__ void publish(X* p, X v) {
  using B = typename Bits<X>::type;
  st_relaxed(reinterpret_cast<B*>(p), to_bits(v));
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
  X* w;  // forward solution, sentinel-filled before the launch
  X* z;  // backward solution, sentinel-filled before the launch
  const IO* b;
  IO* out;
  int nd, d0;
};

// Row operands loaded before the row's entries (their latency overlaps the
// gathers): forward -- the right-hand side s[p] b[perm[p]]; backward -- the
// 2x2 partner and the permutation entry.
template <typename V, typename X, typename IO>
struct RowHead {
  X rhs;
  int pp, perm;
};

template <typename V, typename X, typename IO>
__device__ __forceinline__ RowHead<V, X, IO> row_head(const ApplyArgs<V, X, IO>& a, int kind, int p) {
  using W = typename ValueReg<V, X>::type;
  RowHead<V, X, IO> h{zero<X>(), -1, 0};
  h.perm = __ldg(a.perm + p);
  if (kind == PH_FWD) h.rhs = mul(ldw<W>(a.scale + p), from_io<X>(__ldg(a.b + h.perm)));
  else h.pp = __ldg(a.partner + p);
  return h;
}

// Final value of row p of a sweep, given the row's dot product `acc` with
// the solution entries it depends on.
template <typename V, typename X, typename IO>
__device__ __forceinline__ void finish_value(const ApplyArgs<V, X, IO>& a, int kind, int p, X acc,
                                             const RowHead<V, X, IO>& h, Waiter& wt) {
  using W = typename ValueReg<V, X>::type;
  if (kind == PH_FWD) {
    publish(a.w + p, sub(h.rhs, acc));
  } else {
    X d = mul(ldw<W>(a.dd + p), take(a.w + p, wt));
    if (h.pp >= 0) d = add(d, mul(ldw<W>(a.dof + p), take(a.w + h.pp, wt)));
    const X zp = sub(d, acc);
    publish(a.z + p, zp);
    a.out[h.perm] = to_io<IO>(mul(ldw<W>(a.scale + p), zp));
  }
}

template <typename V, typename X, typename IO, int G>
__device__ __forceinline__ void finish_row(const ApplyArgs<V, X, IO>& a, int kind, int p, X acc, int lane,
                                           const RowHead<V, X, IO>& h, Waiter& wt) {
  acc = norm(acc);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc = add(acc, shfl_xor(acc, o, G));
  if (p >= 0 && lane == 0) finish_value(a, kind, p, acc, h, wt);
}

// Rows of one level, G threads per row; each group handles two rows at a
// time with their loads interleaved (index/value loads of both rows first,
// then the gathers), so every memory latency is shared by two rows.
template <typename V, typename X, typename IO, int G>
__device__ __forceinline__ void level_rows(const ApplyArgs<V, X, IO>& a, int kind, int p0, int p1, int cta,
                                           Waiter& wt) {
  using W = typename ValueReg<V, X>::type;
  const int lane = threadIdx.x % G;
  const int64_t groups = (int64_t)gridDim.x * blockDim.x / G;
  const int64_t g0 = ((int64_t)cta * blockDim.x + threadIdx.x) / G;
  const int* ptr = kind == PH_FWD ? a.Lptr : a.Uptr;
  const int* col = kind == PH_FWD ? a.Lcol : a.Ucol;
  const V* val = kind == PH_FWD ? a.Lval : a.Uval;
  const X* x = kind == PH_FWD ? a.w : a.z;  // vector read through the columns
  // entries per lane and row per batch (fewer with binary64 values, which
  // take twice the registers)
  constexpr int B = sizeof(V) == 8 ? 4 : 8;
  for (int64_t base = p0; base < p1; base += 2 * groups) {
    const int64_t ra = base + g0, rb = base + groups + g0;
    const int pa = ra < p1 ? (int)ra : -1;
    const int pb = rb < p1 ? (int)rb : -1;
    int qa = 0, ea = 0, qb = 0, eb = 0;
    RowHead<V, X, IO> ha{zero<X>(), -1, 0}, hb{zero<X>(), -1, 0};
    if (pa >= 0) {
      qa = __ldg(ptr + pa) + lane;
      ea = __ldg(ptr + pa + 1);
      if (lane == 0) ha = row_head(a, kind, pa);
    }
    if (pb >= 0) {
      qb = __ldg(ptr + pb) + lane;
      eb = __ldg(ptr + pb + 1);
      if (lane == 0) hb = row_head(a, kind, pb);
    }
    // two partial sums per row halve the dependent chain of FMAs
    X acca = zero<X>(), accb = zero<X>(), acca2 = zero<X>(), accb2 = zero<X>();
    while (qa < ea || qb < eb) {
      // lanes past the end of a row gather nothing
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
      // both rows' gathers in flight at once
      int cab[2 * B];
      X xab[2 * B];
#pragma unroll
      for (int i = 0; i < B; ++i) {
        cab[i] = ca[i];
        cab[B + i] = cb[i];
      }
      gather(x, cab, xab, wt);
#pragma unroll
      for (int i = 0; i < B; i += 2) {
        mac(acca, va[i], xab[i]);
        mac(accb, vb[i], xab[B + i]);
        mac(acca2, va[i + 1], xab[i + 1]);
        mac(accb2, vb[i + 1], xab[B + i + 1]);
      }
      qa += B * G;
      qb += B * G;
    }
    acca = add(norm(acca), norm(acca2));
    accb = add(norm(accb), norm(accb2));
    finish_row<V, X, IO, G>(a, kind, pa, acca, lane, ha, wt);
    finish_row<V, X, IO, G>(a, kind, pb, accb, lane, hb, wt);
  }
}

// Rows of one level with G = 64..512 threads per row (G / 32 warps, 512 / G
// rows per CTA): for few, long rows, such as the deepest levels, whose rows
// collect the fill of every earlier level.  Warp partial sums meet in
// shared memory.  The row loop is uniform across the CTA (it depends on the
// block index only), as the CTA barriers inside it require.
template <typename V, typename X, typename IO, int G>
__device__ __forceinline__ void level_rows_wide(const ApplyArgs<V, X, IO>& a, int kind, int p0, int p1, int cta,
                                                Waiter& wt) {
  using VR = typename ValueReg<V, X>::type;
  constexpr int NW = G / 32;                // warps per row
  constexpr int RPC = kPersistThreads / G;  // rows per CTA and pass
  constexpr int B = 8;                      // entries per thread and batch
  __shared__ X part[kPersistThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = threadIdx.x / G, t = threadIdx.x % G;
  const int* ptr = kind == PH_FWD ? a.Lptr : a.Uptr;
  const int* col = kind == PH_FWD ? a.Lcol : a.Ucol;
  const V* val = kind == PH_FWD ? a.Lval : a.Uval;
  const X* x = kind == PH_FWD ? a.w : a.z;
  for (int64_t base = p0 + (int64_t)cta * RPC; base < p1; base += (int64_t)gridDim.x * RPC) {
    const int p = base + slot < p1 ? (int)(base + slot) : -1;
    X acc = zero<X>(), acc2 = zero<X>();
    RowHead<V, X, IO> h{zero<X>(), -1, 0};
    if (p >= 0 && t == 0) h = row_head(a, kind, p);
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
        X xv[B];
        gather(x, c, xv, wt);
#pragma unroll
        for (int i = 0; i < B; i += 2) {
          mac(acc, v[i], xv[i]);
          mac(acc2, v[i + 1], xv[i + 1]);
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
      for (int j = 0; j < NW; ++j) sum = add(sum, part[slot * NW + j]);
      finish_value(a, kind, p, sum, h, wt);
    }
    __syncthreads();  // part[] is reused by the next pass
  }
}

template <typename V, typename X, typename IO>
__global__ void __launch_bounds__(kPersistThreads, 1)
ildl_apply_persistent_kernel(ApplyArgs<V, X, IO> a, const int4* __restrict__ phases, int nphase, int* err,
                             unsigned long long* stamps) {
  using W = typename ValueReg<V, X>::type;
  Waiter wt{0u, false, err};
  if (stamps && blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    stamps[0] = t;  // start (CTA 0)
  }
  for (int ph = 0; ph < nphase; ++ph) {
    const int4 P = phases[ph];  // kind, p0, p1, G | first CTA << 16
    const int kind = P.x, p0 = P.y, p1 = P.z, G = P.w & 0xFFFF;
    // the phase's rows start at CTA P.w >> 16: consecutive small phases land
    // on different CTAs, whose loads are then issued while the previous
    // level is still being computed (not after it, as on one CTA)
    const int cta = (int)((blockIdx.x + gridDim.x - (unsigned)(P.w >> 16) % gridDim.x) % gridDim.x);
    if (kind == PH_GATHER) {
      // level 0: rows without entries, w = s b[perm]
      for (int p = p0 + blockIdx.x * blockDim.x + threadIdx.x; p < p1; p += gridDim.x * blockDim.x)
        publish(a.w + p, mul(ldw<W>(a.scale + p), from_io<X>(__ldg(a.b + __ldg(a.perm + p)))));
    } else if (kind == PH_DENSE) {
      const int lane = threadIdx.x & 31;
      const int warps = (gridDim.x * blockDim.x) >> 5;
      for (int r = (cta * blockDim.x + threadIdx.x) >> 5; r < a.nd; r += warps) {
        const V* row = a.dense + (int64_t)r * a.nd;
        X acc = zero<X>(), acc2 = zero<X>();
        for (int c0 = lane; c0 < a.nd; c0 += 8 * 32) {
          W rv[8];
          X wv[8];
          int cc[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int c = c0 + 32 * i;
            rv[i] = c < a.nd ? ldw<W>(row + c) : W(0);
            cc[i] = c < a.nd ? c : -1;
          }
          gather(a.w + a.d0, cc, wv, wt);
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
          publish(a.z + a.d0 + r, acc);
          a.out[__ldg(a.perm + a.d0 + r)] = to_io<IO>(mul(ldw<W>(a.scale + a.d0 + r), acc));
        }
      }
    } else {
      switch (G) {  // threads per row, fixed per phase at upload
        case 4: level_rows<V, X, IO, 4>(a, kind, p0, p1, cta, wt); break;
        case 8: level_rows<V, X, IO, 8>(a, kind, p0, p1, cta, wt); break;
        case 16: level_rows<V, X, IO, 16>(a, kind, p0, p1, cta, wt); break;
        case 32: level_rows<V, X, IO, 32>(a, kind, p0, p1, cta, wt); break;
        case 64: level_rows_wide<V, X, IO, 64>(a, kind, p0, p1, cta, wt); break;
        case 128: level_rows_wide<V, X, IO, 128>(a, kind, p0, p1, cta, wt); break;
        case 256: level_rows_wide<V, X, IO, 256>(a, kind, p0, p1, cta, wt); break;
        default: level_rows_wide<V, X, IO, 512>(a, kind, p0, p1, cta, wt); break;
      }
    }
    if (stamps && cta == 0 && threadIdx.x == 0) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      stamps[ph + 1] = t;  // when the phase's first CTA is done with it (phases overlap)
    }
  }

}

}  // namespace
}  // namespace ajd
