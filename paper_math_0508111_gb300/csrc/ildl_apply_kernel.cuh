// The persistent preconditioner apply kernel (device code only): all of
// x = K^{-1} b in one cooperative launch.  Included by ildl.cu; kept in its
// own file so that measurements of this kernel can be tied to its source
// (bench.py keys recorded DRAM counters to this file's hash).
//
// Level scheduling with per-phase completion counters.  The positions are
// ordered level by level; a row of the forward sweep reads only solution
// entries of earlier levels, a row of the backward sweep only entries of
// later levels (and its own forward value).  The phase list (level 0, the
// forward levels, the dense tail, the backward levels) is walked in order by
// every CTA, but only the CTAs that own rows of a phase take part in it:
// each of them, once its rows are written, adds one to the phase's counter
// (release), and a CTA about to compute a phase first waits (one thread,
// acquire polls) until every earlier phase's counter has reached its number
// of participants.  The loads of the phase's row pointers, indices and
// values are issued before that wait, so they are in flight while the
// previous level is still being computed; only the gathers of solution
// entries follow it.  Consecutive phases start on different CTAs (the
// first CTA of each phase rotates round the grid), so the CTAs of a small
// phase are idle, with their loads issued, when the level before completes.
// All CTAs are resident (cooperative launch, one CTA per SM) and a phase
// waits only on earlier phases, so every wait ends; the waits are bounded
// anyway: after kSpinLimit polls the thread records a timeout in `err` and
// its CTA returns (the host reports JD_EDEVICE).
#pragma once
#include "ildl_impl.cuh"

namespace ajd {
namespace {

// Phase kinds: level 0 (no dependencies), forward level, dense trailing
// block, backward level.  A phase descriptor is the int4
// (kind | participating CTAs << 8, first row, end row, threads per row |
// first CTA << 16).
enum { PH_GATHER = 0, PH_FWD = 1, PH_DENSE = 2, PH_BWD = 3 };
constexpr int kPersistThreads = 512;
constexpr unsigned kSpinLimit = 1u << 22;  // polls of one wait (~0.2-1 s)

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
  X* w;  // forward solution
  X* z;  // backward solution
  const IO* b;
  IO* out;
  int nd, d0;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Completion bookkeeping of one CTA: counters of the phases, the number of
// phases this CTA knows to be complete (all phases < known), the timeout
// flag.  wait() is called by every thread of the CTA at the same point.
struct Progress {
  const int4* phases;
  unsigned* done;
  int* err;
  int* known;   // shared
  int* failed;  // shared

  // every phase < ph complete; false after a timeout
  __device__ __forceinline__ bool wait(int ph) {
    if (threadIdx.x == 0) {
      int r = *known;
      while (r < ph && !*failed) {
        const unsigned need = (unsigned)(phases[r].x >> 8);
        unsigned spins = 0;
        while (ld_acquire_u32(done + r) < need) {
          ++spins;
          if ((spins & 1023u) == 0 && *((volatile int*)err)) { *failed = 1; break; }
          if (spins > kSpinLimit) {
            atomicExch(err, 1);
            *failed = 1;
            break;
          }
          if (spins > 32) __nanosleep(32);
        }
        ++r;
      }
      *known = r;
    }
    __syncthreads();
    return *failed == 0;
  }

  // this CTA's rows of phase ph are written
  __device__ __forceinline__ void arrive(int ph) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(done + ph) : "memory");
    }
  }
};

// Row operands that do not depend on other rows, loaded before the row's
// entries (and, for a phase's first rows, before the wait): the permutation
// entry; forward -- the right-hand side s[p] b[perm[p]]; backward -- the
// 2x2 partner, the row's entries of D^{-1} and its scale.  Backward rows
// also need D^{-1} w, formed after the wait (bwd_rhs) while the entries'
// gathers are in flight.
template <typename V, typename X, typename IO>
struct RowHead {
  using W = typename ValueReg<V, X>::type;
  X rhs;
  int pp, perm;
  W dd, dof, sc;
};

template <typename V, typename X, typename IO>
__device__ __forceinline__ RowHead<V, X, IO> row_head(const ApplyArgs<V, X, IO>& a, int kind, int p) {
  using W = typename ValueReg<V, X>::type;
  RowHead<V, X, IO> h{zero<X>(), -1, 0, W(0), W(0), W(0)};
  h.perm = __ldg(a.perm + p);
  if (kind == PH_FWD) {
    h.rhs = mul(ldw<W>(a.scale + p), from_io<X>(__ldg(a.b + h.perm)));
  } else {
    h.pp = __ldg(a.partner + p);
    h.dd = ldw<W>(a.dd + p);
    h.dof = ldw<W>(a.dof + p);
    h.sc = ldw<W>(a.scale + p);
  }
  return h;
}

// backward row p: rhs = (D^{-1} w)_p, from the forward sweep's values
template <typename V, typename X, typename IO>
__device__ __forceinline__ void bwd_rhs(const ApplyArgs<V, X, IO>& a, int p, RowHead<V, X, IO>& h) {
  X d = mul(h.dd, ldx(a.w + p));
  if (h.pp >= 0) d = add(d, mul(h.dof, ldx(a.w + h.pp)));
  h.rhs = d;
}

// Final value of row p of a sweep, given the row's dot product `acc` with
// the solution entries it depends on.
template <typename V, typename X, typename IO>
__device__ __forceinline__ void finish_value(const ApplyArgs<V, X, IO>& a, int kind, int p, X acc,
                                             const RowHead<V, X, IO>& h) {
  const X v = sub(h.rhs, acc);
  if (kind == PH_FWD) {
    stx(a.w + p, v);
  } else {
    stx(a.z + p, v);
    a.out[h.perm] = to_io<IO>(mul(h.sc, v));
  }
}

template <typename V, typename X, typename IO, int G>
__device__ __forceinline__ void finish_row(const ApplyArgs<V, X, IO>& a, int kind, int p, X acc, int lane,
                                           const RowHead<V, X, IO>& h) {
  acc = norm(acc);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc = add(acc, shfl_xor(acc, o, G));
  if (p >= 0 && lane == 0) finish_value(a, kind, p, acc, h);
}

// Rows of one level, G threads per row; each group handles two rows at a
// time with their loads interleaved (index/value loads of both rows first,
// then the gathers), so every memory latency is shared by two rows.  The
// first row pair's pointers, heads and first batch of entries are loaded
// before the wait for the earlier phases; while a pair's entries are
// gathered, the next pair's pointers and heads are already being loaded.
template <typename V, typename X, typename IO, int G>
__device__ __forceinline__ bool level_rows(const ApplyArgs<V, X, IO>& a, int kind, int p0, int p1, int cta,
                                           Progress& pg, int ph) {
  using W = typename ValueReg<V, X>::type;
  // entries per lane and row per batch (fewer with binary64 values or
  // float-float work vectors, which take twice the registers)
  constexpr int B = sizeof(V) == 8 ? 4 : (sizeof(X) == 8 ? 6 : 8);
  const int lane = threadIdx.x % G;
  const int64_t groups = (int64_t)gridDim.x * blockDim.x / G;
  const int64_t g0 = ((int64_t)cta * blockDim.x + threadIdx.x) / G;
  const int* ptr = kind == PH_FWD ? a.Lptr : a.Uptr;
  const int* col = kind == PH_FWD ? a.Lcol : a.Ucol;
  const V* val = kind == PH_FWD ? a.Lval : a.Uval;
  const X* x = kind == PH_FWD ? a.w : a.z;  // vector read through the columns
  int64_t base = p0;
  int pa = -1, pb = -1, qa = 0, ea = 0, qb = 0, eb = 0;
  RowHead<V, X, IO> ha{}, hb{};
  int ca[B], cb[B];
  W va[B], vb[B];
  // lanes past the end of a row gather nothing
  auto load_batch = [&]() {
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const int q1 = qa + i * G, q2 = qb + i * G;
      const bool o1 = q1 < ea, o2 = q2 < eb;
      ca[i] = o1 ? __ldg(col + q1) : -1;
      va[i] = o1 ? ldw<W>(val + q1) : W(0);
      cb[i] = o2 ? __ldg(col + q2) : -1;
      vb[i] = o2 ? ldw<W>(val + q2) : W(0);
    }
  };
  // pointers and heads of the pair at `at` (rows beyond p1: -1)
  auto load_heads = [&](int64_t at, int& ra, int& rb, int& sa, int& ta, int& sb, int& tb, RowHead<V, X, IO>& h1,
                        RowHead<V, X, IO>& h2) {
    const int64_t r1 = at + g0, r2 = at + groups + g0;
    ra = r1 < p1 ? (int)r1 : -1;
    rb = r2 < p1 ? (int)r2 : -1;
    sa = ta = sb = tb = 0;
    if (ra >= 0) {
      sa = __ldg(ptr + ra) + lane;
      ta = __ldg(ptr + ra + 1);
      if (lane == 0) h1 = row_head(a, kind, ra);
    }
    if (rb >= 0) {
      sb = __ldg(ptr + rb) + lane;
      tb = __ldg(ptr + rb + 1);
      if (lane == 0) h2 = row_head(a, kind, rb);
    }
  };
  load_heads(base, pa, pb, qa, ea, qb, eb, ha, hb);
  load_batch();
  if (!pg.wait(ph)) return false;
  while (base < p1) {
    if (kind == PH_BWD && lane == 0) {
      if (pa >= 0) bwd_rhs(a, pa, ha);
      if (pb >= 0) bwd_rhs(a, pb, hb);
    }
    // the next pair's pointers and heads, in flight during this pair's work
    const int64_t nbase = base + 2 * groups;
    int npa = -1, npb = -1, nqa = 0, nea = 0, nqb = 0, neb = 0;
    RowHead<V, X, IO> nha{}, nhb{};
    if (nbase < p1) load_heads(nbase, npa, npb, nqa, nea, nqb, neb, nha, nhb);
    // two partial sums per row halve the dependent chain of FMAs
    X acca = zero<X>(), accb = zero<X>(), acca2 = zero<X>(), accb2 = zero<X>();
    while (qa < ea || qb < eb) {
      X xa[B], xb[B];
#pragma unroll
      for (int i = 0; i < B; ++i) {  // both rows' gathers in flight at once
        xa[i] = ca[i] >= 0 ? ldx(x + ca[i]) : zero<X>();
        xb[i] = cb[i] >= 0 ? ldx(x + cb[i]) : zero<X>();
      }
#pragma unroll
      for (int i = 0; i < B; i += 2) {
        mac(acca, va[i], xa[i]);
        mac(accb, vb[i], xb[i]);
        mac(acca2, va[i + 1], xa[i + 1]);
        mac(accb2, vb[i + 1], xb[i + 1]);
      }
      qa += B * G;
      qb += B * G;
      load_batch();
    }
    acca = add(norm(acca), norm(acca2));
    accb = add(norm(accb), norm(accb2));
    finish_row<V, X, IO, G>(a, kind, pa, acca, lane, ha);
    finish_row<V, X, IO, G>(a, kind, pb, accb, lane, hb);
    base = nbase;
    if (base < p1) {
      pa = npa;
      pb = npb;
      qa = nqa;
      ea = nea;
      qb = nqb;
      eb = neb;
      ha = nha;
      hb = nhb;
      load_batch();
    }
  }
  return true;
}

// Rows of one level with G = 64..512 threads per row (G / 32 warps, 512 / G
// rows per CTA): for few, long rows, such as the deepest levels, whose rows
// collect the fill of every earlier level.  Warp partial sums meet in
// shared memory.  The row loop is uniform across the CTA (it depends on the
// block index only), as the CTA barriers inside it require.  The first
// pass's row and first batch are loaded before the wait.
template <typename V, typename X, typename IO, int G>
__device__ __forceinline__ bool level_rows_wide(const ApplyArgs<V, X, IO>& a, int kind, int p0, int p1, int cta,
                                                Progress& pg, int ph) {
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
  int64_t base = p0 + (int64_t)cta * RPC;
  int p = -1, q = 0, e = 0;
  RowHead<V, X, IO> h{};
  int c[B];
  VR v[B];
  auto load_batch = [&]() {
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const bool o = q + i * G < e;
      c[i] = o ? __ldg(col + q + i * G) : -1;
      v[i] = o ? ldw<VR>(val + q + i * G) : VR(0);
    }
  };
  auto load_row = [&]() {
    p = base + slot < p1 ? (int)(base + slot) : -1;
    q = e = 0;
    if (p >= 0) {
      q = __ldg(ptr + p) + t;
      e = __ldg(ptr + p + 1);
      if (t == 0) h = row_head(a, kind, p);
    }
    load_batch();
  };
  load_row();
  if (!pg.wait(ph)) return false;
  for (; base < p1; base += (int64_t)gridDim.x * RPC) {
    if (kind == PH_BWD && p >= 0 && t == 0) bwd_rhs(a, p, h);
    X acc = zero<X>(), acc2 = zero<X>();
    while (q < e) {
      X xv[B];
#pragma unroll
      for (int i = 0; i < B; ++i) xv[i] = c[i] >= 0 ? ldx(x + c[i]) : zero<X>();
#pragma unroll
      for (int i = 0; i < B; i += 2) {
        mac(acc, v[i], xv[i]);
        mac(acc2, v[i + 1], xv[i + 1]);
      }
      q += B * G;
      load_batch();
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
      finish_value(a, kind, p, sum, h);
    }
    __syncthreads();  // part[] is reused by the next pass
    if (base + (int64_t)gridDim.x * RPC < p1) {
      base += (int64_t)gridDim.x * RPC;
      load_row();
      base -= (int64_t)gridDim.x * RPC;
    }
  }
  return true;
}

// The dense trailing block: z_d = D^{-1} w_d with its stored inverse, one
// warp per row; the first row's first chunk is loaded before the wait.
template <typename V, typename X, typename IO>
__device__ __forceinline__ bool dense_rows(const ApplyArgs<V, X, IO>& a, int cta, Progress& pg, int ph) {
  using W = typename ValueReg<V, X>::type;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  int r = (cta * blockDim.x + threadIdx.x) >> 5;
  W rv[8];
  auto load_chunk = [&](int c0) {
    const V* row = a.dense + (int64_t)r * a.nd;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = c0 + 32 * i;
      rv[i] = (r < a.nd && c < a.nd) ? ldw<W>(row + c) : W(0);
    }
  };
  load_chunk(lane);
  if (!pg.wait(ph)) return false;
  for (; r < a.nd; r += warps) {
    X acc = zero<X>(), acc2 = zero<X>();
    for (int c0 = lane; c0 < a.nd; c0 += 8 * 32) {
      X wv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int c = c0 + 32 * i;
        wv[i] = c < a.nd ? ldx(a.w + a.d0 + c) : zero<X>();
      }
#pragma unroll
      for (int i = 0; i < 8; i += 2) {
        mac(acc, rv[i], wv[i]);
        mac(acc2, rv[i + 1], wv[i + 1]);
      }
      if (c0 + 8 * 32 < a.nd) load_chunk(c0 + 8 * 32);
    }
    acc = add(norm(acc), norm(acc2));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = add(acc, shfl_xor(acc, o, 32));
    if (lane == 0) {
      stx(a.z + a.d0 + r, acc);
      a.out[__ldg(a.perm + a.d0 + r)] = to_io<IO>(mul(ldw<W>(a.scale + a.d0 + r), acc));
    }
    if (r + warps < a.nd) {
      r += warps;
      load_chunk(lane);
      r -= warps;
    }
  }
  return true;
}

template <typename V, typename X, typename IO>
__global__ void __launch_bounds__(kPersistThreads, 1)
ildl_apply_persistent_kernel(ApplyArgs<V, X, IO> a, const int4* __restrict__ phases, int nphase, unsigned* done,
                             int* err, unsigned long long* stamps) {
  using W = typename ValueReg<V, X>::type;
  __shared__ int s_known, s_failed;
  if (threadIdx.x == 0) {
    s_known = 0;
    s_failed = 0;
    if (stamps && blockIdx.x == 0) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      stamps[0] = t;  // start (CTA 0)
    }
  }
  __syncthreads();
  Progress pg{phases, done, err, &s_known, &s_failed};
  for (int ph = 0; ph < nphase; ++ph) {
    const int4 P = phases[ph];
    const int kind = P.x & 0xFF, parts = P.x >> 8, p0 = P.y, p1 = P.z, G = P.w & 0xFFFF;
    // rotated CTA index: the phase's rows start at CTA P.w >> 16
    const int cta = (int)((blockIdx.x + gridDim.x - (unsigned)(P.w >> 16) % gridDim.x) % gridDim.x);
    if (cta >= parts) continue;  // no rows of this phase here (uniform over the CTA)
    bool ok = true;
    if (kind == PH_GATHER) {
      // level 0: rows without entries, w = s b[perm]; nothing to wait for
      for (int p = p0 + cta * blockDim.x + threadIdx.x; p < p1; p += gridDim.x * blockDim.x)
        stx(a.w + p, mul(ldw<W>(a.scale + p), from_io<X>(__ldg(a.b + __ldg(a.perm + p)))));
    } else if (kind == PH_DENSE) {
      ok = dense_rows(a, cta, pg, ph);
    } else {
      switch (G) {  // threads per row, fixed per phase at upload
        case 1: ok = level_rows<V, X, IO, 1>(a, kind, p0, p1, cta, pg, ph); break;
        case 2: ok = level_rows<V, X, IO, 2>(a, kind, p0, p1, cta, pg, ph); break;
        case 4: ok = level_rows<V, X, IO, 4>(a, kind, p0, p1, cta, pg, ph); break;
        case 8: ok = level_rows<V, X, IO, 8>(a, kind, p0, p1, cta, pg, ph); break;
        case 16: ok = level_rows<V, X, IO, 16>(a, kind, p0, p1, cta, pg, ph); break;
        case 32: ok = level_rows<V, X, IO, 32>(a, kind, p0, p1, cta, pg, ph); break;
        case 64: ok = level_rows_wide<V, X, IO, 64>(a, kind, p0, p1, cta, pg, ph); break;
        case 128: ok = level_rows_wide<V, X, IO, 128>(a, kind, p0, p1, cta, pg, ph); break;
        case 256: ok = level_rows_wide<V, X, IO, 256>(a, kind, p0, p1, cta, pg, ph); break;
        default: ok = level_rows_wide<V, X, IO, 512>(a, kind, p0, p1, cta, pg, ph); break;
      }
    }
    if (!ok) return;  // a wait timed out (uniform over the CTA)
    pg.arrive(ph);
    if (stamps && cta == 0 && threadIdx.x == 0) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      stamps[ph + 1] = t;  // when the phase's first CTA is done with it (phases overlap)
    }
  }
}

}  // namespace
}  // namespace ajd
