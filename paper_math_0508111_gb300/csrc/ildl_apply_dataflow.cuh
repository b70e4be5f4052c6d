// The dataflow form of the preconditioner apply (device code only): the same
// x = K^{-1} b as ildl_apply_persistent_kernel, in one cooperative launch,
// but without any per-level synchronisation.
//
// The work vectors w (forward sweep) and z (backward sweep) are filled with
// a sentinel (every bit set) before the launch.  A row is computed as soon as
// the solution entries it reads exist: each gathered entry is read with a
// relaxed GPU-scope load and, while it still holds the sentinel, read again
// (the value is the message, so no fence or counter is involved); a finished
// row is written with one single-copy-atomic store.  The level schedule then
// only fixes the order in which warps take rows, not when they may start:
// rows of the next level whose inputs are complete run while the previous
// level is still finishing its other rows, and the level-to-level latency is
// one store-to-load round trip instead of a grid-wide completion count.
//
// Work units in one global sequence: level 0 (32 rows per unit), the forward
// levels, the dense tail (one row per unit), the backward levels in reverse
// order; a forward or backward unit is 32/G rows of one level with G lanes
// per row (G <= 32).  Every unit reads only entries written by units earlier
// in the sequence (the rows of a level are independent; forward rows read
// earlier levels, backward rows later levels and the forward values).  Warp
// i of the grid takes units i, i + W, i + 2W, ... (W warps in all, units
// spread over the SMs first), in increasing order.  All warps are resident
// (cooperative launch), so the warp that holds the earliest unfinished unit
// has every input it needs: the apply cannot deadlock.  The waits are
// bounded anyway: a load that still reads the sentinel after kSpinLimit
// polls records a timeout in `err` and its warp returns; the other warps
// see the flag within a few hundred polls and return too.
#pragma once
#include "ildl_apply_kernel.cuh"

namespace ajd {
namespace {

// One work-vector element as a word that a single load or store moves
// whole: binary32 and binary64 as themselves, float-float (hi, lo) as one
// 64-bit word with hi in the low half (its memory layout).
template <typename X>
struct FlowWord {
  using U = unsigned long long;
};
template <>
struct FlowWord<float> {
  using U = unsigned;
};

__device__ __forceinline__ unsigned ld_flow(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned long long ld_flow(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_flow(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_flow(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ float from_word(unsigned w, float*) { return __uint_as_float(w); }
__device__ __forceinline__ double from_word(unsigned long long w, double*) { return __longlong_as_double((long long)w); }
__device__ __forceinline__ df64 from_word(unsigned long long w, df64*) {
  return df64{__uint_as_float((unsigned)w), __uint_as_float((unsigned)(w >> 32))};
}
template <typename X>
__device__ __forceinline__ X word_value(typename FlowWord<X>::U w) {
  return from_word(w, (X*)nullptr);
}

// The word of a computed value; a value whose bits happen to equal the
// sentinel (a NaN with every payload bit set) is stored as the default NaN
// instead, so that it is never taken for "not yet written".
__device__ __forceinline__ unsigned value_word(float v) {
  const unsigned w = __float_as_uint(v);
  return w == ~0u ? 0x7fffffffu : w;
}
__device__ __forceinline__ unsigned long long value_word(double v) {
  const unsigned long long w = (unsigned long long)__double_as_longlong(v);
  return w == ~0ull ? 0x7fffffffffffffffull : w;
}
__device__ __forceinline__ unsigned long long value_word(df64 v) {
  const unsigned long long w = ((unsigned long long)__float_as_uint(v.lo) << 32) | __float_as_uint(v.hi);
  return w == ~0ull ? 0x7fffffff7fffffffull : w;
}

template <typename X>
__device__ __forceinline__ const typename FlowWord<X>::U* words(const X* p) {
  return reinterpret_cast<const typename FlowWord<X>::U*>(p);
}
template <typename X>
__device__ __forceinline__ void put(X* p, X v) {
  st_flow(reinterpret_cast<typename FlowWord<X>::U*>(p), value_word(v));
}

// Wait until the word at p is written (w holds its first read).  False after
// this lane's timeout or once another warp has recorded one.
template <typename U>
__device__ __forceinline__ bool settle(const U* p, U& w, int* err) {
  if (w != ~U(0)) return true;
  unsigned spins = 0;
  do {
    ++spins;
    if (spins > kSpinLimit) {
      atomicExch(err, 1);
      return false;
    }
    if ((spins & 255u) == 0 && *((volatile int*)err)) return false;
    if (spins > 4) __nanosleep(48);
    w = ld_flow(p);
  } while (w == ~U(0));
  return true;
}

// Wait until every gathered word of a batch is written.  While a warp waits
// for the level before to finish, one lane polls one address: the lane that
// holds the warp's pending entry of the most recent level (the largest
// column in a forward sweep, the smallest in a backward sweep, since
// positions are ordered level by level) reloads it until it is written;
// thousands of lanes each polling their own entries would crowd the few L2
// lines that the level being finished writes.  Once it is written the level
// is nearly done, and every lane reloads its pending entries together, round
// by round, until none is left.
template <int B, typename U>
__device__ __forceinline__ bool settle_batch(const U* xw, const int (&c)[B], U (&xv)[B], int* err, bool backward) {
  const int lane = threadIdx.x & 31;
  // key of a pending column: larger = written later (-1: none pending)
  int mine = -1;
#pragma unroll
  for (int i = 0; i < B; ++i)
    if (c[i] >= 0 && xv[i] == ~U(0)) mine = max(mine, backward ? 0x7fffffff - c[i] : c[i]);
  int top = mine;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) top = max(top, __shfl_xor_sync(0xffffffffu, top, o));
  if (top < 0) return true;
  unsigned spins = 0;
  const int leader = __ffs(__ballot_sync(0xffffffffu, mine == top)) - 1;
  int bad = 0;
  if (lane == leader) {
    const int col = backward ? 0x7fffffff - top : top;
    U w = ld_flow(xw + col);
    while (w == ~U(0)) {
      ++spins;
      if (spins > kSpinLimit) {
        atomicExch(err, 1);
        bad = 1;
        break;
      }
      if ((spins & 255u) == 0 && *((volatile int*)err)) {
        bad = 1;
        break;
      }
      if (spins > 2) __nanosleep(32);
      w = ld_flow(xw + col);
    }
  }
  if (__shfl_sync(0xffffffffu, bad, leader)) return false;
  spins = 0;
  for (;;) {
    bool pend = false;
#pragma unroll
    for (int i = 0; i < B; ++i)
      if (c[i] >= 0 && xv[i] == ~U(0)) {
        xv[i] = ld_flow(xw + c[i]);
        pend |= xv[i] == ~U(0);
      }
    if (!__any_sync(0xffffffffu, pend)) return true;
    ++spins;
    if (spins > kSpinLimit) {
      if (lane == 0) atomicExch(err, 1);
      return false;
    }
    if ((spins & 255u) == 0 && *((volatile int*)err)) return false;
    __nanosleep(32);
  }
}

// Rows of one level, G lanes per row, 32/G rows per unit: this warp's units
// k, k + kstep, ... below kend of the level, in order.  The next unit's row
// pointers and heads are loaded before the current unit's gathers, and its
// first batch of indices and values right after them, so a unit costs about
// one memory round trip beyond the waits for its inputs.  Returns false
// after a timeout (uniform over the warp).
template <typename V, typename X, typename IO, int G>
__device__ __forceinline__ bool flow_rows(const ApplyArgs<V, X, IO>& a, int kind, int p0, int p1, int k, int kstep,
                                          int kend, int* err) {
  using W = typename ValueReg<V, X>::type;
  using U = typename FlowWord<X>::U;
  constexpr int B = 8;  // entries per lane and batch
  constexpr int R = 32 / G;
  const int lane = threadIdx.x & 31, t = lane % G, grp = lane / G;
  const bool bwd = kind == PH_BWD;
  const int* ptr = bwd ? a.Uptr : a.Lptr;
  const int* col = bwd ? a.Ucol : a.Lcol;
  const V* val = bwd ? a.Uval : a.Lval;
  const U* xw = words(bwd ? a.z : a.w);  // vector read through the columns
  const U* ww = words(a.w);
  // row state: pointers, head, forward values (backward rows), one batch
  int p = -1, q = 0, e = 0;
  RowHead<V, X, IO> h{};
  U w0 = 0, w1 = 0;
  int c[B];
  W v[B];
  int np = -1, nq = 0, ne = 0;
  RowHead<V, X, IO> nh{};
  U nw0 = 0, nw1 = 0;
  auto start = [&](int kk, int& rp, int& rq, int& re, RowHead<V, X, IO>& rh, U& rw0, U& rw1) {
    const int r = p0 + kk * R + grp;
    rp = r < p1 ? r : -1;
    rq = re = 0;
    if (rp >= 0) {
      rq = __ldg(ptr + rp) + t;
      re = __ldg(ptr + rp + 1);
      if (t == 0) {
        rh = row_head(a, kind, rp);
        if (bwd) {
          rw0 = ld_flow(ww + rp);
          if (rh.pp >= 0) rw1 = ld_flow(ww + rh.pp);
        }
      }
    }
  };
  auto batch = [&]() {
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const bool o = q + i * G < e;
      c[i] = o ? __ldg(col + q + i * G) : -1;
      v[i] = o ? ldw<W>(val + q + i * G) : W(0);
    }
  };
  start(k, p, q, e, h, w0, w1);
  batch();
  for (;;) {
    const bool more = k + kstep < kend;
    if (more) start(k + kstep, np, nq, ne, nh, nw0, nw1);  // in flight during this unit
    X acc = zero<X>(), acc2 = zero<X>();
    bool first = true;
    while (__any_sync(0xffffffffu, q < e)) {  // uniform over the warp (lanes past their row gather nothing)
      if (!first) batch();
      first = false;
      U xv[B];
#pragma unroll
      for (int i = 0; i < B; ++i) xv[i] = c[i] >= 0 ? ld_flow(xw + c[i]) : U(0);  // all-zero word: 0
      if (!settle_batch<B>(xw, c, xv, err, bwd)) return false;
#pragma unroll
      for (int i = 0; i < B; i += 2) {
        mac(acc, v[i], word_value<X>(xv[i]));
        mac(acc2, v[i + 1], word_value<X>(xv[i + 1]));
      }
      q += B * G;
    }
    bool ok = true;
    if (bwd && p >= 0 && t == 0) {
      // rhs = (D^{-1} w)_p from the forward values of the row and its partner
      if (!settle(ww + p, w0, err) || (h.pp >= 0 && !settle(ww + h.pp, w1, err))) ok = false;
      X d = mul(h.dd, word_value<X>(w0));
      if (h.pp >= 0) d = add(d, mul(h.dof, word_value<X>(w1)));
      h.rhs = d;
    }
    if (__any_sync(0xffffffffu, !ok)) return false;
    acc = add(norm(acc), norm(acc2));
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc = add(acc, shfl_xor(acc, o, G));
    if (p >= 0 && t == 0) {
      const X r = sub(h.rhs, acc);
      if (bwd) {
        put(a.z + p, r);
        a.out[h.perm] = to_io<IO>(mul(h.sc, r));
      } else {
        put(a.w + p, r);
      }
    }
    if (!more) return true;
    k += kstep;
    p = np;
    q = nq;
    e = ne;
    h = nh;
    w0 = nw0;
    w1 = nw1;
    batch();
  }
}

// Row r of the dense trailing block: z_d[r] = (D_d^{-1} w_d)[r], one warp.
template <typename V, typename X, typename IO>
__device__ __forceinline__ bool flow_dense_row(const ApplyArgs<V, X, IO>& a, int r, int* err) {
  using W = typename ValueReg<V, X>::type;
  using U = typename FlowWord<X>::U;
  constexpr int B = 16;
  const int lane = threadIdx.x & 31;
  const V* row = a.dense + (int64_t)r * a.nd;
  const U* wd = words(a.w + a.d0);
  X acc = zero<X>(), acc2 = zero<X>();
  for (int base = 0; base < a.nd; base += 32 * B) {  // uniform over the warp
    int c[B];
    W v[B];
    U xv[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const int col = base + lane + 32 * i;
      c[i] = col < a.nd ? col : -1;
      v[i] = col < a.nd ? ldw<W>(row + col) : W(0);
      xv[i] = col < a.nd ? ld_flow(wd + col) : U(0);
    }
    if (!settle_batch<B>(wd, c, xv, err, false)) return false;
#pragma unroll
    for (int i = 0; i < B; i += 2) {
      mac(acc, v[i], word_value<X>(xv[i]));
      mac(acc2, v[i + 1], word_value<X>(xv[i + 1]));
    }
  }
  acc = add(norm(acc), norm(acc2));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc = add(acc, shfl_xor(acc, o, 32));
  if (lane == 0) {
    put(a.z + a.d0 + r, acc);
    a.out[__ldg(a.perm + a.d0 + r)] = to_io<IO>(mul(ldw<W>(a.scale + a.d0 + r), acc));
  }
  return true;
}

template <typename V, typename X, typename IO>
__global__ void __launch_bounds__(kPersistThreads, 1)
ildl_apply_dataflow_kernel(ApplyArgs<V, X, IO> a, const int4* __restrict__ units, int nseg, int nunits, int* err,
                           unsigned long long* stamps) {
  using W = typename ValueReg<V, X>::type;
  const int lane = threadIdx.x & 31;
  if (stamps && blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    stamps[0] = t;  // start (CTA 0)
  }
  const int warps = (int)(gridDim.x * (blockDim.x >> 5));
  int sg = 0;
  for (int u = (int)((threadIdx.x >> 5) * gridDim.x + blockIdx.x); u < nunits; u += warps) {
    while (sg + 1 < nseg && __ldg(&units[sg + 1].w) <= u) ++sg;
    const int4 S = __ldg(units + sg);
    const int kind = S.x & 0xFF, G = S.x >> 8, k = u - S.w;
    const int kend = (sg + 1 < nseg ? __ldg(&units[sg + 1].w) : nunits) - S.w;  // units of the segment
    bool ok = true;
    if (kind == PH_GATHER) {
      // level 0: rows without entries, w = s b[perm]
      const int p = S.y + 32 * k + lane;
      if (p < S.z) put(a.w + p, mul(ldw<W>(a.scale + p), from_io<X>(__ldg(a.b + __ldg(a.perm + p)))));
    } else if (kind == PH_DENSE) {
      ok = flow_dense_row(a, k, err);
    } else {
      // all of this warp's units of the level at once (k, k + warps, ...)
      switch (G) {  // lanes per row, fixed per level at upload
        case 1: ok = flow_rows<V, X, IO, 1>(a, kind, S.y, S.z, k, warps, kend, err); break;
        case 2: ok = flow_rows<V, X, IO, 2>(a, kind, S.y, S.z, k, warps, kend, err); break;
        case 4: ok = flow_rows<V, X, IO, 4>(a, kind, S.y, S.z, k, warps, kend, err); break;
        case 8: ok = flow_rows<V, X, IO, 8>(a, kind, S.y, S.z, k, warps, kend, err); break;
        case 16: ok = flow_rows<V, X, IO, 16>(a, kind, S.y, S.z, k, warps, kend, err); break;
        default: ok = flow_rows<V, X, IO, 32>(a, kind, S.y, S.z, k, warps, kend, err); break;
      }
      u += (kend - 1 - k) / warps * warps;  // the last of those units
    }
    if (!ok) return;  // a wait timed out (uniform over the warp)
    if (stamps && lane == 0) {
      // diagnostics: when the segment's last unit finished
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      atomicMax(stamps + 1 + sg, t);
    }
  }
}

}  // namespace
}  // namespace ajd
