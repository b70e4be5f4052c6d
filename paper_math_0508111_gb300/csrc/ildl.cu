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
#include <memory>
#include <mutex>
#include <new>
#include <cstdio>
#include <cstdlib>
#include <type_traits>

#include "anderson_impl.cuh"
#include "ildl_impl.cuh"
#include "jd_impl.cuh"
#include "ildl_setup.h"
#include "ildl_apply_kernel.cuh"
#include "ildl_apply_dataflow.cuh"
#include "schur_gpu.h"
#include "dense_inverse.h"

namespace ajd {
namespace {

// Apply form of factors that are not autotuned (ildl_params.apply_form < 0):
// 1 = the dataflow kernel, 0 = the level-counter kernel.
constexpr int kDefaultApplyForm = 1;

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
  cudaFree(d.w);  // z lies in the same allocation
  cudaFree(d.phases);
  cudaFree(d.units);
  cudaFree(d.bar);
  cudaFree(d.done);
  cudaFree(d.wdf);  // and zdf in wdf's
  d = DevFactor<T>();
}

template <typename S, typename D, class Alloc>
int upload(D** dst, const std::vector<S, Alloc>& src, cudaStream_t st) {
  *dst = nullptr;
  if (src.empty()) return JD_OK;
  const size_t n = src.size();
  cudaError_t e = cudaMalloc(dst, n * sizeof(D));
  if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? JD_ENOMEM : JD_EDEVICE, "ildl upload: %s", cudaGetErrorString(e));
  if constexpr (std::is_same<S, D>::value) {
    AJD_CUDA(cudaMemcpyAsync(*dst, src.data(), n * sizeof(D), cudaMemcpyHostToDevice, st));
    AJD_CUDA(cudaStreamSynchronize(st));
  } else {
    dvec<D> tmp(n);  // first touched by the parallel conversion
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) tmp[i] = D(src[i]);
    AJD_CUDA(cudaMemcpyAsync(*dst, tmp.data(), n * sizeof(D), cudaMemcpyHostToDevice, st));
    AJD_CUDA(cudaStreamSynchronize(st));  // tmp is released on return
  }
  return JD_OK;
}

// Phase list of the persistent apply for factor F.  Threads per row: enough
// rows in flight to cover the grid, and about four stored entries per thread
// of a row (a power of two in 1..512), times 2^shift (the autotuner's knob).
// Each phase's rows start at the CTA after the last one the previous phase
// used (round robin over the grid), so that the CTAs of a small phase are
// idle while the level before it is computed and have its loads in flight by
// then; the first CTA goes in the high half of .w, the number of CTAs that
// own rows (the phase's participants, which signal its completion) in the
// high bits of .x.  Level 0 (rows without entries) only forms w = s b[perm];
// later forward rows form their right-hand side s[p] b[perm[p]] themselves.
std::vector<int4> build_phase_list(const HostFactor& F, int shift) {
  std::vector<int4> ph;
  const std::vector<int>& lvp = F.level_ptr;
  const int nl = F.nlev;
  const double threads_total = (double)sm_count() * kPersistThreads;
  auto pick_g = [&](int rows, double avg) {
    const double want = std::max(std::min(threads_total / std::max(rows, 1), avg / 4.0), std::min(avg / 8.0, 32.0));
    int g = 1;
    while (g < 512 && 2 * g <= want) g *= 2;
    for (int i = 0; i < shift && g < 512; ++i) g *= 2;
    for (int i = 0; i > shift && g > 1; --i) g /= 2;
    return g;
  };
  const int grid = sm_count();
  int cursor = 0;
  auto add_phase = [&](int kind, int p0, int p1, int g) {
    const int64_t threads = (int64_t)(p1 - p0) * (kind == PH_DENSE ? 32 : g);
    const int ctas = (int)std::min<int64_t>(grid, (threads + kPersistThreads - 1) / kPersistThreads);
    ph.push_back(make_int4(kind | (ctas << 8), p0, p1, g | (cursor << 16)));
    cursor = (cursor + ctas) % grid;
  };
  add_phase(PH_GATHER, lvp[0], lvp[1], 1);
  for (int l = 1; l <= nl; ++l) {
    const int p0 = lvp[l], p1 = lvp[l + 1];
    if (p1 <= p0) continue;
    const double avg = (double)(F.Lptr[p1] - F.Lptr[p0]) / (p1 - p0);
    add_phase(PH_FWD, p0, p1, pick_g(p1 - p0, avg));
  }
  if (F.n_dense > 0) add_phase(PH_DENSE, lvp[nl], lvp[nl + 1], 32);
  for (int l = nl - 1; l >= 0; --l) {
    const int p0 = lvp[l], p1 = lvp[l + 1];
    if (p1 <= p0) continue;
    const double avg = (double)(F.Uptr[p1] - F.Uptr[p0]) / (p1 - p0);
    add_phase(PH_BWD, p0, p1, pick_g(p1 - p0, avg));
  }
  return ph;
}

// Unit segments of the dataflow apply for factor F, in the order the units
// are taken: level 0 (32 rows per unit), the forward levels, the dense tail
// (one row per unit), the backward levels from the last to level 0.  Lanes
// per row: about six stored entries per lane, so that a lane's batch of
// eight loads is mostly full (a power of two in 1..32), times 2^shift.  Each int4 is (kind | G << 8, first row, end row, first
// unit); *nunits receives the total.
std::vector<int4> build_flow_list(const HostFactor& F, int shift, int* nunits) {
  std::vector<int4> seg;
  const std::vector<int>& lvp = F.level_ptr;
  const int nl = F.nlev;
  auto pick_g = [&](double avg) {
    int g = 1;
    while (g < 32 && 2 * g <= avg / 6.0) g *= 2;
    for (int i = 0; i < shift && g < 32; ++i) g *= 2;
    for (int i = 0; i > shift && g > 1; --i) g /= 2;
    return g;
  };
  int64_t u = 0;
  auto add = [&](int kind, int p0, int p1, int g) {
    const int per = kind == PH_DENSE ? 1 : 32 / g;  // rows per unit
    seg.push_back(make_int4(kind | (g << 8), p0, p1, (int)u));
    u += (p1 - p0 + per - 1) / per;
  };
  add(PH_GATHER, lvp[0], lvp[1], 1);
  for (int l = 1; l <= nl; ++l) {
    const int p0 = lvp[l], p1 = lvp[l + 1];
    if (p1 <= p0) continue;
    add(PH_FWD, p0, p1, pick_g((double)(F.Lptr[p1] - F.Lptr[p0]) / (p1 - p0)));
  }
  if (F.n_dense > 0) add(PH_DENSE, lvp[nl], lvp[nl + 1], 32);
  for (int l = nl - 1; l >= 0; --l) {
    const int p0 = lvp[l], p1 = lvp[l + 1];
    if (p1 <= p0) continue;
    add(PH_BWD, p0, p1, pick_g((double)(F.Uptr[p1] - F.Uptr[p0]) / (p1 - p0)));
  }
  *nunits = (int)u;
  return seg;
}

template <typename T>
int upload_dataflow_units(const HostFactor& F, DevFactor<T>& d, int shift, cudaStream_t st) {
  int nu = 0;
  const std::vector<int4> seg = build_flow_list(F, shift, &nu);
  if (!d.units || (int)seg.size() != d.nseg) {
    cudaFree(d.units);
    d.units = nullptr;
    AJD_CUDA(cudaMalloc(&d.units, std::max<size_t>(1, seg.size()) * sizeof(int4)));
  }
  if (!seg.empty()) AJD_CUDA(cudaMemcpyAsync(d.units, seg.data(), seg.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
  AJD_CUDA(cudaStreamSynchronize(st));
  d.nseg = (int)seg.size();
  d.nunits = nu;
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
  // w and z adjacent (z = w + n), so that the dataflow apply fills both with
  // its sentinel in one memset; z is not a separate allocation
  AJD_CUDA(cudaMalloc(&d.w, 2 * nb * sizeof(T)));
  d.z = d.w + nb;
  if (poison) AJD_CUDA(cudaMemsetAsync(d.w, 0xFF, 2 * nb * sizeof(T), st));
  if (sizeof(T) == 4) {  // float-float work vectors of the mixed apply
    AJD_CUDA(cudaMalloc(&d.wdf, 2 * nb * sizeof(float2)));
    d.zdf = d.wdf + nb;
    if (poison) AJD_CUDA(cudaMemsetAsync(d.wdf, 0xFF, 2 * nb * sizeof(float2), st));
  }
  // phase list of the persistent apply (threads-per-row rule unscaled; the
  // autotuner may replace it once the factor is on the device)
  const std::vector<int4> ph = build_phase_list(F, 0);
  d.nphase = (int)ph.size();
  AJD_CUDA(cudaMalloc(&d.phases, std::max<size_t>(1, ph.size()) * sizeof(int4)));
  if (!ph.empty()) {
    AJD_CUDA(cudaMemcpyAsync(d.phases, ph.data(), ph.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    AJD_CUDA(cudaStreamSynchronize(st));
  }
  // status words: [64] the timeout flag of the apply's waits (its own
  // 128-byte line); completion counters of the phases
  AJD_CUDA(cudaMalloc(&d.bar, 96 * sizeof(unsigned)));
  AJD_CUDA(cudaMalloc(&d.done, std::max<size_t>(1, ph.size()) * sizeof(unsigned)));
  AJD_CUDA(cudaMemsetAsync(d.bar, 0, 96 * sizeof(unsigned), st));
  AJD_CUDA(cudaStreamSynchronize(st));
  AJD_TRY(upload_dataflow_units(F, d, 0, st));
  d.form = F.apply_form;
  int per_sm = 0, per_sm_flow = 0;
  AJD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ildl_apply_persistent_kernel<T, T, T>, kPersistThreads, 0));
  AJD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_flow, ildl_apply_dataflow_kernel<T, T, T>,
                                                         kPersistThreads, 0));
  if (per_sm < 1 || per_sm_flow < 1) return fail(JD_EDEVICE, "ildl: persistent apply kernel cannot be resident");
  d.grid = sm_count();  // one CTA per SM
  d.ready = true;
  return JD_OK;
}

thread_local bool tl_serialize_applies = false;
std::mutex g_chain_mu;
cudaEvent_t g_chain_last = nullptr;  // completion of the last serialised apply

}  // namespace

void set_apply_serialization(bool on) { tl_serialize_applies = on; }
bool apply_serialization() { return tl_serialize_applies; }

// Events that the autotuner has recorded around the next apply of this
// thread: `begin` after the apply has joined the chain of serialised
// applies (so waiting for another solve's apply is not timed), `end` after
// its kernel.
thread_local cudaEvent_t tl_time_begin = nullptr, tl_time_end = nullptr;

// Cooperative launch of `kernel` on d.grid CTAs after `pre` (the apply's
// memsets), ordered behind the previous serialised apply when this thread
// serialises its applies.
template <typename V, typename Pre>
int launch_cooperative(const DevFactor<V>& d, const void* kernel, void** args, cudaStream_t s, Pre&& pre) {
  auto body = [&]() -> int {
    if (tl_time_begin) AJD_CUDA(cudaEventRecord(tl_time_begin, s));
    AJD_TRY(pre());
    AJD_CUDA(cudaLaunchCooperativeKernel(kernel, dim3(d.grid), dim3(kPersistThreads), args, 0, s));
    if (tl_time_end) AJD_CUDA(cudaEventRecord(tl_time_end, s));
    return JD_OK;
  };
  if (tl_serialize_applies) {
    // concurrent solvers: this apply starts on the device only after the
    // previous serialised apply (of any thread) has finished, so no two of
    // these grid-wide cooperative kernels ever run at the same time
    std::lock_guard<std::mutex> lk(g_chain_mu);
    if (g_chain_last) AJD_CUDA(cudaStreamWaitEvent(s, g_chain_last, 0));
    AJD_TRY(body());
    cudaEvent_t ev = nullptr;
    AJD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    AJD_CUDA(cudaEventRecord(ev, s));
    if (g_chain_last) cudaEventDestroy(g_chain_last);  // released once it has completed
    g_chain_last = ev;
  } else {
    AJD_TRY(body());
  }
  return JD_OK;
}

// One dataflow apply: w and z filled with the "not yet written" sentinel,
// then the kernel.
template <typename V, typename X, typename IO>
int launch_apply_dataflow(const ildl_s* f, const DevFactor<V>& d, X* w, X* z, const IO* b, IO* out, cudaStream_t s) {
  const HostFactor& F = f->F;
  ApplyArgs<V, X, IO> a{d.perm, d.scale, d.Lptr, d.Lcol, d.Lval, d.Uptr, d.Ucol, d.Uval, d.dd, d.dof, d.partner,
                        d.dense, w, z, b, out, F.n_dense, F.level_ptr[F.nlev]};
  auto fill = [&]() -> int {
    if (z == w + F.n) {  // the factor's own work vectors: one fill
      AJD_CUDA(cudaMemsetAsync(w, 0xFF, 2 * (size_t)F.n * sizeof(X), s));
    } else {
      AJD_CUDA(cudaMemsetAsync(w, 0xFF, (size_t)F.n * sizeof(X), s));
      AJD_CUDA(cudaMemsetAsync(z, 0xFF, (size_t)F.n * sizeof(X), s));
    }
    return JD_OK;
  };
  const int4* units = d.units;
  int nseg = d.nseg, nunits = d.nunits;
  int* err = reinterpret_cast<int*>(d.bar + 64);
  // AJD_APPLY_TIMING=1: record when each segment's last unit finished
  // (globaltimer) and print a per-kind summary of the apply to stderr
  static const bool timing = std::getenv("AJD_APPLY_TIMING") != nullptr;
  unsigned long long* stamps = nullptr;
  if (timing) {
    AJD_CUDA(cudaMalloc(&stamps, (nseg + 1) * sizeof(unsigned long long)));
    AJD_CUDA(cudaMemsetAsync(stamps, 0, (nseg + 1) * sizeof(unsigned long long), s));
  }
  void* args[] = {&a, &units, &nseg, &nunits, &err, &stamps};
  AJD_TRY(launch_cooperative(d, (const void*)ildl_apply_dataflow_kernel<V, X, IO>, args, s, fill));
  count_launches(timing ? 4 : 3);
  if (timing) {
    std::vector<unsigned long long> t(nseg + 1);
    std::vector<int4> sg(nseg);
    AJD_CUDA(cudaMemcpyAsync(t.data(), stamps, (nseg + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    AJD_CUDA(cudaMemcpyAsync(sg.data(), d.units, nseg * sizeof(int4), cudaMemcpyDeviceToHost, s));
    AJD_CUDA(cudaStreamSynchronize(s));
    cudaFree(stamps);
    // a segment's share: how far its completion moved the running maximum
    double kind_us[4] = {0, 0, 0, 0};
    int kind_n[4] = {0, 0, 0, 0};
    unsigned long long last = t[0];
    for (int i = 0; i < nseg; ++i) {
      const unsigned long long ti = std::max(t[i + 1], last);
      const double us = (ti - last) * 1e-3;
      last = ti;
      kind_us[sg[i].x & 0xFF] += us;
      kind_n[sg[i].x & 0xFF]++;
      if (std::getenv("AJD_APPLY_TIMING_ALL"))
        std::fprintf(stderr, "segment %d kind %d rows %d G %d units from %d: done at %.2f us (+%.2f)\n", i,
                     sg[i].x & 0xFF, sg[i].z - sg[i].y, sg[i].x >> 8, sg[i].w, (t[i + 1] - t[0]) * 1e-3, us);
    }
    std::fprintf(stderr, "dataflow apply %.1f us: gather %.1f (%d) fwd %.1f (%d) dense %.1f (%d) bwd %.1f (%d)\n",
                 (last - t[0]) * 1e-3, kind_us[0], kind_n[0], kind_us[1], kind_n[1], kind_us[2], kind_n[2], kind_us[3],
                 kind_n[3]);
  }
  return JD_OK;
}

// One persistent apply with factor values V, work vectors X, caller vectors
// IO, in the factor's apply form.
template <typename V, typename X, typename IO>
int launch_apply(const ildl_s* f, const DevFactor<V>& d, X* w, X* z, const IO* b, IO* out, cudaStream_t s) {
  if (!d.ready) return fail(JD_EINVAL, "ildl_apply: factor has no device copy (use ildl_create)");
  const HostFactor& F = f->F;
  if (F.n == 0 || d.nphase == 0) return JD_OK;
  if (d.form == 1) return launch_apply_dataflow<V, X, IO>(f, d, w, z, b, out, s);
  ApplyArgs<V, X, IO> a{d.perm, d.scale, d.Lptr, d.Lcol, d.Lval, d.Uptr, d.Ucol, d.Uval, d.dd, d.dof, d.partner,
                        d.dense, w, z, b, out, F.n_dense, F.level_ptr[F.nlev]};
  // the phases' completion counters start at zero
  auto clear = [&]() -> int {
    AJD_CUDA(cudaMemsetAsync(d.done, 0, (size_t)d.nphase * sizeof(unsigned), s));
    return JD_OK;
  };
  const int4* ph = d.phases;
  int np = d.nphase;
  unsigned* done = d.done;
  int* err = reinterpret_cast<int*>(d.bar + 64);
  // AJD_APPLY_TIMING=1: record the start of every phase (globaltimer, CTA 0)
  // and print a per-kind summary of the next apply to stderr (diagnostics)
  static const bool timing = std::getenv("AJD_APPLY_TIMING") != nullptr;
  unsigned long long* stamps = nullptr;
  if (timing) AJD_CUDA(cudaMalloc(&stamps, (np + 1) * sizeof(unsigned long long)));
  void* args[] = {&a, &ph, &np, &done, &err, &stamps};
  AJD_TRY(launch_cooperative(d, (const void*)ildl_apply_persistent_kernel<V, X, IO>, args, s, clear));
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
      kind_us[phs[i].x & 0xFF] += us;
      kind_n[phs[i].x & 0xFF]++;
      if (std::getenv("AJD_APPLY_TIMING_ALL"))
        std::fprintf(stderr, "phase %d kind %d rows %d G %d cta %d ctas %d: %.2f us\n", i, phs[i].x & 0xFF,
                     phs[i].z - phs[i].y, phs[i].w & 0xFFFF, phs[i].w >> 16, phs[i].x >> 8, us);
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
  const DevFactor<float>& d = f->d32;
  if (!d.wdf) return fail(JD_EINVAL, "ildl_apply: no mixed-precision work vectors");
  return launch_apply<float, df64, double>(f, d, reinterpret_cast<df64*>(d.wdf), reinterpret_cast<df64*>(d.zdf), b,
                                           out, s);
}

// Timeout flag of the persistent apply (sticky until cleared): JD_EDEVICE if
// a wait of the apply gave up.
int ildl_check_device_error(const ildl_s* f, cudaStream_t s) {
  for (int prec = 0; prec < 2; ++prec) {
    const unsigned* bar = prec == 0 ? f->d64.bar : f->d32.bar;
    if (!bar) continue;
    int e = 0;
    AJD_CUDA(cudaMemcpyAsync(&e, bar + 64, sizeof(int), cudaMemcpyDeviceToHost, s));
    AJD_CUDA(cudaStreamSynchronize(s));
    if (e) return fail(JD_EDEVICE, "ildl_apply: a device-side wait timed out");
  }
  return JD_OK;
}

template int ildl_apply_dev<double>(const ildl_s*, const double*, double*, cudaStream_t);
template int ildl_apply_dev<float>(const ildl_s*, const float*, float*, cudaStream_t);

// Invert the dense trailing block (host matrix in, host inverse out) on the
// current device (blocked Gauss-Jordan, csrc/dense_inverse.cu).
int invert_dense_on_device(dvec<double>& M, int m, cudaStream_t st) {
  if (m == 0) return JD_OK;
  const size_t bytes = (size_t)m * m * sizeof(double);
  double *A = nullptr, *X = nullptr;
  int* bad = nullptr;
  cudaError_t e = cudaMalloc(&A, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&X, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&bad, sizeof(int));
  int rc = JD_OK;
  if (e == cudaSuccess) e = cudaMemcpyAsync(A, M.data(), bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    rc = dense_inverse_device(A, X, m, bad, st);
    int hbad = 0;
    if (rc == JD_OK) {
      e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(M.data(), X, bytes, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e == cudaSuccess && hbad) rc = fail(JD_ESETUP, "ildl: the final dense block (%d rows) is singular", m);
    }
  }
  if (e != cudaSuccess) rc = fail(JD_EDEVICE, "ildl dense inverse: %s", cudaGetErrorString(e));
  cudaFree(A);
  cudaFree(X);
  cudaFree(bad);
  return rc;
}

namespace {

// Autotuning of the apply, per factor: both apply forms (dataflow, level
// counters), each with the rule's threads per row and with every level's
// threads per row halved and doubled, are timed on the device (CUDA events
// on the setup stream: one warm-up and the fastest of three timed applies of
// a zero vector; the apply's work does not depend on the values) and the
// fastest is kept, the level counters only when faster by more than 25%
// (the timings are taken while other setups may share the device).
// A form fixed by the caller is tuned over the threads per row only.  The
// timed applies join the chain that orders the applies of concurrent solves,
// so they never run beside one.  Only factors of at least kTuneMinRows rows
// are tuned (below, a whole apply takes tens of microseconds and the choice
// matters little).
constexpr int kTuneMinRows = 200000;

template <typename T>
int set_apply_shape(const HostFactor& F, DevFactor<T>& d, int form, int shift, cudaStream_t st) {
  // the level-counter list always stays valid (the allocation-free apply
  // launches that form whatever the factor's choice)
  const std::vector<int4> ph = build_phase_list(F, form == 0 ? shift : 0);
  AJD_CUDA(cudaMemcpyAsync(d.phases, ph.data(), ph.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
  AJD_TRY(upload_dataflow_units(F, d, form == 1 ? shift : 0, st));  // synchronises st
  d.form = form;
  return JD_OK;
}

template <typename T>
int autotune_apply(ildl_s* f, DevFactor<T>& d, int form_req, cudaStream_t st) {
  const HostFactor& F = f->F;
  if (F.n < kTuneMinRows || d.nphase == 0) return JD_OK;
  double* b = nullptr;
  double* x = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool was = tl_serialize_applies;
  tl_serialize_applies = true;
  int rc = JD_OK;
  // the fastest of three timed applies after one warm-up: the setups of
  // other problems may share the device meanwhile, and the minimum is the
  // least disturbed of the three
  auto run = [&](double* ms) -> int {
    *ms = 0.0;
    for (int rep = 0; rep < 4; ++rep) {
      // events recorded inside the launch, after the wait for the chain
      tl_time_begin = e0;
      tl_time_end = e1;
      int r;
      if constexpr (sizeof(T) == 8) {
        r = launch_apply<double, double, double>(f, d, d.w, d.z, b, x, st);
      } else {
        r = launch_apply<float, df64, double>(f, d, reinterpret_cast<df64*>(d.wdf), reinterpret_cast<df64*>(d.zdf),
                                              b, x, st);
      }
      tl_time_begin = tl_time_end = nullptr;
      AJD_TRY(r);
      AJD_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      AJD_CUDA(cudaEventElapsedTime(&t, e0, e1));
      if (rep == 1 || (rep > 1 && t < *ms)) *ms = t;
    }
    return JD_OK;
  };
  auto body = [&]() -> int {
    AJD_CUDA(cudaMalloc(&b, sizeof(double) * (size_t)F.n));
    AJD_CUDA(cudaMalloc(&x, sizeof(double) * (size_t)F.n));
    AJD_CUDA(cudaMemsetAsync(b, 0, sizeof(double) * (size_t)F.n, st));
    AJD_CUDA(cudaEventCreate(&e0));
    AJD_CUDA(cudaEventCreate(&e1));
    // the dataflow form first; the level-counter form replaces it only when
    // clearly faster (by more than kFormMargin): alone on the device it is
    // slower in every precision, and timing noise under load must not flip
    // the choice
    constexpr double kFormMargin = 0.25;
    int best_form = -1, best_shift = 0;
    double best_ms = 0.0;
    for (int form : {1, 0}) {
      if (form_req >= 0 && form != form_req) continue;
      for (int shift : {0, -1, 1}) {
        AJD_TRY(set_apply_shape(F, d, form, shift, st));
        double ms = 0.0;
        AJD_TRY(run(&ms));
        f->F.apply_tune_ms[form][shift + 1] = ms;
        if (std::getenv("AJD_SETUP_VERBOSE"))
          std::fprintf(stderr, "ildl apply autotune: form %d shift %+d: %.3f ms\n", form, shift, ms);
        const double bar = (best_form == 1 && form == 0) ? best_ms * (1.0 - kFormMargin) : best_ms;
        if (best_form < 0 || ms < bar) {
          best_ms = ms;
          best_form = form;
          best_shift = shift;
        }
      }
    }
    AJD_TRY(set_apply_shape(F, d, best_form, best_shift, st));
    f->F.apply_form = best_form;
    f->F.apply_shift = best_shift;
    return JD_OK;
  };
  rc = body();
  tl_serialize_applies = was;
  cudaFree(b);
  cudaFree(x);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}

}  // namespace

int ildl_upload_all(ildl_s* f, cudaStream_t st, int copies, bool tune, int form_req) {
  using Clock = std::chrono::steady_clock;
  auto ms_since = [](Clock::time_point t) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t).count();
  };
  const bool verbose = std::getenv("AJD_SETUP_VERBOSE") != nullptr;
  auto t = Clock::now();
  if (f->F.dense_is_matrix) {
    AJD_TRY(invert_dense_on_device(f->F.dense_inv, f->F.n_dense, st));
    f->F.dense_is_matrix = false;
  }
  if (verbose) std::fprintf(stderr, "ildl dense inverse on the device (%d rows): %.1f ms\n", f->F.n_dense, ms_since(t));
  t = Clock::now();
  f->F.apply_form = form_req >= 0 ? form_req : kDefaultApplyForm;
  f->F.apply_shift = 0;
  if (copies & kCopyF64) AJD_TRY(upload_factor<double>(f->F, f->d64, st));
  if (copies & kCopyF32) AJD_TRY(upload_factor<float>(f->F, f->d32, st));
  if (verbose) std::fprintf(stderr, "ildl upload (copies %d): %.1f ms\n", copies, ms_since(t));
  t = Clock::now();
  if (tune) {
    // tuned on the copy a solve uses first (binary32 for the mixed and
    // binary32 solves); the other copy takes the same choice
    if (copies & kCopyF32) AJD_TRY(autotune_apply<float>(f, f->d32, form_req, st));
    else if (copies & kCopyF64) AJD_TRY(autotune_apply<double>(f, f->d64, form_req, st));
    if ((copies & kCopyF32) && (copies & kCopyF64))
      AJD_TRY(set_apply_shape(f->F, f->d64, f->F.apply_form, f->F.apply_shift, st));
    if (verbose)
      std::fprintf(stderr, "ildl apply autotune (form %d shift %d): %.1f ms\n", f->F.apply_form, f->F.apply_shift,
                   ms_since(t));
  }
  return JD_OK;
}

void ildl_free_device(ildl_s* f) {
  free_dev(f->d64);
  free_dev(f->d32);
}

// CSR of A - sigma I for a lattice (host, from the binary64 potential).
int lattice_csr(const anderson_s* h, const std::vector<double>& eps, const std::vector<double>& bonds, double sigma,
                SymCsr& A) {
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
    // neighbour (xx, yy, zz) across the bond of direction d stored at site
    // `lower` (the site it leaves in the +d direction)
    auto add = [&](int xx, int yy, int zz, int d, bool minus) {
      if (per) {
        xx = (xx + L) % L;
        yy = (yy + L) % L;
        zz = (zz + L) % L;
      } else if (xx < 0 || xx >= L || yy < 0 || yy >= L || zz < 0 || zz >= L) {
        return;
      }
      const int64_t t = xx + (int64_t)L * (yy + (int64_t)L * zz);
      nb[k] = (int)t;
      nv[k] = bonds.empty() ? h->hop : bonds[3 * (minus ? t : s) + d];
      ++k;
    };
    add(x - 1, y, z, 0, true);
    add(x + 1, y, z, 0, false);
    add(x, y - 1, z, 1, true);
    add(x, y + 1, z, 1, false);
    add(x, y, z - 1, 2, true);
    add(x, y, z + 1, 2, false);
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
  p->n_dense = 0;
  p->matching = -1;
  p->aggressive = 0.0;
  p->setup_device = -1;
  p->autotune = -1;
  p->apply_form = -1;
  return JD_OK;
}

extern "C" int ildl_default_gamma(int64_t n, int offdiag, double* gamma) {
  if (n < 1 || !gamma) return fail(JD_EINVAL, "ildl_default_gamma: n >= 1 and a non-NULL gamma required");
  *gamma = default_gamma(n, offdiag != 0);
  return JD_OK;
}

static int check_params(const ildl_params* p, ildl_params& out) {
  if (p) out = *p;
  else ildl_params_default(&out);
  if (!(out.kappa > 1.0)) return fail(JD_EINVAL, "ildl: kappa must be > 1");
  if (!std::isfinite(out.drop) && out.drop > 0) return fail(JD_EINVAL, "ildl: drop must be finite");
  if (out.gamma >= 1.0 || std::isnan(out.gamma)) return fail(JD_EINVAL, "ildl: gamma must be < 1");
  if (!(out.aggressive >= 0.0 && out.aggressive < 1.0))
    return fail(JD_EINVAL, "ildl: aggressive dropping tau must be in [0, 1)");
  if (out.apply_form < -1 || out.apply_form > 1) return fail(JD_EINVAL, "ildl: apply_form must be -1, 0 or 1");
  if (out.max_levels < 1 || out.n_dense < 0 || out.n_dense > 8000)
    return fail(JD_EINVAL, "ildl: max_levels >= 1 and 0 <= n_dense <= 8000 required");
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
    std::unique_ptr<SchurEngine> eng;
    if (prm.setup_device > 0) eng = make_device_schur(0);
    int rc = build_ildl(B, prm, f->F, true, eng.get());
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
  // off-diagonal disorder (Section 7): the factor loses more by ignoring
  // weak couplings, so the default threshold is min(0.02, 1/sqrt(n)) instead
  // of min(0.02, 5/sqrt(n)) -- five times smaller from L = 40 on, 0.0053
  // against 0.02 at L = 33 (measured with SQMR on A x = b: at L = 33, 78-80
  // iterations with 0.02, 29-43 with 1/sqrt(n))
  if (prm.gamma < 0.0) prm.gamma = default_gamma(h->n, h->bond64 != nullptr);
  try {
    std::vector<double> eps(h->n), bonds(h->bond64 ? 3 * h->n : 0);
    AJD_CUDA(cudaMemcpyAsync(eps.data(), h->eps64, h->n * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (h->bond64)
      AJD_CUDA(cudaMemcpyAsync(bonds.data(), h->bond64, 3 * h->n * sizeof(double), cudaMemcpyDeviceToHost, st));
    AJD_CUDA(cudaStreamSynchronize(st));
    SymCsr A;
    lattice_csr(h, eps, bonds, sigma, A);
    ildl_s* f = new ildl_s();
    f->device = h->device;
    const auto t0 = std::chrono::steady_clock::now();
    // the levels' Schur complements on the lattice's device unless asked
    // for on the host
    std::unique_ptr<SchurEngine> eng;
    if (prm.setup_device != 0) eng = make_device_schur(st);
    int rc = build_ildl(A, prm, f->F, /*dense_on_host=*/false, eng.get());
    eng.reset();
    if (std::getenv("AJD_SETUP_VERBOSE"))
      std::fprintf(stderr, "ildl host build: %.1f ms\n",
                   std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
    if (rc == JD_OK) rc = ildl_upload_all(f, st, copies, prm.autotune != 0, prm.apply_form);
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
  info->aggressive_dropped = F.n_aggressive;
  info->apply_shift = F.apply_shift;
  info->apply_form = F.apply_form;
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

extern "C" int ildl_dataflow_schedule(ildl_t f, int shift, int* seg, int cap, int* nseg, int* nunits) {
  if (!f || !nseg || !nunits) return fail(JD_EINVAL, "ildl_dataflow_schedule: NULL argument");
  if (shift < -1 || shift > 1) return fail(JD_EINVAL, "ildl_dataflow_schedule: shift must be -1, 0 or 1");
  int nu = 0;
  const std::vector<int4> ph = build_flow_list(f->F, shift, &nu);
  *nseg = (int)ph.size();
  *nunits = nu;
  if (cap < (int)ph.size() || (!seg && !ph.empty()))
    return fail(JD_EINVAL, "ildl_dataflow_schedule: room for %d segments, %zu needed", cap, ph.size());
  for (size_t i = 0; i < ph.size(); ++i) {
    int* o = seg + 5 * i;
    o[0] = ph[i].x & 0xFF;
    o[1] = ph[i].x >> 8;
    o[2] = ph[i].y;
    o[3] = ph[i].z;
    o[4] = ph[i].w;
  }
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
  if (f->d64.ready || f->d32.ready) {
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
// under an allocator that forbids it (a memory pool reserved up front, an
// embedding runtime that owns all device memory).  ildl_apply_noalloc serves
// them: it launches the same persistent kernel as ildl_apply but takes its
// scratch (the two work vectors and the status words) from one
// file-scope device array instead of the factor's own buffers.  Nothing is
// allocated or freed.  The call is synchronous: it waits for the apply and
// reads its timeout flag before returning.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxN = 131072;  // largest order served (L <= 50 lattices)
constexpr int kNoAllocMaxPhases = 4096;   // phase counters (2 per sparse level + 2 per factor)
constexpr size_t kNoAllocVecBytes = (size_t)kNoAllocMaxN * sizeof(double);
// w, z, status words, phase counters
constexpr size_t kNoAllocBytes = 2 * kNoAllocVecBytes + 512 + kNoAllocMaxPhases * sizeof(unsigned);

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
  // the array keeps the previous call's contents: the timeout flag and the
  // phase counters (behind the status words) must start at zero; w and z
  // are written before they are read
  unsigned* done = bar + 128;
  AJD_CUDA(cudaMemsetAsync(bar, 0, 128 * sizeof(unsigned) + (size_t)d.nphase * sizeof(unsigned), s));
  const int4* ph = d.phases;
  int np = d.nphase;
  int* err = reinterpret_cast<int*>(bar + 64);
  unsigned long long* stamps = nullptr;
  void* args[] = {&a, &ph, &np, &done, &err, &stamps};
  {
    // ordered behind the applies of concurrent served solves (the same
    // event chain), so this grid-wide kernel never runs beside one of them
    std::lock_guard<std::mutex> lk(g_chain_mu);
    if (g_chain_last) AJD_CUDA(cudaStreamWaitEvent(s, g_chain_last, 0));
    AJD_CUDA(cudaLaunchCooperativeKernel((void*)ildl_apply_persistent_kernel<V, X, IO>, dim3(d.grid),
                                         dim3(kPersistThreads), args, 0, s));
    cudaEvent_t ev = nullptr;
    AJD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    AJD_CUDA(cudaEventRecord(ev, s));
    if (g_chain_last) cudaEventDestroy(g_chain_last);
    g_chain_last = ev;
  }
  count_launches(2);
  int herr = 0;
  AJD_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  AJD_CUDA(cudaStreamSynchronize(s));
  if (herr) return fail(JD_EDEVICE, "ildl_apply_noalloc: a device-side wait timed out");
  return JD_OK;
}

}  // namespace

extern "C" int ildl_apply_noalloc(ildl_t f, const void* b, void* x, int precision, void* stream) {
  if (!f || !b || !x) return fail(JD_EINVAL, "ildl_apply_noalloc: NULL argument");
  if (b == x) return fail(JD_EINVAL, "ildl_apply_noalloc: b and x must be distinct");
  if ((int64_t)f->F.n > kNoAllocMaxN)
    return fail(JD_EINVAL, "ildl_apply_noalloc: order %d exceeds the static scratch limit of %lld rows", f->F.n,
                (long long)kNoAllocMaxN);
  const int nphase = std::max(f->d64.nphase, f->d32.nphase);
  if (nphase > kNoAllocMaxPhases)
    return fail(JD_EINVAL, "ildl_apply_noalloc: %d phases exceed the static scratch limit of %d", nphase,
                kNoAllocMaxPhases);
  // the scratch array looked up below is the current device's; the
  // factor's arrays live on f->device
  int cur = 0;
  AJD_CUDA(cudaGetDevice(&cur));
  if (cur != f->device)
    return fail(JD_EINVAL, "ildl_apply_noalloc: current device %d is not the factor's device %d", cur, f->device);
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
    if (!f->d32.ready) return fail(JD_EINVAL, "ildl_apply_noalloc: factor has no device copy");
    return launch_apply_static<float, df64, double>(f, f->d32, static_cast<const double*>(b), static_cast<double*>(x),
                                              scratch, s);
  }
  return fail(JD_EINVAL, "ildl_apply_noalloc: unknown precision %d", precision);
}
