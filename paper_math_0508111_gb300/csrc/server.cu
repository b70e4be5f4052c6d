// Request loop for many independent eigensolves (jd_server_*): admission by
// a device-memory budget, preconditioner builds on host threads, concurrent
// solves on per-slot CUDA streams.
#include <omp.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "jd_impl.cuh"

namespace ajd {
namespace {

using Clock = std::chrono::steady_clock;

enum State { QUEUED = 0, BUILDING = 1, READY = 2, SOLVING = 3, DONE = 4 };

struct Request {
  uint64_t id = 0;
  int L = 0, bc = 0, k = 0, flags = 0;
  double W = 0.0, sigma = 0.0, tol = 0.0;
  uint64_t seed = 0;
  size_t est = 0;
  State state = QUEUED;
  Clock::time_point t_submit, t_done;
  anderson_s* h = nullptr;
  ildl_s* pc = nullptr;
  int status = JD_OK;
  std::string msg;
  std::vector<double> evals, evecs;
  jd_stats st{};
};

size_t estimate_bytes(int L, int k, const jd_params& p) {
  const double n = (double)L * L * L;
  const double nd = std::min(n, (double)(p.ildl.n_dense > 0 ? p.ildl.n_dense : default_n_dense((int64_t)n)));
  const double fill = n > nd ? 60.0 : 0.0;  // stored entries of L per row (56.6 measured at L = 100)
  const int kint = k + 2;
  const int jmin = p.jmin > 0 ? p.jmin : std::max(2 * kint, 10);
  const int jmax = std::min(64, p.jmax > 0 ? p.jmax : jmin + 15);
  const double per_row = 12.0                      // potential, binary64 + binary32
                         + 160.0 + 56.0 * fill     // device copies of the factor (bound: all three)
                         + 8.0 * (4.0 * jmax + kint + 4) + 8.0 * (2.0 * (kint + 1) + 8);  // solver
  return (size_t)(n * per_row + nd * nd * 16.0) + ((size_t)64 << 20);
}

}  // namespace
}  // namespace ajd

struct jd_server_s {
  jd_server_params prm{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<ajd::Request*> pending, ready;
  std::unordered_map<uint64_t, std::unique_ptr<ajd::Request>> all;
  size_t reserved = 0, peak_reserved = 0;
  uint64_t next_id = 1;
  int64_t submitted = 0, completed = 0, failed = 0;
  int building = 0, solving = 0, peak_solving = 0;
  bool stop = false;
  std::vector<std::thread> workers;
};

namespace ajd {
namespace {

void finish(jd_server_s* S, Request* r, int status, const char* msg) {
  // caller holds S->mu
  r->status = status;
  if (msg) r->msg = msg;
  r->state = DONE;
  r->t_done = Clock::now();
  if (status != JD_OK && status != JD_ENOCONV) ++S->failed;
  else ++S->completed;
  S->cv.notify_all();
}

void build_loop(jd_server_s* S, int omp_threads) {
  cudaSetDevice(S->device);
  omp_set_num_threads(omp_threads);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // admission: arrival order, while the estimate fits the budget (a
      // request always fits an empty server: jd_submit rejected larger ones)
      S->cv.wait(lk, [&] {
        return S->stop || (!S->pending.empty() &&
                           (S->reserved == 0 || S->reserved + S->pending.front()->est <= S->prm.hbm_budget));
      });
      if (S->stop) break;
      r = S->pending.front();
      S->pending.pop_front();
      S->reserved += r->est;
      S->peak_reserved = std::max(S->peak_reserved, S->reserved);
      r->state = BUILDING;
      ++S->building;
    }
    const auto t0 = Clock::now();
    anderson_t h = nullptr;
    ildl_t pc = nullptr;
    int rc = anderson_create(r->L, r->W, r->seed, r->bc, &h);
    if (rc == JD_OK)
      rc = ildl_create_on_stream(h, r->sigma, &S->prm.solve.ildl, &pc, st, copy_for_precision(S->prm.solve.precision));
    const std::string msg = rc == JD_OK ? std::string() : std::string(jd_last_error());
    const double ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    std::lock_guard<std::mutex> lk(S->mu);
    --S->building;
    if (rc != JD_OK) {
      if (pc) ildl_destroy(pc);
      if (h) anderson_destroy(h);
      S->reserved -= r->est;
      finish(S, r, rc, msg.c_str());
      continue;
    }
    if (S->stop) {  // the server is shutting down: drop the request
      ildl_destroy(pc);
      anderson_destroy(h);
      S->reserved -= r->est;
      finish(S, r, JD_EINVAL, "jd_server_destroy: request dropped");
      continue;
    }
    r->h = h;
    r->pc = pc;
    r->st.setup_ms = ms;
    r->state = READY;
    S->ready.push_back(r);
    S->cv.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

void solve_loop(jd_server_s* S) {
  cudaSetDevice(S->device);
  set_apply_serialization(true);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || !S->ready.empty(); });
      if (S->stop) break;
      r = S->ready.front();
      S->ready.pop_front();
      r->state = SOLVING;
      ++S->solving;
      S->peak_solving = std::max(S->peak_solving, S->solving);
    }
    const int64_t n = r->h->n;
    r->evals.assign(r->k, 0.0);
    if (r->flags & JD_SUBMIT_VECTORS) r->evecs.assign((size_t)n * r->k, 0.0);
    const double setup_ms = r->st.setup_ms;
    ildl_info(r->pc, &r->st.ildl);
    jd_stats st_out{};
    int rc = solve_problem(r->h, r->pc, S->prm.solve, r->sigma, r->k, r->tol, r->evals.data(),
                           r->evecs.empty() ? nullptr : r->evecs.data(), &st_out, st);
    const std::string msg = rc == JD_OK ? std::string() : std::string(jd_last_error());
    st_out.setup_ms = setup_ms;
    st_out.ildl = r->st.ildl;
    ildl_destroy(r->pc);
    anderson_destroy(r->h);
    std::lock_guard<std::mutex> lk(S->mu);
    r->pc = nullptr;
    r->h = nullptr;
    r->st = st_out;
    --S->solving;
    S->reserved -= r->est;
    finish(S, r, rc, msg.c_str());
  }
  set_apply_serialization(false);
  if (st) cudaStreamDestroy(st);
}

int take_result(jd_server_s* S, std::unordered_map<uint64_t, std::unique_ptr<Request>>::iterator it, double* evals,
                double* evecs, jd_stats* st, double* latency_ms) {
  // caller holds S->mu; the request is DONE
  Request* r = it->second.get();
  if (evals && !r->evals.empty()) std::memcpy(evals, r->evals.data(), sizeof(double) * r->evals.size());
  if (evecs && !r->evecs.empty()) std::memcpy(evecs, r->evecs.data(), sizeof(double) * r->evecs.size());
  if (st) *st = r->st;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  const int status = r->status;
  const std::string msg = r->msg;
  S->all.erase(it);
  if (status != JD_OK) return fail(status, "%s", msg.c_str());
  return JD_OK;
}

}  // namespace
}  // namespace ajd

using namespace ajd;

extern "C" int jd_server_params_default(jd_server_params* p) {
  if (!p) return fail(JD_EINVAL, "jd_server_params_default: NULL");
  std::memset(p, 0, sizeof(*p));
  p->hbm_budget = 0;
  p->slots = 4;
  p->setup_threads = 2;
  return jd_params_default(&p->solve);
}

extern "C" int jd_server_estimate(int L, int k, size_t* bytes) {
  if (!bytes || L < 1 || k < 1) return fail(JD_EINVAL, "jd_server_estimate: bad arguments");
  jd_params p;
  jd_params_default(&p);
  *bytes = estimate_bytes(L, k, p);
  return JD_OK;
}

extern "C" int jd_server_create(const jd_server_params* p, jd_server_t* out) {
  if (!out) return fail(JD_EINVAL, "jd_server_create: out is NULL");
  *out = nullptr;
  jd_server_params prm;
  if (p) prm = *p;
  else jd_server_params_default(&prm);
  if (prm.slots == 0) prm.slots = 4;
  if (prm.setup_threads == 0) prm.setup_threads = 2;
  if (prm.slots < 1 || prm.slots > 64 || prm.setup_threads < 1 || prm.setup_threads > 64)
    return fail(JD_EINVAL, "jd_server_create: slots and setup_threads must be in 1..64");
  if (prm.solve.precond) return fail(JD_EINVAL, "jd_server_create: solve.precond must be NULL");
  jd_params norm;
  AJD_TRY(normalize_jd_params(&prm.solve, norm));
  prm.solve = norm;
  int dev = 0;
  AJD_CUDA(cudaGetDevice(&dev));
  if (prm.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    AJD_CUDA(cudaMemGetInfo(&fr, &tot));
    prm.hbm_budget = (size_t)(0.8 * (double)fr);
  }
  jd_server_s* S = new (std::nothrow) jd_server_s();
  if (!S) return fail(JD_ENOMEM, "jd_server_create: host allocation failed");
  S->prm = prm;
  S->device = dev;
  const int hw = std::max(1, omp_get_max_threads());
  // the solving threads wait on the device in blocking synchronisation and
  // need almost no CPU: the host cores go to the setups
  const int omp_each = std::max(1, hw / prm.setup_threads);
  try {
    for (int t = 0; t < prm.setup_threads; ++t) S->workers.emplace_back(build_loop, S, omp_each);
    for (int t = 0; t < prm.slots; ++t) S->workers.emplace_back(solve_loop, S);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv.notify_all();
    for (auto& w : S->workers) w.join();
    delete S;
    return fail(JD_ENOMEM, "jd_server_create: cannot start worker threads");
  }
  *out = S;
  return JD_OK;
}

extern "C" int jd_submit(jd_server_t S, int L, double W, uint64_t seed, int bc, double sigma, int k, double tol,
                         int flags, uint64_t* ticket) {
  if (!S || !ticket) return fail(JD_EINVAL, "jd_submit: NULL argument");
  if (bc != JD_PERIODIC && bc != JD_HARDWALL) return fail(JD_EINVAL, "jd_submit: bad bc");
  if ((bc == JD_PERIODIC && L < 3) || L < 1 || (int64_t)L * L * L >= ((int64_t)1 << 31))
    return fail(JD_EINVAL, "jd_submit: bad L = %d", L);
  if (!(W >= 0.0) || !std::isfinite(W)) return fail(JD_EINVAL, "jd_submit: W must be finite and >= 0");
  if (!std::isfinite(sigma)) return fail(JD_EINVAL, "jd_submit: sigma must be finite");
  if (k < 1 || k > 64 || (int64_t)k >= (int64_t)L * L * L) return fail(JD_EINVAL, "jd_submit: bad k = %d", k);
  if (!(tol > 0.0)) return fail(JD_EINVAL, "jd_submit: tol must be > 0");
  auto r = std::make_unique<Request>();
  r->L = L;
  r->W = W;
  r->seed = seed;
  r->bc = bc;
  r->sigma = sigma;
  r->k = k;
  r->tol = tol;
  r->flags = flags;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  r->est = estimate_bytes(L, k, S->prm.solve);
  if (r->est > S->prm.hbm_budget)
    return fail(JD_ENOMEM, "jd_submit: estimated %zu bytes exceed the budget of %zu", r->est, S->prm.hbm_budget);
  if (S->stop) return fail(JD_EINVAL, "jd_submit: server is stopping");
  r->id = S->next_id++;
  *ticket = r->id;
  S->pending.push_back(r.get());
  S->all.emplace(r->id, std::move(r));
  ++S->submitted;
  S->cv.notify_all();
  return JD_OK;
}

extern "C" int jd_poll(jd_server_t S, uint64_t ticket, double* evals, double* evecs, jd_stats* st,
                       double* latency_ms) {
  if (!S) return fail(JD_EINVAL, "jd_poll: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return fail(JD_EINVAL, "jd_poll: unknown ticket %llu", (unsigned long long)ticket);
  if (it->second->state != DONE) return JD_EAGAIN;
  return take_result(S, it, evals, evecs, st, latency_ms);
}

extern "C" int jd_wait(jd_server_t S, uint64_t ticket, double* evals, double* evecs, jd_stats* st,
                       double* latency_ms, double timeout_s) {
  if (!S) return fail(JD_EINVAL, "jd_wait: NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return fail(JD_EINVAL, "jd_wait: unknown ticket %llu", (unsigned long long)ticket);
  Request* r = it->second.get();
  auto done = [&] { return r->state == DONE; };
  if (timeout_s < 0) S->cv.wait(lk, done);
  else if (!S->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) return JD_EAGAIN;
  return take_result(S, it, evals, evecs, st, latency_ms);
}

extern "C" int jd_server_info_get(jd_server_t S, jd_server_info* info) {
  if (!S || !info) return fail(JD_EINVAL, "jd_server_info_get: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(info, 0, sizeof(*info));
  info->submitted = S->submitted;
  info->completed = S->completed;
  info->failed = S->failed;
  info->queued = (int)S->pending.size();
  info->building = S->building;
  info->ready = (int)S->ready.size();
  info->solving = S->solving;
  info->peak_solving = S->peak_solving;
  info->hbm_budget = S->prm.hbm_budget;
  info->reserved_bytes = S->reserved;
  info->peak_reserved_bytes = S->peak_reserved;
  return JD_OK;
}

extern "C" int jd_server_destroy(jd_server_t S) {
  if (!S) return JD_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (Request* r : S->pending) finish(S, r, JD_EINVAL, "jd_server_destroy: request dropped");
    S->pending.clear();
    for (Request* r : S->ready) {  // built, not yet solving: released below
      S->reserved -= r->est;
      finish(S, r, JD_EINVAL, "jd_server_destroy: request dropped");
    }
    S->ready.clear();
  }
  S->cv.notify_all();
  for (auto& w : S->workers) w.join();
  for (auto& kv : S->all) {  // built but never solved
    if (kv.second->pc) ildl_destroy(kv.second->pc);
    if (kv.second->h) anderson_destroy(kv.second->h);
  }
  delete S;
  return JD_OK;
}
