// Host construction of the multilevel incomplete LDL^T preconditioner.
//
// Per level (Section 6.3: reordering, scaling and factorization are applied
// recursively to the Schur complement of the postponed part):
//   1. maximum-product matching (Section 5.1, Eqs. (5.1)-(5.2)) by a sparse
//      shortest-augmenting-path assignment solver with dual potentials;
//   2. symmetric scaling from the duals (entries <= 1 in modulus, matched
//      entries equal to 1; Section 4.2) and the split of the matching's
//      cycles into 1x1 and 2x2 candidate pivots (Section 5.2);
//   3. the 1x1 / 2x2 choice by the d1/d2 block diagonal dominance rule and
//      inverse-based pivoting: a pivot is only taken if the level's
//      ||L^{-1}||_1 stays <= kappa, otherwise it is postponed (Section 6.2);
//   4. ordering: instead of AMD on the compressed graph (Section 5.3), an
//      independent set of the compressed graph's candidates (couplings below
//      gamma ignored) is eliminated, best pivots first.  Each level's block of
//      pivots is then block diagonal, so every level is ONE parallel step of
//      the triangular solves on the GPU;
//   5. the level's column block of L is dropped at epsilon/kappa (Section
//      6.2), optionally sparsified further by the aggressive dropping of
//      Section 6.3, and the Schur complement S = C - L D L^T formed
//      explicitly and dropped at epsilon/kappa; the recursion continues on S
//      until it is small enough to be factored densely.
// The levels are finally concatenated into one global unit lower triangular
// L (rows ordered level by level), one block diagonal D and one scaling.
#include "ildl_setup.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <memory>
#include <numeric>
#include <functional>
#include <type_traits>
#include <utility>
#include <cstdio>
#include <cstdlib>

#include <omp.h>
#include <parallel/algorithm>

namespace ajd {

int fail(int code, const char* fmt, ...);

namespace {

using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

constexpr double kInf = std::numeric_limits<double>::infinity();

// Resize a buffer whose contents are about to be overwritten: within its
// capacity nothing moves; beyond it the old block is released first (no
// copy of stale contents, no second block alive at once).
template <class V>
void resize_discard(V& v, size_t n) {
  if (n > v.capacity()) V().swap(v);
  v.resize(n);
}

// Ascending sort of a short int array: insertion sort up to `small`
// entries (few moves on nearly sorted input, no mispredicted partitions),
// std::sort above.
void sort_ints(int* a, int n, int small) {
  if (n > small) {
    std::sort(a, a + n);
    return;
  }
  for (int x = 1; x < n; ++x) {
    const int c = a[x];
    int y = x;
    for (; y > 0 && a[y - 1] > c; --y) a[y] = a[y - 1];
    a[y] = c;
  }
}

double lookup(const SymCsr& S, int i, int j) {
  const int* b = S.col.data() + S.ptr[i];
  const int* e = S.col.data() + S.ptr[i + 1];
  const int* p = std::lower_bound(b, e, j);
  return (p != e && *p == j) ? S.val[p - S.col.data()] : 0.0;
}

// Natural logarithm of a positive normal double by the atanh series:
// x = m 2^e with m in [sqrt(1/2), sqrt(2)), ln x = e ln 2 + 2 atanh(s),
// s = (m - 1) / (m + 1), |s| < 0.1716, atanh(s) = s + s^3/3 + ... summed to
// s^19 (the first omitted term is below 1e-16 relative).  Used only to build
// the table of log_pos.
double log_series(double x) {
  uint64_t b;
  std::memcpy(&b, &x, sizeof(b));
  int e = (int)((b >> 52) & 0x7ff) - 1023;
  b = (b & 0x000fffffffffffffull) | 0x3ff0000000000000ull;  // mantissa in [1, 2)
  double m;
  std::memcpy(&m, &b, sizeof(m));
  if (m > 1.4142135623730951) {
    m *= 0.5;
    ++e;
  }
  const double s = (m - 1.0) / (m + 1.0), s2 = s * s;
  double t = 1.0 / 19.0;
  for (int k = 17; k >= 1; k -= 2) t = t * s2 + 1.0 / k;
  return (double)e * 0.6931471805599453 + 2.0 * s * t;
}

// Table of the division-free logarithm: the mantissa range [1, 2) is cut
// into 128 intervals [c_k, c_k + 1/128), c_k = 1 + k/128, with 1/c_k and
// ln c_k stored (computed once, by IEEE division and the series above, so
// the table is the same on every machine).
struct LogTable {
  double inv[128], logc[128];
  LogTable() {
    for (int k = 0; k < 128; ++k) {
      const double c = 1.0 + k / 128.0;
      inv[k] = 1.0 / c;
      logc[k] = k == 0 ? 0.0 : log_series(c);
    }
  }
};
const LogTable g_log_table;

// Natural logarithm of a positive finite double without a division (the
// matching takes one per stored entry): x = m 2^e, m in [1, 2) falls in the
// interval k of the table, r = m / c_k - 1 in [0, 1/128) (exact for k = 0,
// so ln 1 = 0 and ln 2^e = e ln 2), and ln x = e ln 2 + ln c_k + ln(1 + r)
// with ln(1 + r) = r - r^2/2 + ... + r^9/9 (first omitted term below
// 1e-20).  Error a few units in the last place; the matching only needs one
// consistent logarithm, and nothing here depends on the host's libm.
inline double log_pos(double x) {
  uint64_t b;
  std::memcpy(&b, &x, sizeof(b));
  const int ef = (int)((b >> 52) & 0x7ff);
  if (ef == 0 || ef == 0x7ff) return std::log(x);  // subnormal, inf, nan
  const int k = (int)((b >> 45) & 127);            // top 7 bits of the mantissa
  const uint64_t mb = (b & 0x000fffffffffffffull) | 0x3ff0000000000000ull;
  double m;
  std::memcpy(&m, &mb, sizeof(m));
  const double r = k == 0 ? m - 1.0 : m * g_log_table.inv[k] - 1.0;
  double t = 1.0 / 9.0;
  t = t * r - 1.0 / 8.0;
  t = t * r + 1.0 / 7.0;
  t = t * r - 1.0 / 6.0;
  t = t * r + 1.0 / 5.0;
  t = t * r - 1.0 / 4.0;
  t = t * r + 1.0 / 3.0;
  t = t * r - 1.0 / 2.0;
  t = t * r + 1.0;
  return (double)(ef - 1023) * 0.6931471805599453 + (g_log_table.logc[k] + r * t);
}

}  // namespace

void log_table_data(const double** inv, const double** logc) {
  *inv = g_log_table.inv;
  *logc = g_log_table.logc;
}

// ---------------------------------------------------------------------------
// Section 5.1: maximise prod_i |a_{sigma(i) i}| <=> minimise sum c_{sigma(i) i}
// with c_ij = log a_i - log |a_ij|, a_i = max_j |a_ij|.  Sparse Kuhn–Munkres:
// a zero-reduced-cost greedy start, then one Dijkstra shortest augmenting
// path per unmatched row over reduced costs c_ij - u_i - v_j >= 0.
// ---------------------------------------------------------------------------
int max_product_matching(const SymCsr& A, std::vector<int>& match_col, std::vector<double>& u,
                         std::vector<double>& v, std::vector<double>& rowmax, MatchWork* work) {
  MatchWork local;
  MatchWork& mw = work ? *work : local;
  const int n = A.n;
  static const bool verbose = std::getenv("AJD_MATCH_VERBOSE") != nullptr;
  const auto t_begin = Clock::now();
  rowmax.assign(n, 0.0);
  std::vector<double> logmax(n);
  const bool known = mw.rowmax_in.size() == (size_t)n;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double r = 0.0;
    if (known) {
      r = mw.rowmax_in[i];
    } else {
      for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) r = std::max(r, std::fabs(A.val[p]));
    }
    if (r == 0.0) r = 1.0;
    rowmax[i] = r;
    logmax[i] = log_pos(r);
  }
  // log|a| of every stored entry (-inf for explicit zeros); the cost of
  // entry p in row i is c_i,col[p] = logmax[i] - loga[p] (+inf for zeros),
  // formed where it is used rather than stored.  v_j = min_i c_ij: by
  // symmetry column j's entries are row j's entries, with the cost taken in
  // the row of the other index, so v comes out of the same pass.  When the
  // logarithms and the initial potentials come with the matrix (loga_in,
  // u_in, v_in: formed on the GPU with the same logarithm and the same exact
  // minima), this pass is skipped.
  const bool given = known && mw.loga_in && mw.u_in.size() == (size_t)n && mw.v_in.size() == (size_t)n &&
                     mw.loga.size() == A.val.size();
  mw.loga_in = false;
  dvec<double>& loga = mw.loga;
  auto entry_log = [&](int64_t p) {
    const double a = std::fabs(A.val[p]);
    return a > 0.0 ? log_pos(a) : -kInf;
  };
  auto cost = [&](int i, int64_t p) { return logmax[i] - loga[p]; };
  if (given) {
    u.swap(mw.u_in);
    v.swap(mw.v_in);
    mw.u_in.clear();
    mw.v_in.clear();
  } else {
    resize_discard(loga, A.val.size());  // filled (first touched) in parallel below
    v.assign(n, kInf);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j) {
      double best = kInf;
      for (int64_t p = A.ptr[j]; p < A.ptr[j + 1]; ++p) {
        const double la = entry_log(p);
        loga[p] = la;
        if (la > -kInf) best = std::min(best, logmax[A.col[p]] - la);
      }
      v[j] = best == kInf ? 0.0 : best;
    }
    u.assign(n, kInf);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
      double best = kInf;
      for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
        const double c = cost(i, p);
        if (c < kInf) best = std::min(best, c - v[A.col[p]]);
      }
      u[i] = best == kInf ? 0.0 : best;
    }
  }
  const double ms_duals = ms_since(t_begin);
  match_col.assign(n, -1);
  std::vector<int> match_row(n, -1);
  // greedy start on zero reduced costs: first every row whose diagonal has
  // zero reduced cost takes it (rows are independent: no conflicts), then
  // the other rows take a free zero-reduced-cost column in row order
  auto zero_rc = [&](int i, int64_t p) {
    const int j = A.col[p];
    const double c = cost(i, p);
    return c < kInf && c - u[i] - v[j] <= 1e-13 * (1.0 + std::fabs(u[i]) + std::fabs(v[j]));
  };
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    // rows are sorted by column: the diagonal by binary search
    const int* b = A.col.data() + A.ptr[i];
    const int* e = A.col.data() + A.ptr[i + 1];
    const int* d = std::lower_bound(b, e, i);
    if (d != e && *d == i && zero_rc(i, d - A.col.data())) {
      match_row[i] = i;
      match_col[i] = i;
    }
  }
  {
    // rounds: every open row proposes its first free zero-reduced-cost
    // column (in parallel); in row order a proposal wins if its column is
    // still free; the losers propose again; rows without a proposal stop
    std::vector<int> todo;
    for (int i = 0; i < n; ++i)
      if (match_row[i] < 0) todo.push_back(i);
    std::vector<int> prop, next;
    while (!todo.empty()) {
      prop.assign(todo.size(), -1);
#pragma omp parallel for schedule(dynamic, 256)
      for (size_t t = 0; t < todo.size(); ++t) {
        const int i = todo[t];
        for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p)
          if (match_col[A.col[p]] < 0 && zero_rc(i, p)) {
            prop[t] = A.col[p];
            break;
          }
      }
      next.clear();
      for (size_t t = 0; t < todo.size(); ++t) {
        const int j = prop[t];
        if (j < 0) continue;
        if (match_col[j] < 0) {
          match_row[todo[t]] = j;
          match_col[j] = todo[t];
        } else {
          next.push_back(todo[t]);
        }
      }
      todo.swap(next);
    }
  }
  // shortest augmenting paths (Dijkstra over reduced costs), run in batches:
  // the searches of a batch run in parallel on the same state; then, in row
  // order, a search is applied if nothing it read (its tree rows and every
  // column it touched) was written by a search applied before it in this
  // batch, and is otherwise run again in the next batch.  Batches depend
  // only on the row order and size, not on the thread count.
  struct Search {
    int s = -1, sink = -1;
    double D = 0.0;
    std::vector<int> touched, scanned, tree_rows, path;  // path: (row, col) pairs from the sink back
    std::vector<int> read;  // columns read but never given a distance (beyond the best sink)
    std::vector<double> tree_d, scanned_d;
  };
  using Work = MatchWork::Search;
  const int nthreads = std::max(1, omp_get_max_threads());
  if ((int)mw.threads.size() < nthreads) mw.threads.resize(nthreads);
  std::vector<Work>& tw = mw.threads;
  auto search = [&](Work& W, Search& R) {
    if (W.dist.size() < (size_t)n) {  // grown entries start at rest
      W.dist.resize(n, kInf);
      W.pred.resize(n, -1);
      W.done.resize(n, 0);
    }
    // min-heap of (distance, column) with lazy deletion, kept in the
    // thread's scratch so that searches do not allocate
    using Item = std::pair<double, int>;
    std::vector<Item>& heap = W.heap;
    heap.clear();
    const std::greater<Item> later;
    R.touched.clear();
    R.scanned.clear();
    R.tree_rows.clear();
    R.tree_d.clear();
    R.scanned_d.clear();
    R.path.clear();
    R.read.clear();
    R.sink = -1;
    int i = R.s;
    double di = 0.0;
    R.tree_rows.push_back(i);
    R.tree_d.push_back(0.0);
    // Columns leave the heap in (distance, index) order and the search ends
    // at the first free column to leave it.  A free column is therefore
    // kept aside as the best sink found so far (lsap, isap) instead of
    // being pushed, and a column that would leave after it is never pushed:
    // the same path and the same scanned columns as a search that pushes
    // everything, with a heap a fraction of the size.  Such columns were
    // still read; they are listed for the batch's conflict test.
    double lsap = kInf;
    int isap = -1;
    auto after_sink = [&](double d, int j) { return d > lsap || (d == lsap && j > isap); };
    for (;;) {
      for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
        const int j = A.col[p];
        const double c = cost(i, p);
        if (W.done[j] || c == kInf) continue;
        const double nd = di + std::max(0.0, c - u[i] - v[j]);
        if (isap >= 0 && after_sink(nd, j)) {
          if (W.dist[j] == kInf) R.read.push_back(j);
          continue;
        }
        if (nd < W.dist[j]) {
          if (W.dist[j] == kInf) R.touched.push_back(j);
          W.dist[j] = nd;
          W.pred[j] = i;
          if (match_col[j] < 0) {
            lsap = nd;
            isap = j;
          } else {
            heap.push_back({nd, j});
            std::push_heap(heap.begin(), heap.end(), later);
          }
        }
      }
      int jmin = -1;
      while (!heap.empty()) {
        const Item top = heap.front();
        if (isap >= 0 && after_sink(top.first, top.second)) break;
        std::pop_heap(heap.begin(), heap.end(), later);
        heap.pop_back();
        if (!W.done[top.second] && top.first == W.dist[top.second]) {
          jmin = top.second;
          break;
        }
      }
      if (jmin < 0) {
        if (isap >= 0) {  // the best free column leaves the heap next
          W.done[isap] = 1;
          R.scanned.push_back(isap);
          R.scanned_d.push_back(lsap);
          R.sink = isap;
        }
        break;  // else no augmenting path from s
      }
      W.done[jmin] = 1;
      R.scanned.push_back(jmin);
      R.scanned_d.push_back(W.dist[jmin]);
      i = match_col[jmin];
      di = W.dist[jmin];
      R.tree_rows.push_back(i);
      R.tree_d.push_back(di);
    }
    if (R.sink >= 0) {
      R.D = W.dist[R.sink];
      for (int j = R.sink;;) {  // alternating path back to s
        const int r = W.pred[j];
        R.path.push_back(r);
        R.path.push_back(j);
        if (r == R.s) break;
        j = match_row[r];
      }
    }
    for (int j : R.touched) {
      W.dist[j] = kInf;
      W.pred[j] = -1;
      W.done[j] = 0;
    }
  };
  const double ms_greedy = ms_since(t_begin) - ms_duals;
  std::vector<int> open;
  for (int i = 0; i < n; ++i)
    if (match_row[i] < 0) open.push_back(i);
  int64_t n_searches = 0, n_scanned = 0;
  int n_batches = 0;
  double ms_par = 0.0;
  int unmatched = 0;
  std::vector<int> wrow(n, -1), wcol(n, -1);  // batch that last wrote a row / column
  std::vector<Search> batch;
  std::vector<int> retry;
  const size_t K = (size_t)std::max(8, std::min(1024, n / 2000));
  int epoch = 0;
  size_t head = 0;
  while (head < open.size() || !retry.empty()) {
    // next batch: rows to run again first, then fresh rows
    std::vector<int> rows;
    rows.swap(retry);
    while (rows.size() < K && head < open.size()) rows.push_back(open[head++]);
    batch.resize(rows.size());
    const auto t_par = Clock::now();
#pragma omp parallel for schedule(dynamic, 1)
    for (size_t t = 0; t < rows.size(); ++t) {
      batch[t].s = rows[t];
      search(tw[omp_get_thread_num()], batch[t]);
    }
    ++epoch;
    if (verbose) ms_par += ms_since(t_par);
    if (verbose) {
      ++n_batches;
      n_searches += (int64_t)rows.size();
      for (size_t t = 0; t < rows.size(); ++t) n_scanned += (int64_t)batch[t].scanned.size();
    }
    for (size_t t = 0; t < rows.size(); ++t) {
      Search& R = batch[t];
      bool clash = false;
      for (int r : R.tree_rows) clash = clash || wrow[r] == epoch;
      for (int j : R.touched) clash = clash || wcol[j] == epoch;
      for (int j : R.read) clash = clash || wcol[j] == epoch;
      if (clash) {
        retry.push_back(R.s);
        continue;
      }
      if (R.sink < 0) {
        ++unmatched;
        continue;
      }
      for (size_t q = 0; q < R.tree_rows.size(); ++q) {
        u[R.tree_rows[q]] += R.D - R.tree_d[q];
        wrow[R.tree_rows[q]] = epoch;
      }
      for (size_t q = 0; q < R.scanned.size(); ++q) {
        v[R.scanned[q]] += R.scanned_d[q] - R.D;
        wcol[R.scanned[q]] = epoch;
      }
      for (size_t q = 0; q < R.path.size(); q += 2) {
        match_row[R.path[q]] = R.path[q + 1];
        match_col[R.path[q + 1]] = R.path[q];
      }
    }
  }
  if (verbose)
    std::fprintf(stderr,
                 "  matching n=%d nnz=%lld: duals %.1f greedy %.1f searches %.1f ms (%zu open rows, %lld searches "
                 "in %d batches, %lld columns scanned, parallel part %.1f ms)\n",
                 n, (long long)A.ptr[n], ms_duals, ms_greedy, ms_since(t_begin) - ms_duals - ms_greedy, open.size(),
                 (long long)n_searches, n_batches, (long long)n_scanned, ms_par);
  if (unmatched) {
    // structurally singular: pair the leftover rows and columns in index
    // order and give them neutral duals (scaling then reduces to 1/sqrt(a_i))
    std::vector<int> fr, fc;
    for (int i = 0; i < n; ++i)
      if (match_row[i] < 0) fr.push_back(i);
    for (int j = 0; j < n; ++j)
      if (match_col[j] < 0) fc.push_back(j);
    for (size_t t = 0; t < fr.size() && t < fc.size(); ++t) {
      match_col[fc[t]] = fr[t];
      u[fr[t]] = 0.0;
      v[fc[t]] = 0.0;
    }
  }
  return unmatched;
}

// ---------------------------------------------------------------------------
// Section 5.2: split the cycles of j -> match_col[j] into 2-cycles and at most
// one 1-cycle per odd cycle.  Consecutive cycle members always share a
// matched entry, so every 2x2 block contains one.  Readings: an even cycle
// takes whichever of its two splits has the larger product of |off-diagonal|
// entries (ties: fewer nonzeros in the merged rows, then the split that
// starts at the cycle's first member); an odd cycle keeps as 1x1 the member
// with the largest |diagonal| (ties: lowest index).
// ---------------------------------------------------------------------------
void split_cycles(const SymCsr& S, const std::vector<int>& match_col,
                  std::vector<std::pair<int, int>>& groups) {
  const int n = S.n;
  groups.clear();
  auto union_nnz = [&](int a, int b) {
    int64_t pa = S.ptr[a], pb = S.ptr[b], cnt = 0;
    while (pa < S.ptr[a + 1] || pb < S.ptr[b + 1]) {
      if (pb >= S.ptr[b + 1] || (pa < S.ptr[a + 1] && S.col[pa] < S.col[pb])) ++pa;
      else if (pa >= S.ptr[a + 1] || S.col[pb] < S.col[pa]) ++pb;
      else { ++pa; ++pb; }
      ++cnt;
    }
    return cnt;
  };
  // the groups of one cycle (members in cycle order, starting at its
  // smallest index), appended to `out`
  auto split = [&](const std::vector<int>& cyc, std::vector<std::pair<int, int>>& out) {
    const int len = (int)cyc.size();
    if (len == 1) {
      out.push_back({cyc[0], -1});
    } else if (len == 2) {
      out.push_back({std::min(cyc[0], cyc[1]), std::max(cyc[0], cyc[1])});
    } else if (len % 2 == 0) {
      double score[2] = {0.0, 0.0};
      int64_t nnz[2] = {0, 0};
      for (int opt = 0; opt < 2; ++opt)
        for (int k = opt; k < len + opt; k += 2) {
          const int a = cyc[k % len], b = cyc[(k + 1) % len];
          score[opt] += std::log(std::fabs(lookup(S, a, b)) + 1e-300);
          nnz[opt] += union_nnz(a, b);
        }
      int opt = 0;
      if (score[1] > score[0] || (score[1] == score[0] && nnz[1] < nnz[0])) opt = 1;
      for (int k = opt; k < len + opt; k += 2) {
        const int a = cyc[k % len], b = cyc[(k + 1) % len];
        out.push_back({std::min(a, b), std::max(a, b)});
      }
    } else {
      int t = 0;
      for (int k = 1; k < len; ++k) {
        const double dk = std::fabs(lookup(S, cyc[k], cyc[k])), dt = std::fabs(lookup(S, cyc[t], cyc[t]));
        if (dk > dt || (dk == dt && cyc[k] < cyc[t])) t = k;
      }
      out.push_back({cyc[t], -1});
      for (int k = 1; k < len; k += 2) {
        const int a = cyc[(t + k) % len], b = cyc[(t + k + 1) % len];
        out.push_back({std::min(a, b), std::max(a, b)});
      }
    }
  };
  std::vector<char> seen(n, 0);
  std::vector<int> cyc;
  bool perm = true;
  for (int j = 0; j < n && perm; ++j) perm = match_col[j] >= 0;
  if (!perm) {
    // a partial matching (chains as well as cycles): one walk per unseen
    // index, in index order
    for (int j0 = 0; j0 < n; ++j0) {
      if (seen[j0]) continue;
      cyc.clear();
      int j = j0;
      do {
        seen[j] = 1;
        cyc.push_back(j);
        j = match_col[j];
      } while (j != j0 && j >= 0 && !seen[j]);
      split(cyc, groups);
    }
    return;
  }
  // a permutation: every cycle is emitted at its smallest member, in index
  // order.  Fixed points and 2-cycles (nearly all of them) are placed in
  // parallel; longer cycles are walked in index order and their groups
  // copied into place.
  std::vector<int> ng(n + 1, 0);  // groups emitted at index j, then offsets
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j) {
    const int k = match_col[j];
    if (k == j) ng[j + 1] = 1;
    else if (match_col[k] == j) ng[j + 1] = j < k ? 1 : 0;
    else ng[j + 1] = -1;  // in a longer cycle
  }
  std::vector<std::pair<int, int>> longg;          // groups of the longer cycles
  std::vector<std::pair<int, int64_t>> longat;     // (leader, first group in longg)
  for (int j0 = 0; j0 < n; ++j0) {
    if (ng[j0 + 1] >= 0 || seen[j0]) continue;
    cyc.clear();
    int j = j0;
    do {
      seen[j] = 1;
      cyc.push_back(j);
      j = match_col[j];
    } while (j != j0);
    const size_t before = longg.size();
    split(cyc, longg);
    longat.push_back({j0, (int64_t)before});
    for (size_t q = 1; q < cyc.size(); ++q) ng[cyc[q] + 1] = 0;
    ng[j0 + 1] = (int)(longg.size() - before);
  }
  for (int j = 0; j < n; ++j) ng[j + 1] += ng[j];
  groups.resize(ng[n]);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j) {
    const int k = match_col[j];
    if (k == j) groups[ng[j]] = {j, -1};
    else if (match_col[k] == j && j < k) groups[ng[j]] = {j, k};
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (size_t c = 0; c < longat.size(); ++c) {
    const int j0 = longat[c].first;
    const int64_t from = longat[c].second;
    for (int q = 0; q < ng[j0 + 1] - ng[j0]; ++q) groups[ng[j0] + q] = longg[from + q];
  }
}

namespace {

struct Cand {
  int a, b;   // nodes (b = -1 for 1x1)
  double q;   // max column 1-norm of the would-be L block
};

struct Trip {
  int r, c;   // original indices
  double v;
};

// Stable parallel bucket scatter: items 0..N-1, taken in order, go to the
// buckets key(i) in [0, nb) so that every bucket keeps its items in item
// order.  The items are cut into contiguous chunks; per-chunk counts give
// every (chunk, bucket) pair its own run of slots.  On return ptr holds the
// nb + 1 bucket offsets and emit(i, slot) has been called once per item.
template <class Key, class Emit>
void stable_scatter(int64_t N, int nb, Key key, std::vector<int64_t>& ptr, Emit emit) {
  const int T = (int)std::max<int64_t>(1, std::min<int64_t>(omp_get_max_threads(), N / 16384));
  std::vector<unsigned> cnt((size_t)T * nb, 0u);
#pragma omp parallel for schedule(static)
  for (int t = 0; t < T; ++t) {
    unsigned* c = cnt.data() + (size_t)t * nb;
    for (int64_t i = N * t / T; i < N * (t + 1) / T; ++i) ++c[key(i)];
  }
  ptr.assign((size_t)nb + 1, 0);
#pragma omp parallel for schedule(static)
  for (int b = 0; b < nb; ++b) {
    unsigned run = 0;  // offsets within the bucket, by chunk
    for (int t = 0; t < T; ++t) {
      const unsigned c = cnt[(size_t)t * nb + b];
      cnt[(size_t)t * nb + b] = run;
      run += c;
    }
    ptr[(size_t)b + 1] = run;
  }
  for (int b = 0; b < nb; ++b) ptr[(size_t)b + 1] += ptr[b];
#pragma omp parallel for schedule(static)
  for (int t = 0; t < T; ++t) {
    unsigned* c = cnt.data() + (size_t)t * nb;
    for (int64_t i = N * t / T; i < N * (t + 1) / T; ++i) {
      const int b = key(i);
      emit(i, ptr[b] + c[b]++);
    }
  }
}

// Stable placement of items into the rows of a CSR array, in two passes
// that keep the writes inside the cache.  produce(g, f) calls f(item) for
// the items of group g (g = 0..G-1, each group a contiguous run of the item
// order); item.r is the destination row in [0, nr), item.c and item.v the
// stored column and value.  On return row r holds its items in item order
// at ptr[r] .. ptr[r + 1] of (col, val), whatever G is.  Pass 1 moves the
// items, group by group, into buckets of 256 consecutive rows (few write
// streams); pass 2 places each bucket's items into its rows.
template <class Produce, class ColOut, class ValOut>
void stable_place(int G, int nr, Produce produce, std::vector<int64_t>& ptr, dvec<Trip>& tmp, ColOut& col,
                  ValOut& val) {
  constexpr int kShift = 8;
  const int nblk = (nr >> kShift) + 1;
  dvec<unsigned> cnt((size_t)G * nr);  // each group zeroes its own counts
#pragma omp parallel for schedule(static)
  for (int g = 0; g < G; ++g) {
    unsigned* c = cnt.data() + (size_t)g * nr;
    std::fill(c, c + nr, 0u);
    produce(g, [&](const Trip& t) { ++c[t.r]; });
  }
  std::vector<int64_t> boff((size_t)G * nblk), bptr(nblk + 1, 0);
  ptr.assign((size_t)nr + 1, 0);
#pragma omp parallel for schedule(static)
  for (int b = 0; b < nblk; ++b) {
    const int r0 = b << kShift, r1 = std::min(nr, r0 + (1 << kShift));
    int64_t run = 0;
    for (int g = 0; g < G; ++g) {
      boff[(size_t)g * nblk + b] = run;
      for (int r = r0; r < r1; ++r) run += cnt[(size_t)g * nr + r];
    }
    for (int r = r0; r < r1; ++r) {
      int64_t k = 0;
      for (int g = 0; g < G; ++g) k += cnt[(size_t)g * nr + r];
      ptr[(size_t)r + 1] = k;
    }
    bptr[b + 1] = run;
  }
  for (int r = 0; r < nr; ++r) ptr[(size_t)r + 1] += ptr[r];
  for (int b = 0; b < nblk; ++b) bptr[b + 1] += bptr[b];
  resize_discard(tmp, bptr[nblk]);
  resize_discard(col, ptr[nr]);
  resize_discard(val, ptr[nr]);
#pragma omp parallel for schedule(static)
  for (int g = 0; g < G; ++g) {
    int64_t* bo = boff.data() + (size_t)g * nblk;
    for (int b = 0; b < nblk; ++b) bo[b] += bptr[b];
    produce(g, [&](const Trip& t) { tmp[bo[t.r >> kShift]++] = t; });
  }
#pragma omp parallel for schedule(dynamic, 16)
  for (int b = 0; b < nblk; ++b) {
    const int r0 = b << kShift, r1 = std::min(nr, r0 + (1 << kShift));
    int64_t next[1 << kShift];
    for (int r = r0; r < r1; ++r) next[r - r0] = ptr[r];
    for (int64_t q = bptr[b]; q < bptr[b + 1]; ++q) {
      const Trip& t = tmp[q];
      const int64_t slot = next[t.r - r0]++;
      col[slot] = t.c;
      val[slot] = t.v;
    }
  }
}

// Gauss–Jordan inverse with partial pivoting (row-major, in place on a copy).
bool dense_inverse(int m, dvec<double>& M, dvec<double>& inv) {
  inv.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) inv[(size_t)i * m + i] = 1.0;
  for (int c = 0; c < m; ++c) {
    int piv = c;
    double best = std::fabs(M[(size_t)c * m + c]);
    for (int r = c + 1; r < m; ++r) {
      const double a = std::fabs(M[(size_t)r * m + c]);
      if (a > best) { best = a; piv = r; }
    }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    if (piv != c) {
      for (int k = 0; k < m; ++k) {
        std::swap(M[(size_t)c * m + k], M[(size_t)piv * m + k]);
        std::swap(inv[(size_t)c * m + k], inv[(size_t)piv * m + k]);
      }
    }
    const double d = 1.0 / M[(size_t)c * m + c];
    double* Mc = &M[(size_t)c * m];
    double* Ic = &inv[(size_t)c * m];
    for (int k = 0; k < m; ++k) { Mc[k] *= d; Ic[k] *= d; }
#pragma omp parallel for schedule(static)
    for (int r = 0; r < m; ++r) {
      if (r == c) continue;
      const double f = M[(size_t)r * m + c];
      if (f == 0.0) continue;
      double* Mr = &M[(size_t)r * m];
      double* Ir = &inv[(size_t)r * m];
      for (int k = c; k < m; ++k) Mr[k] -= f * Mc[k];
      for (int k = 0; k < m; ++k) Ir[k] -= f * Ic[k];
    }
  }
  // symmetrise (the exact inverse of a symmetric matrix is symmetric)
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) {
      const double s = 0.5 * (inv[(size_t)i * m + j] + inv[(size_t)j * m + i]);
      inv[(size_t)i * m + j] = inv[(size_t)j * m + i] = s;
    }
  return true;
}

}  // namespace

// Dense tail: n/16 clamped to 1000..3000 rows.  Its Gauss-Jordan inversion
// costs O(n_dense^3) binary64 work on a GPU whose FP64 pipe is narrow (0.14 s
// at 2946 rows in the blocked form), while the extra sparse levels that a
// smaller tail leaves cost little in the dataflow apply; the bound keeps the
// inversion short when setups share the device with solves.
int default_n_dense(int64_t n) { return (int)std::max<int64_t>(1000, std::min<int64_t>(3000, n / 16)); }

double default_gamma(int64_t n, bool offdiag) {
  // weak-coupling threshold of the independent sets; by default it shrinks
  // with the drop tolerance (measured: a fixed 0.02 loses the preconditioner
  // at n = 10^6 while 5/sqrt(n) keeps it).  Off-diagonal disorder (Section
  // 7) loses more by ignoring weak couplings: 1/sqrt(n) there.
  const double rn = std::sqrt((double)std::max<int64_t>(n, 1));
  return std::min(0.02, (offdiag ? 1.0 : 5.0) / rn);
}

int build_ildl(const SymCsr& A, const ildl_params& prm, HostFactor& F, bool dense_on_host, SchurEngine* engine) {
  const auto t_start = Clock::now();
  const int n = A.n;
  if (n <= 0) return fail(JD_EINVAL, "ildl: empty matrix");
  const double kappa = prm.kappa > 1.0 ? prm.kappa : 5.0;
  const double eps_drop = prm.drop < 0.0 ? 1.0 / std::sqrt((double)n) : prm.drop;
  const double tau = eps_drop / kappa;
  const double agg_tau = prm.aggressive > 0.0 ? prm.aggressive : 0.0;  // Section 6.3, 0 = off

  const double gamma = prm.gamma < 0.0 ? default_gamma(n, false) : prm.gamma;
  const int max_levels = prm.max_levels > 0 ? prm.max_levels : 64;
  const int n_dense = prm.n_dense > 0 ? prm.n_dense : default_n_dense(n);
  constexpr int kDenseHardMax = 8000;

  F = HostFactor();
  F.n = n;
  F.nnz_A = (int64_t)A.col.size();

  SymCsr S = A;
  std::vector<int> gid(n);
  std::iota(gid.begin(), gid.end(), 0);
  std::vector<double> cum(n, 1.0);

  std::vector<int> order;          // original ids in elimination order
  order.reserve(n);
  std::vector<int> level_ptr{0};
  std::vector<double> dd(n, 0.0), dof(n, 0.0);
  std::vector<int> part(n, -1);    // partner original id
  std::vector<double> sc(n, 1.0);  // final scaling of each original node
  // entries of L as (row, column, value) in original numbering, appended
  // level by level; room for a typical fill is reserved up front (pages are
  // only touched when written) so that growing it rarely copies
  dvec<Trip> trips;
  trips.reserve((size_t)n * 64);
  double t_match = 0.0;

  // per-level scratch kept across levels: the levels shrink, so after the
  // first few every buffer is reused from memory that is already mapped
  // (fresh large blocks would fault in every page again at every level)
  MatchWork mwork;
  SymCsr Snext;                                      // next level's S
  dvec<int> lnode;                                   // L_F: B node (local index)
  dvec<double> lval;
  dvec<int> agg_node;                                // L_F after aggressive dropping
  dvec<double> agg_val;
  std::vector<std::vector<int>> ucol;                // per-chunk row output
  std::vector<std::vector<double>> uval;
  dvec<int> rec_row, rec_blk, crow;                  // Schur records
  dvec<double> rec_a, rec_b, c1, c2;
  dvec<int64_t> rec_slot;
  dvec<unsigned> mirror_cnt;
  dvec<Trip> mirror_tmp;                             // lower entries bucketed by column block
  struct RowWork {                                   // per thread; accv and mark all zero at rest
    std::vector<double> accv;
    std::vector<char> mark;
    std::unique_ptr<int[]> cols;                      // uninitialised
    int cap = 0;
  };
  std::vector<RowWork> rwork(std::max(1, omp_get_max_threads()));

  const bool verbose = std::getenv("AJD_SETUP_VERBOSE") != nullptr;
  if (engine) {
    const int erc = engine->begin(S);
    if (erc != JD_OK) return erc;
  }
  int level = 0;
  for (;; ++level) {
    const auto t_level = Clock::now();
    const int m = S.n;
    if (m == 0) break;
    if (m <= n_dense || (level >= max_levels && m <= kDenseHardMax)) break;
    if (level >= 4 * max_levels) return fail(JD_ESETUP, "ildl: %d rows left after %d levels", m, level);

    // 1-2. matching, scaling, candidate groups
    auto tm = Clock::now();
    std::vector<int> mc;
    std::vector<double> u, v, rmax;
    std::vector<double> d(m);
    std::vector<std::pair<int, int>> groups;
    const bool use_matching = prm.matching != 0 && (prm.matching < 0 || level < prm.matching);
    if (use_matching) {
      max_product_matching(S, mc, u, v, rmax, &mwork);
#pragma omp parallel for schedule(static)
      for (int i = 0; i < m; ++i) d[i] = std::sqrt(std::exp(u[i] + v[i]) / rmax[i]);
      if (level == 0)
        for (int j = 0; j < m; ++j) F.n_matched_offdiag += (mc[j] != j);
    } else {
      for (int i = 0; i < m; ++i) {
        double r = 0.0;
        for (int64_t p = S.ptr[i]; p < S.ptr[i + 1]; ++p) r = std::max(r, std::fabs(S.val[p]));
        d[i] = r > 0.0 ? 1.0 / std::sqrt(r) : 1.0;
      }
    }
    // scale, and in the same pass collect what the candidates need:
    // d1 = sum_{k != i} |s_ki| / |s_ii| (the 1-norm of the would-be L column)
    std::vector<double> diag(m), offsum(m);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) {
      cum[i] *= d[i];
      double o = 0.0, dg = 0.0;
      for (int64_t p = S.ptr[i]; p < S.ptr[i + 1]; ++p) {
        const int c = S.col[p];
        const double sv = S.val[p] * (d[i] * d[c]);
        S.val[p] = sv;
        if (c == i) dg = sv;
        else o += std::fabs(sv);
      }
      diag[i] = dg;
      offsum[i] = o;
    }
    if (engine) {
      const int erc = engine->scale(d.data(), m);
      if (erc != JD_OK) return erc;
    }
    if (use_matching) {
      split_cycles(S, mc, groups);
    } else {
      groups.reserve(m);
      for (int i = 0; i < m; ++i) groups.push_back({i, -1});
    }
    const double tm_ms = ms_since(tm);
    t_match += tm_ms;
    const auto t_cand = Clock::now();

    // 3. candidates: d1 from the scaling pass above; d2 = sum_k
    // ||(s_ki, s_kj) B^{-1}||_1 for a 2x2 block
    auto d1_of = [&](int i) { return diag[i] != 0.0 ? offsum[i] / std::fabs(diag[i]) : kInf; };
    // one or two candidates per group, computed in parallel and compacted in
    // group order (the same list a sequential pass produces)
    const int ng = (int)groups.size();
    std::vector<Cand> g1(ng), g2(ng);
    std::vector<char> gcount(ng, 1);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int gi = 0; gi < ng; ++gi) {
      const auto& g = groups[gi];
      if (g.second < 0) {
        g1[gi] = {g.first, -1, d1_of(g.first)};
        continue;
      }
      const int i = g.first, j = g.second;
      const double sij = 0.5 * (lookup(S, i, j) + lookup(S, j, i));
      const double a = diag[i], c = diag[j];
      const double det = a * c - sij * sij;
      const double d1 = std::min(d1_of(i), d1_of(j));
      bool use2 = false;
      double q2 = kInf;
      if (std::fabs(det) > 1e-300 && std::isfinite(det)) {
        const double i00 = c / det, i01 = -sij / det, i11 = a / det;
        double cs1 = 0.0, cs2 = 0.0, d2 = 0.0;
        int64_t pa = S.ptr[i], pb = S.ptr[j];
        const int64_t ea = S.ptr[i + 1], eb = S.ptr[j + 1];
        while (pa < ea || pb < eb) {
          int k;
          double ski = 0.0, skj = 0.0;
          if (pb >= eb || (pa < ea && S.col[pa] < S.col[pb])) { k = S.col[pa]; ski = S.val[pa++]; }
          else if (pa >= ea || S.col[pb] < S.col[pa]) { k = S.col[pb]; skj = S.val[pb++]; }
          else { k = S.col[pa]; ski = S.val[pa++]; skj = S.val[pb++]; }
          if (k == i || k == j) continue;
          const double r1 = ski * i00 + skj * i01, r2 = ski * i01 + skj * i11;
          cs1 += std::fabs(r1);
          cs2 += std::fabs(r2);
          d2 += std::fabs(r1) + std::fabs(r2);
          // the terms are non-negative: once d2 reaches d1 the block is not
          // taken, whatever follows (same outcome as the full sum)
          if (!(d2 < d1)) break;
        }
        if (d2 < d1) {  // Section 6.2: 2x2 update only if d2 < d1
          use2 = true;
          q2 = std::max(cs1, cs2);
        }
      }
      if (use2) {
        g1[gi] = {i, j, q2};
      } else {
        g1[gi] = {i, -1, d1_of(i)};
        g2[gi] = {j, -1, d1_of(j)};
        gcount[gi] = 2;
      }
    }
    const double tc_groups = ms_since(t_cand);
    std::vector<Cand> cands;
    cands.reserve(m);
    for (int gi = 0; gi < ng; ++gi) {
      cands.push_back(g1[gi]);
      if (gcount[gi] == 2) cands.push_back(g2[gi]);
    }
    __gnu_parallel::stable_sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) {
      if (x.q != y.q) return x.q < y.q;
      return x.a < y.a;
    });

    const double tc_sort = ms_since(t_cand) - tc_groups;
    // 4. independent set of pivots, best first; inverse-based acceptance
    // 1 + q <= kappa (||L^{-1}||_1 of this level)
    std::vector<char> blocked(m, 0), inB(m, 0);
    std::vector<int> acc;  // indices into cands
    auto block_nbrs = [&](int x) {
      blocked[x] = 1;
      for (int64_t p = S.ptr[x]; p < S.ptr[x + 1]; ++p) blocked[S.col[p]] |= (char)(std::fabs(S.val[p]) > gamma);
    };
    auto try_accept = [&](double qmax) {
      for (size_t t = 0; t < cands.size(); ++t) {
        const Cand& cd = cands[t];
        if (!(cd.q <= qmax)) break;
        if (blocked[cd.a] || (cd.b >= 0 && blocked[cd.b])) continue;
        acc.push_back((int)t);
        inB[cd.a] = 1;
        if (cd.b >= 0) inB[cd.b] = 1;
        block_nbrs(cd.a);
        if (cd.b >= 0) block_nbrs(cd.b);
      }
    };
    try_accept(kappa - 1.0);
    if ((int64_t)acc.size() * 200 < m && m > n_dense) {
      // the level would stall: widen the bound on ||L^{-1}|| for this level
      // step by step (recorded as a relaxed level), never beyond 64 kappa
      ++F.n_relaxed;
      for (double f = 2.0; f <= 64.0 && (int64_t)acc.size() * 200 < m; f *= 2.0) try_accept(f * kappa - 1.0);
    }
    if (acc.empty()) return fail(JD_ESETUP, "ildl: no usable pivot at level %d (%d rows)", level, m);

    const double tc_ms = ms_since(t_cand);
    if (verbose)
      std::fprintf(stderr, "  candidates: groups %.1f sort %.1f independent set %.1f ms\n", tc_groups, tc_sort,
                   tc_ms - tc_groups - tc_sort);
    const auto t_lf = Clock::now();
    // 5. local numbering: B in accepted order, C in index order (both
    // built in parallel: block positions and C indices from prefix sums)
    const int nacc_blocks = (int)acc.size();
    std::vector<int> blk_of(m, -1), cidx(m, -1);
    std::vector<double> binv(3 * acc.size());  // symmetric 2x2 (or 1x1) inverse per block
    std::vector<double> bmat(3 * acc.size());
    const int level_start = (int)order.size();
    std::vector<int> bpos(nacc_blocks + 1, 0);  // first position of each block in the level
    for (int b = 0; b < nacc_blocks; ++b) bpos[b + 1] = bpos[b] + (cands[acc[b]].b < 0 ? 1 : 2);
    order.resize((size_t)level_start + bpos[nacc_blocks]);
    int n2 = 0;
#pragma omp parallel for schedule(static) reduction(+ : n2)
    for (int b = 0; b < nacc_blocks; ++b) {
      const Cand& cd = cands[acc[b]];
      const int o = level_start + bpos[b];
      blk_of[cd.a] = b;
      if (cd.b < 0) {
        const double piv = diag[cd.a];
        bmat[3 * b] = piv;
        binv[3 * b] = 1.0 / piv;
        binv[3 * b + 1] = binv[3 * b + 2] = 0.0;
        order[o] = gid[cd.a];
        sc[gid[cd.a]] = cum[cd.a];
        dd[gid[cd.a]] = 1.0 / piv;
        dof[gid[cd.a]] = 0.0;
        part[gid[cd.a]] = -1;
      } else {
        blk_of[cd.b] = b;
        const double a = diag[cd.a], c = diag[cd.b];
        const double s = 0.5 * (lookup(S, cd.a, cd.b) + lookup(S, cd.b, cd.a));
        const double det = a * c - s * s;
        bmat[3 * b] = a;
        bmat[3 * b + 1] = s;
        bmat[3 * b + 2] = c;
        binv[3 * b] = c / det;
        binv[3 * b + 1] = -s / det;
        binv[3 * b + 2] = a / det;
        order[o] = gid[cd.a];
        order[o + 1] = gid[cd.b];
        sc[gid[cd.a]] = cum[cd.a];
        sc[gid[cd.b]] = cum[cd.b];
        dd[gid[cd.a]] = c / det;
        dd[gid[cd.b]] = a / det;
        dof[gid[cd.a]] = dof[gid[cd.b]] = -s / det;
        part[gid[cd.a]] = gid[cd.b];
        part[gid[cd.b]] = gid[cd.a];
        ++n2;
      }
    }
    F.n_2x2 += n2;
    level_ptr.push_back((int)order.size());
    F.level_sizes.push_back((int)order.size() - level_start);
    // C nodes in index order: per-chunk counts, then each chunk numbers its own
    std::vector<int> cnodes;
    int mc_n = 0;
    {
      const int T = std::max(1, std::min(omp_get_max_threads(), m / 16384));
      std::vector<int> ccnt(T + 1, 0);
#pragma omp parallel for schedule(static)
      for (int t = 0; t < T; ++t) {
        int k = 0;
        for (int i = (int)((int64_t)m * t / T); i < (int)((int64_t)m * (t + 1) / T); ++i) k += !inB[i];
        ccnt[t + 1] = k;
      }
      for (int t = 0; t < T; ++t) ccnt[t + 1] += ccnt[t];
      mc_n = ccnt[T];
      cnodes.resize(mc_n);
#pragma omp parallel for schedule(static)
      for (int t = 0; t < T; ++t) {
        int k = ccnt[t];
        for (int i = (int)((int64_t)m * t / T); i < (int)((int64_t)m * (t + 1) / T); ++i)
          if (!inB[i]) {
            cidx[i] = k;
            cnodes[k++] = i;
          }
      }
    }

    // 6. L_F = F D_B^{-1}, dropped at tau, built from the pivot blocks' own
    // rows: S is symmetric, so row a of S holds column a of F.  Each block
    // emits (C row, node, value) for the C rows its nodes reach, blocks in
    // elimination order (node a before node b), and a stable placement by C
    // row lists every row's entries by block -- the rows that a pass over
    // all C rows gives, at the cost of the pivot rows alone.
    std::vector<int64_t> lptr;
    {
      const int nacc = (int)acc.size();
      const int G = std::max(1, std::min(omp_get_max_threads(), nacc / 256));
      auto produce = [&](int g, auto&& emit) {
        const int b0 = (int)((int64_t)nacc * g / G), b1 = (int)((int64_t)nacc * (g + 1) / G);
        for (int b = b0; b < b1; ++b) {
          const Cand& cd = cands[acc[b]];
          if (cd.b < 0) {
            for (int64_t p = S.ptr[cd.a]; p < S.ptr[cd.a + 1]; ++p) {
              const int r = cidx[S.col[p]];
              if (r < 0) continue;  // B nodes
              const double l = S.val[p] * binv[3 * b];
              if (std::fabs(l) >= tau && l != 0.0) emit(Trip{r, cd.a, l});
            }
            continue;
          }
          // 2x2: (s_ka, s_kb) for every row k that rows a and b reach
          int64_t pa = S.ptr[cd.a], pb = S.ptr[cd.b];
          const int64_t ea = S.ptr[cd.a + 1], eb = S.ptr[cd.b + 1];
          while (pa < ea || pb < eb) {
            int k;
            double fa = 0.0, fb = 0.0;
            if (pb >= eb || (pa < ea && S.col[pa] < S.col[pb])) { k = S.col[pa]; fa = S.val[pa++]; }
            else if (pa >= ea || S.col[pb] < S.col[pa]) { k = S.col[pb]; fb = S.val[pb++]; }
            else { k = S.col[pa]; fa = S.val[pa++]; fb = S.val[pb++]; }
            const int r = cidx[k];
            if (r < 0) continue;
            const double l1 = fa * binv[3 * b] + fb * binv[3 * b + 1];
            const double l2 = fa * binv[3 * b + 1] + fb * binv[3 * b + 2];
            if (std::fabs(l1) >= tau && l1 != 0.0) emit(Trip{r, cd.a, l1});
            if (std::fabs(l2) >= tau && l2 != 0.0) emit(Trip{r, cd.b, l2});
          }
        }
      };
      stable_place(G, mc_n, produce, lptr, mirror_tmp, lnode, lval);
    }
    const int nchunk = std::max(1, std::min(mc_n, 8 * omp_get_max_threads()));
    if ((int)ucol.size() < nchunk) {
      ucol.resize(nchunk);
      uval.resize(nchunk);
    }
    if (agg_tau > 0.0 && lptr[mc_n] > 0) {
      // 6b. aggressive dropping (Section 6.3): l_ij goes when |l_ij| <=
      // tau / (nu_i * #column j), nu_i = ||L_level^{-1} e_i||, which is 1 for
      // every row i of the block (the level's L is [I 0; L_F I]).  Done
      // before the Schur complement, which is then formed from the sparser
      // block.
      std::vector<int> ccount(m, 0);
#pragma omp parallel for schedule(static)
      for (int64_t p = 0; p < lptr[mc_n]; ++p) {
#pragma omp atomic
        ++ccount[lnode[p]];
      }
      std::vector<int64_t> nptr(mc_n + 1, 0);
#pragma omp parallel for schedule(static)
      for (int r = 0; r < mc_n; ++r) {
        int64_t k = 0;
        for (int64_t p = lptr[r]; p < lptr[r + 1]; ++p) k += std::fabs(lval[p]) > agg_tau / ccount[lnode[p]];
        nptr[r + 1] = k;
      }
      for (int r = 0; r < mc_n; ++r) nptr[r + 1] += nptr[r];
      resize_discard(agg_node, nptr[mc_n]);
      resize_discard(agg_val, nptr[mc_n]);
#pragma omp parallel for schedule(static)
      for (int r = 0; r < mc_n; ++r) {
        int64_t o = nptr[r];
        for (int64_t p = lptr[r]; p < lptr[r + 1]; ++p)
          if (std::fabs(lval[p]) > agg_tau / ccount[lnode[p]]) {
            agg_node[o] = lnode[p];
            agg_val[o++] = lval[p];
          }
      }
      F.n_aggressive += lptr[mc_n] - nptr[mc_n];
      lptr.swap(nptr);
      lnode.swap(agg_node);
      lval.swap(agg_val);
    }
    {
      const size_t base = trips.size();
      trips.resize(base + (size_t)lptr[mc_n]);
#pragma omp parallel for schedule(static)
      for (int r = 0; r < mc_n; ++r) {
        const int k = cnodes[r];
        for (int64_t p = lptr[r]; p < lptr[r + 1]; ++p) trips[base + p] = {gid[k], gid[lnode[p]], lval[p] / cum[k]};
      }
    }

    const double tl_ms = ms_since(t_lf);
    const auto t_schur = Clock::now();
    // 7. Schur complement S' = S_CC - L_F D_B L_F^T (upper triangle, then
    // mirrored so that S' is exactly symmetric), dropped at tau off the
    // diagonal.  Column access to L_F per B block:
    // One record per (block, C row) -- the row's L_F values for the block's
    // nodes a and b -- grouped by block with rows ascending: the entries of
    // a row are ordered by block (a block's one or two nodes adjacent), so
    // the records are the runs of equal block; built per row in parallel and
    // grouped by a stable parallel scatter.
    std::vector<int64_t> rrec(mc_n + 1, 0);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < mc_n; ++r) {
      int cnt = 0, last = -1;
      for (int64_t p = lptr[r]; p < lptr[r + 1]; ++p) {
        const int b = blk_of[lnode[p]];
        if (b != last) { ++cnt; last = b; }
      }
      rrec[r + 1] = cnt;
    }
    for (int r = 0; r < mc_n; ++r) rrec[r + 1] += rrec[r];
    const int64_t nrec = rrec[mc_n];
    resize_discard(rec_row, nrec);
    resize_discard(rec_blk, nrec);
    resize_discard(rec_a, nrec);
    resize_discard(rec_b, nrec);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < mc_n; ++r) {
      int64_t q = rrec[r] - 1;
      int last = -1;
      for (int64_t p = lptr[r]; p < lptr[r + 1]; ++p) {
        const int b = blk_of[lnode[p]];
        if (b != last) {
          ++q;
          last = b;
          rec_row[q] = r;
          rec_blk[q] = b;
          rec_a[q] = 0.0;
          rec_b[q] = 0.0;
        }
        if (lnode[p] == cands[acc[b]].a) rec_a[q] = lval[p];
        else rec_b[q] = lval[p];
      }
    }
    std::vector<int64_t> cptr;
    resize_discard(crow, nrec);
    resize_discard(c1, nrec);
    resize_discard(c2, nrec);
    resize_discard(rec_slot, nrec);  // where record i (row order) sits in its block's list
    stable_scatter(nrec, (int)acc.size(), [&](int64_t i) { return rec_blk[i]; }, cptr, [&](int64_t i, int64_t slot) {
      crow[slot] = rec_row[i];
      c1[slot] = rec_a[i];
      c2[slot] = rec_b[i];
      rec_slot[i] = slot;
    });
    const double ts_rec = ms_since(t_schur);
    double ts_num = 0.0;
    SymCsr& Sn = Snext;
    std::vector<double>& next_rowmax = mwork.rowmax_in;  // the next matching's row maxima
    if (engine) {
      // S' on the engine (the GPU), from the records above
      std::vector<char> is2(acc.size());
      for (size_t b = 0; b < acc.size(); ++b) is2[b] = cands[acc[b]].b >= 0;
      SchurLevel lv;
      lv.m = m;
      lv.mc_n = mc_n;
      lv.nblk = (int)acc.size();
      lv.sptr = S.ptr.data();
      lv.cidx = cidx.data();
      lv.cnodes = cnodes.data();
      lv.rrec = rrec.data();
      lv.rec_blk = rec_blk.data();
      lv.rec_slot = rec_slot.data();
      lv.cptr = cptr.data();
      lv.crow = crow.data();
      lv.c1 = c1.data();
      lv.c2 = c2.data();
      lv.bmat = bmat.data();
      lv.is2x2 = is2.data();
      lv.tau = tau;
      // the next level's matching potentials come with S' when it matches
      const bool next_matches = prm.matching != 0 && (prm.matching < 0 || level + 1 < prm.matching);
      const int erc = next_matches ? engine->schur(lv, Sn, next_rowmax, &mwork.u_in, &mwork.v_in, &mwork.loga)
                                   : engine->schur(lv, Sn, next_rowmax, nullptr, nullptr, nullptr);
      mwork.loga_in = next_matches && erc == JD_OK;
      if (erc != JD_OK) return erc;
      ts_num = ms_since(t_schur) - ts_rec;
    } else {
      // upper triangle of S', row by row: chunk ch holds the rows of its row
      // range in order; rowcnt[r] entries per row (diagonal included)
      std::vector<int> rowcnt(mc_n, 0);
      // a new row is typically as long as the old ones: room for about 3/4 of
      // an old row per upper row, so that the chunk buffers rarely grow
      const double upper_guess = 0.75 * (double)S.ptr[m] / m + 8.0;
      {
#pragma omp parallel
        {
          RowWork& rw = rwork[omp_get_thread_num()];
          if (rw.cap < mc_n) {
            rw.accv.assign(mc_n, 0.0);
            rw.mark.assign(mc_n, 0);
            // the row's columns in first-touch order; never more than mc_n,
            // and written ahead of the count (below), so left uninitialised
            rw.cols.reset(new int[(size_t)mc_n + 1]);
            rw.cap = mc_n;
          }
          double* const accv = rw.accv.data();
          char* const mark = rw.mark.data();
          int* const cols = rw.cols.get();
#pragma omp for schedule(dynamic, 1)
          for (int ch = 0; ch < nchunk; ++ch) {
            const int r0 = (int)((int64_t)mc_n * ch / nchunk), r1 = (int)((int64_t)mc_n * (ch + 1) / nchunk);
            ucol[ch].clear();
            uval[ch].clear();
            ucol[ch].reserve((size_t)((r1 - r0) * upper_guess));
            uval[ch].reserve((size_t)((r1 - r0) * upper_guess));
            for (int r = r0; r < r1; ++r) {
              const int k = cnodes[r];
              if (lptr[r] == lptr[r + 1]) {
                // no elimination update reaches this row: S' row = S row on C
                // (column order is preserved by the C numbering)
                const size_t before = ucol[ch].size();
                for (int64_t p = S.ptr[k]; p < S.ptr[k + 1]; ++p) {
                  const int c = cidx[S.col[p]];
                  if (c < r) continue;
                  if (c == r || std::fabs(S.val[p]) >= tau) {
                    ucol[ch].push_back(c);
                    uval[ch].push_back(S.val[p]);
                  }
                }
                rowcnt[r] = (int)(ucol[ch].size() - before);
                continue;
              }
              int nc = 0;
              for (int64_t p = S.ptr[k]; p < S.ptr[k + 1]; ++p) {
                const int c = cidx[S.col[p]];
                if (c < r) continue;  // B columns have cidx -1
                if (!mark[c]) { mark[c] = 1; cols[nc++] = c; }
                accv[c] += S.val[p];
              }
              if (!mark[r]) { mark[r] = 1; cols[nc++] = r; }
              // the blocks of row r of L_F (its records, in block order) with
              // their (l_a, l_b) values; `me` is the row's record in the
              // block's column list (rows ascending)
              for (int64_t i = rrec[r]; i < rrec[r + 1]; ++i) {
                const int b = rec_blk[i];
                const int64_t me = rec_slot[i];
                const double la = c1[me], lb = c2[me];
                double wa, wb;  // (l_a, l_b) * D_b
                if (cands[acc[b]].b < 0) { wa = la * bmat[3 * b]; wb = 0.0; }
                else {
                  wa = la * bmat[3 * b] + lb * bmat[3 * b + 1];
                  wb = la * bmat[3 * b + 1] + lb * bmat[3 * b + 2];
                }
                // about half the updates reach a column for the first time:
                // the column is stored unconditionally and counted only then
                // (no unpredictable branch)
                const int64_t te = cptr[b + 1];
                if (cands[acc[b]].b < 0) {
                  // 1x1 block: wb = 0 and every c2 is 0, so wb * c2 is +0 (the
                  // same sum as the general form, without the second operand)
                  for (int64_t t = me; t < te; ++t) {
                    const int q = crow[t];  // q >= r because rows are ascending
                    cols[nc] = q;
                    nc += !mark[q];
                    mark[q] = 1;
                    accv[q] -= wa * c1[t] + 0.0;
                  }
                } else {
                  for (int64_t t = me; t < te; ++t) {
                    const int q = crow[t];
                    cols[nc] = q;
                    nc += !mark[q];
                    mark[q] = 1;
                    accv[q] -= wa * c1[t] + wb * c2[t];
                  }
                }
              }
              // drop first (branch-free: a dropped column is cleared, a kept
              // one rewritten unchanged), then sort only the entries that stay
              int keep = 0;
              for (int x = 0; x < nc; ++x) {
                const int c = cols[x];
                const double a = accv[c];
                const bool kept = c == r || std::fabs(a) >= tau;
                cols[keep] = c;
                keep += kept;
                accv[c] = kept ? a : 0.0;
                mark[c] = kept;
              }
              // the columns arrive as a few ascending runs (the old row, then
              // the new columns of each block in row order): insertion sort
              // moves little on such input and beats a general sort up to a
              // few hundred entries
              sort_ints(cols, keep, 256);
              const size_t before = ucol[ch].size();
              for (int x = 0; x < keep; ++x) {
                const int c = cols[x];
                ucol[ch].push_back(c);
                uval[ch].push_back(accv[c]);
                accv[c] = 0.0;
                mark[c] = 0;
              }
              rowcnt[r] = (int)(ucol[ch].size() - before);
            }
          }
        }
      }
      ts_num = ms_since(t_schur) - ts_rec;
      // mirror the upper triangle into a full symmetric CSR: row c holds its
      // lower entries (r, c), r < c, in increasing r, then its own upper
      // entries.  Scattering the lower entries straight into their rows would
      // miss the cache on almost every write, so they go through a bucket
      // pass: (1) groups of consecutive chunks (increasing r) copy their upper
      // rows and append each lower entry to the bucket of its column block,
      // behind the entries of the groups before them; (2) each block, small
      // enough to stay in cache, moves its bucket into the rows in bucket
      // order.  Both keep increasing r per column whatever the group count.
      Sn.n = mc_n;
      next_rowmax.resize(mc_n);
      {
        const int64_t nup = [&] {
          int64_t s = 0;
          for (int ch = 0; ch < nchunk; ++ch) s += (int64_t)ucol[ch].size();
          return s;
        }();
        const int G = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)omp_get_max_threads(), (int64_t)nchunk, nup / 16384}));
        constexpr int kBlkShift = 8;  // 256 columns per block
        const int nblk = (mc_n >> kBlkShift) + 1;
        auto chunk_row0 = [&](int ch) { return (int)((int64_t)mc_n * ch / nchunk); };
        dvec<unsigned>& cnt = mirror_cnt;  // per group: lower entries per column
        resize_discard(cnt, (size_t)G * mc_n);
#pragma omp parallel for schedule(static)
        for (int g = 0; g < G; ++g) {
          unsigned* c = cnt.data() + (size_t)g * mc_n;
          std::fill(c, c + mc_n, 0u);
          for (int ch = nchunk * g / G; ch < nchunk * (g + 1) / G; ++ch) {
            const int* col = ucol[ch].data();
            int64_t q = 0;
            for (int r = chunk_row0(ch); r < chunk_row0(ch + 1); ++r)
              for (const int64_t e = q + rowcnt[r]; q < e; ++q)
                if (col[q] != r) ++c[col[q]];
          }
        }
        std::vector<int> lowcnt(mc_n);
        std::vector<int64_t> boff((size_t)G * nblk);  // per group: its first slot in each bucket
        std::vector<int64_t> bptr(nblk + 1, 0);       // bucket b = lower entries of columns [256 b, 256 b + 256)
#pragma omp parallel for schedule(static)
        for (int b = 0; b < nblk; ++b) {
          const int c0 = b << kBlkShift, c1 = std::min(mc_n, c0 + (1 << kBlkShift));
          int64_t run = 0;
          for (int g = 0; g < G; ++g) {
            boff[(size_t)g * nblk + b] = run;
            for (int c = c0; c < c1; ++c) run += cnt[(size_t)g * mc_n + c];
          }
          for (int c = c0; c < c1; ++c) {
            unsigned k = 0;
            for (int g = 0; g < G; ++g) k += cnt[(size_t)g * mc_n + c];
            lowcnt[c] = (int)k;
          }
          bptr[b + 1] = run;
        }
        for (int b = 0; b < nblk; ++b) bptr[b + 1] += bptr[b];
        Sn.ptr.assign(mc_n + 1, 0);
        for (int r = 0; r < mc_n; ++r) Sn.ptr[r + 1] = Sn.ptr[r] + lowcnt[r] + rowcnt[r];
        resize_discard(Sn.col, Sn.ptr[mc_n]);
        resize_discard(Sn.val, Sn.ptr[mc_n]);
        resize_discard(mirror_tmp, bptr[nblk]);
#pragma omp parallel for schedule(static)
        for (int g = 0; g < G; ++g) {
          int64_t* bo = boff.data() + (size_t)g * nblk;
          for (int b = 0; b < nblk; ++b) bo[b] += bptr[b];
          for (int ch = nchunk * g / G; ch < nchunk * (g + 1) / G; ++ch) {
            const int* col = ucol[ch].data();
            const double* val = uval[ch].data();
            int64_t q = 0;
            for (int r = chunk_row0(ch); r < chunk_row0(ch + 1); ++r) {
              int64_t o = Sn.ptr[r] + lowcnt[r];
              double mx = 0.0;  // max |entry| of the row's upper part
              for (const int64_t e = q + rowcnt[r]; q < e; ++q, ++o) {
                const int cc = col[q];
                Sn.col[o] = cc;
                Sn.val[o] = val[q];
                mx = std::max(mx, std::fabs(val[q]));
                if (cc != r) mirror_tmp[bo[cc >> kBlkShift]++] = {r, cc, val[q]};
              }
              next_rowmax[r] = mx;
            }
          }
        }
#pragma omp parallel for schedule(dynamic, 16)
        for (int b = 0; b < nblk; ++b) {
          const int c0 = b << kBlkShift, c1 = std::min(mc_n, c0 + (1 << kBlkShift));
          int64_t next[1 << kBlkShift];  // write position of each column of the block
          double mx[1 << kBlkShift];     // max |entry| of the column's lower part
          for (int c = c0; c < c1; ++c) {
            next[c - c0] = Sn.ptr[c];
            mx[c - c0] = 0.0;
          }
          for (int64_t t = bptr[b]; t < bptr[b + 1]; ++t) {
            const Trip& e = mirror_tmp[t];
            const int64_t slot = next[e.c - c0]++;
            Sn.col[slot] = e.r;
            Sn.val[slot] = e.v;
            mx[e.c - c0] = std::max(mx[e.c - c0], std::fabs(e.v));
          }
          // row maxima of S' for the next level's matching (max is exact, so
          // the same as a pass over the finished rows)
          for (int c = c0; c < c1; ++c) next_rowmax[c] = std::max(next_rowmax[c], mx[c - c0]);
        }
      }
    }
    // next level's numbering
    std::vector<int> gid2(mc_n);
    std::vector<double> cum2(mc_n);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < mc_n; ++r) {
      gid2[r] = gid[cnodes[r]];
      cum2[r] = cum[cnodes[r]];
    }
    gid.swap(gid2);
    cum.swap(cum2);
    if (verbose)
      std::fprintf(stderr, "ildl level %d: m=%d B=%zu C=%d nnzS'/row=%.1f nnzLF=%zu | match %.1f cand %.1f LF %.1f schur %.1f (records %.1f numeric %.1f) total %.1f ms\n",
                   level, m, acc.size(), mc_n, mc_n ? (double)Sn.col.size() / mc_n : 0.0, lnode.size(), tm_ms, tc_ms, tl_ms,
                   ms_since(t_schur), ts_rec, ts_num, ms_since(t_level));
    std::swap(S, Snext);
  }
  const int nlev = level;
  const int nd = S.n;
  {
    // the level scratch is not needed any more: release it before the
    // global assembly allocates the factor
    auto release = [](auto& v) { std::remove_reference_t<decltype(v)>().swap(v); };
    release(mwork.loga);
    release(mwork.threads);
    release(mwork.rowmax_in);
    release(mwork.u_in);
    release(mwork.v_in);
    release(Snext.ptr);
    release(Snext.col);
    release(Snext.val);
    release(lnode);
    release(lval);
    release(agg_node);
    release(agg_val);
    release(ucol);
    release(uval);
    release(rec_row);
    release(rec_blk);
    release(crow);
    release(rec_a);
    release(rec_b);
    release(c1);
    release(c2);
    release(rec_slot);
    release(mirror_cnt);
    release(rwork);
  }
  // trailing dense block
  dvec<double> dense_inv;
  if (nd > 0) {
    dvec<double> M((size_t)nd * nd);  // rows zeroed and filled in parallel
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nd; ++i) {
      double* row = M.data() + (size_t)i * nd;
      std::fill(row, row + nd, 0.0);
      for (int64_t p = S.ptr[i]; p < S.ptr[i + 1]; ++p) row[S.col[p]] = S.val[p];
    }
    const auto t_dense = Clock::now();
    if (dense_on_host) {
      if (!dense_inverse(nd, M, dense_inv))
        return fail(JD_ESETUP, "ildl: the final dense block (%d rows) is singular", nd);
    } else {
      dense_inv.swap(M);  // inverted on the device by the caller
      F.dense_is_matrix = true;
    }
    if (verbose) std::fprintf(stderr, "ildl dense block %d rows: %.1f ms\n", nd, ms_since(t_dense));
    for (int i = 0; i < nd; ++i) {
      order.push_back(gid[i]);
      sc[gid[i]] = cum[i];
    }
  }
  level_ptr.push_back((int)order.size());
  if ((int)order.size() != n) return fail(JD_ESETUP, "ildl: internal error, %zu of %d rows ordered", order.size(), n);

  // global assembly in position space (parallel counting and scattering;
  // every row is sorted afterwards, so the result does not depend on the
  // scatter order)
  const auto t_asm = Clock::now();
  std::vector<int> pos(n);
#pragma omp parallel for schedule(static)
  for (int p = 0; p < n; ++p) pos[order[p]] = p;
  F.nlev = nlev;
  F.n_dense = nd;
  F.perm = order;
  F.scale.resize(n);
#pragma omp parallel for schedule(static)
  for (int p = 0; p < n; ++p) F.scale[p] = sc[order[p]];
  F.level_ptr = level_ptr;
  // L rows: the triplets of a row were appended level by level, and within
  // a level in increasing pivot position, so a stable scatter leaves every
  // row sorted by column
  const int64_t nt = (int64_t)trips.size();
  {
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(omp_get_max_threads(), nt / 16384));
    stable_place(
        G, n,
        [&](int g, auto&& emit) {
          for (int64_t q = nt * g / G; q < nt * (g + 1) / G; ++q) {
            const Trip& t = trips[q];
            emit(Trip{pos[t.r], pos[t.c], t.v * sc[t.r]});
          }
        },
        F.Lptr, mirror_tmp, F.Lcol, F.Lval);
  }
  trips.clear();
  trips.shrink_to_fit();
  {
    // transpose (rows of L^T = columns of L), entries ordered by row: row
    // groups of about equal entry counts, in row order
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(omp_get_max_threads(), nt / 16384));
    std::vector<int> rcut(G + 1, n);
    rcut[0] = 0;
    for (int g = 1; g < G; ++g)
      rcut[g] = (int)(std::lower_bound(F.Lptr.begin(), F.Lptr.end(), nt * g / G) - F.Lptr.begin());
    stable_place(
        G, n,
        [&](int g, auto&& emit) {
          for (int r = rcut[g]; r < rcut[g + 1]; ++r)
            for (int64_t q = F.Lptr[r]; q < F.Lptr[r + 1]; ++q) emit(Trip{F.Lcol[q], r, F.Lval[q]});
        },
        F.Uptr, mirror_tmp, F.Ucol, F.Uval);
  }
  dvec<Trip>().swap(mirror_tmp);
  F.dinv_d.assign(n, 0.0);
  F.dinv_o.assign(n, 0.0);
  F.partner.assign(n, -1);
#pragma omp parallel for schedule(static)
  for (int p = 0; p < n - nd; ++p) {
    const int o = order[p];
    F.dinv_d[p] = dd[o];
    F.dinv_o[p] = dof[o];
    F.partner[p] = part[o] >= 0 ? pos[part[o]] : -1;
  }
  F.dense_inv.swap(dense_inv);
  double mx = 0.0;
#pragma omp parallel for reduction(max : mx) schedule(static)
  for (int64_t q = 0; q < nt; ++q) mx = std::max(mx, std::fabs(F.Lval[q]));
  F.max_abs_L = mx;
  if (verbose) std::fprintf(stderr, "ildl global assembly: %.1f ms\n", ms_since(t_asm));
  F.t_match_ms = t_match;
  F.t_total_ms = ms_since(t_start);
  F.t_factor_ms = F.t_total_ms - t_match;
  return JD_OK;
}

}  // namespace ajd
