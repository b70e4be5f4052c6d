// Host-side construction of the multilevel incomplete LDL^T preconditioner
// (Sections 5 and 6).  Pure C++ (no CUDA), so it also runs without a GPU.
#pragma once
#include <cstdint>
#include <memory>
#include <utility>
#include <vector>

#include "anderson_jd.h"

namespace ajd {

// std::allocator that leaves elements default-initialised (no zero fill on
// resize): the large per-level arrays of the setup are then first touched
// by the parallel loops that fill them, not by a serial memset.
template <class T>
struct default_init_allocator : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = default_init_allocator<U>;
  };
  default_init_allocator() = default;
  template <class U>
  default_init_allocator(const default_init_allocator<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... Args>
  void construct(U* p, Args&&... args) {
    ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
  }
};
template <class T>
using dvec = std::vector<T, default_init_allocator<T>>;

// Symmetric sparse matrix, both triangles stored, rows sorted by column,
// diagonal entry always present (possibly zero).
struct SymCsr {
  int n = 0;
  std::vector<int64_t> ptr;
  dvec<int> col;
  dvec<double> val;
};

// The factor in global (level-ordered) position space:
//   K^{-1} b = P^T S L^{-T} D^{-1} L^{-1} S P b,
// (P b)[p] = b[perm[p]], S = diag(scale), L unit lower triangular, D block
// diagonal with 1x1/2x2 blocks on levels 0..nlev-1 and one dense block of
// size n_dense on the trailing positions.
struct HostFactor {
  int n = 0;
  int nlev = 0;                   // number of sparse levels
  int n_dense = 0;                // size of the trailing dense block
  std::vector<int> perm;          // position -> original index
  std::vector<double> scale;      // S
  std::vector<int> level_ptr;     // nlev + 2 entries: sparse levels, then the dense block
  std::vector<int64_t> Lptr;      // strictly lower part of L, CSR by rows
  dvec<int> Lcol;
  dvec<double> Lval;
  std::vector<int64_t> Uptr;      // L^T, CSR by rows (= L by columns)
  dvec<int> Ucol;
  dvec<double> Uval;
  std::vector<double> dinv_d;     // per position: diagonal of D^{-1} block
  std::vector<double> dinv_o;     // per position: off-diagonal of D^{-1} block
  std::vector<int> partner;       // per position: 2x2 partner position or -1
  dvec<double> dense_inv;         // n_dense^2, row-major, symmetric
  bool dense_is_matrix = false;   // dense_inv still holds the block itself
  // statistics
  int n_2x2 = 0;
  int n_matched_offdiag = 0;      // rows matched off the diagonal at level 0
  int n_relaxed = 0;              // levels where pivot acceptance was relaxed
  int64_t n_aggressive = 0;       // entries removed by aggressive dropping
  double max_abs_L = 0.0;         // largest |entry| of the global L
  int64_t nnz_A = 0;
  double t_match_ms = 0, t_factor_ms = 0, t_total_ms = 0;
  std::vector<int> level_sizes;   // rows eliminated per sparse level
};

// Build the preconditioner of A (symmetric, e.g. A - sigma I).  Returns
// JD_OK or JD_ESETUP / JD_EINVAL with jd_last_error() set.  With
// dense_on_host = false the trailing dense block is left un-inverted
// (dense_is_matrix) for a device-side inversion.
int build_ildl(const SymCsr& A, const ildl_params& p, HostFactor& F, bool dense_on_host = true);

// Maximum-product transversal of Section 5.1 (Eqs. (5.1)-(5.2)): on return
// match_col[j] is the row matched to column j, u and v are the dual
// potentials of the assignment problem with costs c_ij = log a_i - log|a_ij|,
// a_i = max_j |a_ij|.  Returns the number of unmatched columns (0 when a
// perfect matching exists).
// `work` (optional) holds the scratch arrays between calls, so that a caller
// matching a sequence of matrices (the levels of the factorization) reuses
// memory that is already mapped instead of faulting in fresh pages per call.
struct MatchWork {
  dvec<double> loga;        // log|a| per stored entry
  struct Search {           // per OpenMP thread; at rest: dist = inf, pred = -1, done = 0
    std::vector<double> dist;
    std::vector<int> pred;
    std::vector<char> done;
    std::vector<std::pair<double, int>> heap;
  };
  std::vector<Search> threads;
  // optional: max |a_ij| of every row of the next matrix, when the caller
  // has it already (one pass over the matrix fewer); used if it has n entries
  std::vector<double> rowmax_in;
};
int max_product_matching(const SymCsr& A, std::vector<int>& match_col, std::vector<double>& u,
                         std::vector<double>& v, std::vector<double>& rowmax, MatchWork* work = nullptr);

// Split the cycles of the permutation j -> match_col[j] into 1- and 2-cycles
// (Section 5.2).  `sdiag` and the scaled matrix decide the splits.  Returns
// groups as pairs (a, b) with b = -1 for singletons.
void split_cycles(const SymCsr& S, const std::vector<int>& match_col,
                  std::vector<std::pair<int, int>>& groups);

}  // namespace ajd
