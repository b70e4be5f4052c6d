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
  int apply_shift = 0;            // autotuned threads-per-row scale of the apply, log2
  int apply_form = 0;             // apply kernel: 0 level counters, 1 dataflow
  double apply_tune_ms[2][3] = {{0, 0, 0}, {0, 0, 0}};  // apply time per form and shift -1, 0, +1 (0 = not timed)
  std::vector<int> level_sizes;   // rows eliminated per sparse level
};

// One level's Schur complement S' = S_CC - L_F D_B L_F^T as the level loop
// of build_ildl hands it to a SchurEngine (all arrays host, in the loop's
// local numbering; see the loop for their construction):
//   cidx[m]         C index of each local row, -1 for the level's pivots;
//   cnodes[mc_n]    local row of each C row;
//   rrec[mc_n+1]    records of C row r: rrec[r] .. rrec[r+1], in block order;
//   rec_blk, rec_slot  per record: its pivot block b and its position in the
//                   block's column list;
//   cptr[nblk+1], crow, c1, c2  per block b, its column list cptr[b] ..
//                   cptr[b+1]: C rows (ascending) with the L_F values of
//                   the block's nodes a and b (c2 = 0 for a 1x1 block);
//   bmat[3 nblk]    the symmetric pivot blocks (a, s, c), is2x2[nblk];
//   tau             drop tolerance of S' (off the diagonal).
struct SchurLevel {
  int m = 0, mc_n = 0, nblk = 0;
  const int64_t* sptr = nullptr;  // row pointers of the level matrix S (m + 1)
  const int* cidx = nullptr;
  const int* cnodes = nullptr;
  const int64_t* rrec = nullptr;
  const int* rec_blk = nullptr;
  const int64_t* rec_slot = nullptr;
  const int64_t* cptr = nullptr;
  const int* crow = nullptr;
  const double* c1 = nullptr;
  const double* c2 = nullptr;
  const double* bmat = nullptr;
  const char* is2x2 = nullptr;
  double tau = 0.0;
};

// Computes the Schur complements of the level loop somewhere other than the
// host threads (the GPU).  It keeps its own copy of the level matrix S:
// begin() receives A, scale() the level's scaling d (S_ij *= d_i d_j, the
// same products as the host's), and schur() returns S' -- full symmetric
// CSR, rows sorted, bit for bit what the host code computes -- together with
// the maxima |S'_ij| of its rows, and makes S' its level matrix.
class SchurEngine {
 public:
  virtual ~SchurEngine() = default;
  virtual int begin(const SymCsr& A) = 0;
  virtual int scale(const double* d, int m) = 0;
  // S' of the level, its row maxima and, when u, v and loga are given, the
  // matching's dual potentials of S' and log |s'_ij| of every stored entry
  // (as max_product_matching forms them before its searches: the same bits)
  virtual int schur(const SchurLevel& lv, SymCsr& Sn, std::vector<double>& rowmax, std::vector<double>* u,
                    std::vector<double>* v, dvec<double>* loga) = 0;
};

// Default weak-coupling threshold gamma of the independent sets for an
// order-n matrix: min(0.02, 5/sqrt(n)), or min(0.02, 1/sqrt(n)) for the
// off-diagonal model.
double default_gamma(int64_t n, bool offdiag);

// Default size of the dense trailing block for an order-n matrix (rows).
int default_n_dense(int64_t n);

// Build the preconditioner of A (symmetric, e.g. A - sigma I).  Returns
// JD_OK or JD_ESETUP / JD_EINVAL with jd_last_error() set.  With
// dense_on_host = false the trailing dense block is left un-inverted
// (dense_is_matrix) for a device-side inversion.
int build_ildl(const SymCsr& A, const ildl_params& p, HostFactor& F, bool dense_on_host = true,
               SchurEngine* engine = nullptr);

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
  // optional, with rowmax_in: the initial dual potentials u, v of the next
  // matrix and log|a_ij| of its entries (in loga), formed elsewhere (the GPU
  // that formed the matrix) with the same arithmetic.  Used once if u_in
  // and v_in have n entries and loga_in is set.
  std::vector<double> u_in, v_in;
  bool loga_in = false;
};

// The table of the matching's division-free logarithm (128 values of 1/c_k
// and of ln c_k, c_k = 1 + k/128), for a device copy of the same function.
void log_table_data(const double** inv, const double** logc);
int max_product_matching(const SymCsr& A, std::vector<int>& match_col, std::vector<double>& u,
                         std::vector<double>& v, std::vector<double>& rowmax, MatchWork* work = nullptr);

// Split the cycles of the permutation j -> match_col[j] into 1- and 2-cycles
// (Section 5.2).  `sdiag` and the scaled matrix decide the splits.  Returns
// groups as pairs (a, b) with b = -1 for singletons.
void split_cycles(const SymCsr& S, const std::vector<int>& match_col,
                  std::vector<std::pair<int, int>>& groups);

}  // namespace ajd
