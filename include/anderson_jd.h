/*
 * anderson_jd.h -- C ABI of the GB300 Jacobi–Davidson library for the
 * 3D Anderson model of localization.
 *
 * The library computes the few eigenpairs of the Anderson matrix nearest an
 * interior shift sigma, following O. Schenk, M. Bollhöfer, R. A. Römer,
 * "On large scale diagonalization techniques for the Anderson model of
 * localization" (arXiv math/0508111):
 *   - the matrix of Eq. (1) (Section 3), applied matrix-free;
 *   - the symmetric Jacobi–Davidson method of Section 4.2 with the
 *     correction equation (4.1), solved approximately by simplified QMR;
 *   - the preconditioner of Sections 5 and 6: a maximum-weight-matching
 *     permuted, scaled, multilevel incomplete LDL^T with 1x1/2x2 pivots,
 *     inverse-based pivoting and threshold dropping.
 *
 * Conventions for every call:
 *   - Return value: JD_OK (0) on success, a negative JD_E* code otherwise;
 *     jd_last_error() then gives a one-line message (thread-local).  No C++
 *     exception crosses this interface.
 *   - Handles are opaque and owned by the library; *_destroy(NULL) is a no-op.
 *   - "device pointer" arguments must point to memory of the device that was
 *     current when the handle was created; "host pointer" arguments to
 *     ordinary host memory.  Caller-owned buffers are never freed by the
 *     library.
 *   - Vectors are indexed by lattice site idx = x + L*(y + L*z), x fastest,
 *     0 <= x, y, z < L.  A block of m vectors is column-major: vector j
 *     starts at element j*n.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream are asynchronous with respect to the
 *     host unless stated otherwise.
 */
#ifndef ANDERSON_JD_H
#define ANDERSON_JD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define JD_OK 0
#define JD_EINVAL (-1)      /* invalid argument                               */
#define JD_ENOMEM (-2)      /* host or device allocation failed               */
#define JD_ENOCONV (-3)     /* not all requested eigenpairs converged         */
#define JD_EBREAKDOWN (-4)  /* persistent Krylov breakdown                    */
#define JD_EDEVICE (-5)     /* CUDA error or a device-side wait that timed out*/
#define JD_ESETUP (-6)      /* preconditioner construction failed             */
#define JD_EAGAIN (-7)      /* jd_poll: the request is queued or running      */

/* ---- boundary conditions and precisions -------------------------------- */
#define JD_PERIODIC 0 /* x_{M+1} = x_1 (the default of every table)           */
#define JD_HARDWALL 1 /* x_0 = x_{M+1} = 0 (Section 7, Table 6)               */

#define JD_FP64 0  /* arithmetic in binary64                                  */
#define JD_FP32 1  /* arithmetic in binary32 (vectors and potential in FP32)  */
#define JD_MIXED 2 /* binary32 factor values applied with float-float
                      (hi + lo, ~48-bit) work vectors and sums; SQMR vectors,
                      stencil and everything else binary64                    */

/* Message of the last failing call on this thread ("" if none). */
const char* jd_last_error(void);

/* Library version, as 10000*major + 100*minor + patch. */
int jd_version(void);

/* ======================================================================== *
 *  The Anderson matrix (Section 3, Eq. (1))                                 *
 * ======================================================================== */
typedef struct anderson_s* anderson_t;

/*
 * anderson_create -- an L x L x L Anderson lattice with box disorder.
 *
 * Eq. (1): (A x)_s = eps_s x_s + t * sum_{s' nearest neighbour of s} x_s',
 * with hopping t = -1.  The on-site energies are drawn from the box
 * distribution [-W/2, W/2] (Section 3): eps_s = W * (u_s - 1/2), where
 * u_s = (SplitMix64 output number s for seed `seed`) >> 11, times 2^-53,
 * i.e. the s-th output of Steele–Lea–Flood SplitMix64 (state advanced by
 * 0x9E3779B97F4A7C15, variant-13 finaliser).  The potential is generated on
 * the current device and kept there (binary64 and a binary32 copy); the
 * matrix itself is never stored (Section 3.1: only the diagonal is needed).
 *
 *   L    lattice edge; L >= 3 for JD_PERIODIC, L >= 1 for JD_HARDWALL;
 *        L^3 < 2^31.
 *   W    disorder strength, W >= 0 and finite.
 *   seed any 64-bit value.
 *   bc   JD_PERIODIC or JD_HARDWALL.
 *   out  receives the handle.
 * Errors: JD_EINVAL for bad arguments, JD_ENOMEM / JD_EDEVICE from CUDA.
 * Synchronous: the potential is complete when the call returns.
 */
int anderson_create(int L, double W, uint64_t seed, int bc, anderson_t* out);

/*
 * anderson_create_from_potential -- a lattice whose on-site energies are
 * supplied by the caller (host buffer eps_host[L^3], binary64, site order
 * x fastest) instead of being drawn from the box distribution.  The values
 * are copied to the device (a pinned host buffer makes the copy
 * asynchronous-capable; any host buffer works).  W and seed of the handle are
 * recorded as 0.  Same argument rules as anderson_create; eps must be
 * finite.  Synchronous.
 */
int anderson_create_from_potential(int L, const double* eps_host, int bc, anderson_t* out);

/*
 * anderson_create_offdiag -- the off-diagonal ("inverse") Anderson model of
 * Section 7 (Table 6): the same nearest-neighbour graph as Eq. (1), a
 * constant diagonal `diag` (1.28 at the transition the paper studies) and
 * random hopping on every bond: the bond from site s to its +x, +y, +z
 * neighbour (d = 0, 1, 2) gets t = width * (u_{3s+d} - 1/2) with u_i the
 * i-th value of the SplitMix64 stream of anderson_create (uniform on
 * [-width/2, width/2); width 1 in the paper).  Hard walls drop the bonds
 * that leave the cube.  anderson_norm returns the Gershgorin bound
 * |diag| + 6 max|t| used as ||A|| by jd_solve's tolerance.
 *   L, seed, bc as for anderson_create (3 L^3 < 2^31); diag finite;
 *   width finite, >= 0.
 * Errors: JD_EINVAL, JD_ENOMEM / JD_EDEVICE.  Synchronous.
 */
int anderson_create_offdiag(int L, double diag, double width, uint64_t seed, int bc, anderson_t* out);

/* Copy the hoppings t[3s + d] (binary64, 3 L^3 values, 0 for bonds a hard
 * wall removes) to the caller's host buffer.  JD_EINVAL for a lattice of
 * Eq. (1) (constant hopping -1). */
int anderson_bonds(anderson_t h, double* bonds_host);

/* Release the handle and its device memory.  NULL is a no-op. */
int anderson_destroy(anderson_t h);

/* Number of sites n = L^3. */
int anderson_size(anderson_t h, int64_t* n);

/* Copy the binary64 potential eps[0..n) to the caller's host buffer. */
int anderson_potential(anderson_t h, double* eps_host);

/* ||A|| used for relative tolerances: 6 + max_s |eps_s|, the Gershgorin
 * radius behind the spectral interval [-6 - W/2, 6 + W/2] (Section 3). */
int anderson_norm(anderson_t h, double* norm);

/*
 * anderson_apply -- y = (A - shift I) x for a block of m vectors
 * (the matrix-free 7-point stencil, Eq. (1)).
 *   x, y       device pointers, n*m elements each, column-major, not
 *              overlapping; binary64 if precision == JD_FP64, binary32 if
 *              JD_FP32 (the binary32 path uses the binary32 potential).
 *   m          number of vectors, m >= 1 (m = 0 is a no-op).
 *   stream     cudaStream_t or NULL.
 * Errors: JD_EINVAL (null pointers, m < 0, unknown precision), JD_EDEVICE.
 */
int anderson_apply(anderson_t h, double shift, const void* x, void* y, int m,
                   int precision, void* stream);

/* ======================================================================== *
 *  Preconditioner K ~ A - sigma I (Sections 5 and 6)                        *
 * ======================================================================== */
typedef struct ildl_s* ildl_t;

/* Parameters of the multilevel incomplete LDL^T.  Defaults in brackets. */
typedef struct {
  double kappa;   /* bound on ||L^{-1}|| of each level (inverse-based pivoting,
                     Section 6.2); pivots that would exceed it are postponed
                     to the next level [5, the value used in Section 7]      */
  double drop;    /* drop tolerance epsilon: entries of L and of the Schur
                     complement below epsilon/kappa in modulus are dropped
                     (Section 6.2); < 0 selects 1/sqrt(n) (Section 7), 0
                     disables dropping [-1]                                  */
  double gamma;   /* couplings below gamma (scaled matrix, entries <= 1) are
                     ignored when each level's independent set of pivots is
                     chosen, and dropped between pivots of the same level;
                     0 = exact independence; < 0 selects
                     min(0.02, 5/sqrt(n)), and min(0.02, 1/sqrt(n)) for the
                     lattices of anderson_create_offdiag [-1]                */
  int max_levels; /* maximum number of sparse levels [256]                    */
  int n_dense;    /* the remaining Schur complement is factored densely once
                     it has at most this many rows (at most 8000); 0 = n/16
                     clamped to 1000..3000 (3000 at n = 10^6: the inversion
                     is O(n_dense^3) binary64 work on the device) [0]       */
  int matching;   /* levels that use the maximum-product matching, 1x1/2x2
                     cycle split and symmetric dual scaling (Sections 5.1,
                     5.2); deeper levels use row-max scaling and 1x1
                     candidates; 0 = none, < 0 = every level [-1]            */
  double aggressive; /* tau of the aggressive dropping of Section 6.3: an
                     entry l_ij of a level's column block of L is dropped
                     when |l_ij| <= tau / #(nonzeros of column j of the
                     block); the paper's norm estimate nu_i of L^{-1} e_i is
                     exactly 1 for every row of a level's block.  Applied
                     as soon as the block is computed, so the Schur
                     complement is formed from the sparsified block.
                     0 = off, else 0 < tau < 1 (the paper suggests 0.1) [0] */
  int setup_device; /* where the levels' Schur complements S' = S_CC -
                     L_F D_B L_F^T (Section 6.3) are formed: 1 = on the GPU
                     (the lattice's device for ildl_create, the current
                     device for ildl_setup_csr), 0 = on the host threads,
                     < 0 = GPU for ildl_create and host for ildl_setup_csr.
                     Both give the same factor bit for bit [-1]         */
  int autotune;   /* ildl_create only: time the apply in each form of
                     apply_form with the threads-per-row rule scaled by 1/2,
                     1 and 2 on the device and keep the fastest (factors of
                     at least 200,000 rows; four applies per candidate);
                     0 = off, else on [-1]                                   */
  int apply_form; /* kernel of ildl_apply (the same x in either form, up to
                     the rounding of the row sums): 0 = level sweeps with a
                     completion count per level; 1 = dataflow, every row
                     starts once the entries it reads are written (no
                     per-level synchronisation); < 0 = chosen by the
                     autotuner where it runs (1 unless 0 is faster by more
                     than 25%), else 1 [-1]                                   */
} ildl_params;

/* Fill *p with the defaults above. */
int ildl_params_default(ildl_params* p);

/* The threshold gamma that gamma < 0 selects for an order-n matrix:
 * min(0.02, 5/sqrt(n)), or min(0.02, 1/sqrt(n)) when offdiag != 0 (the
 * lattices of anderson_create_offdiag, Section 7).  Host only; JD_EINVAL if
 * n < 1 or gamma is NULL. */
int ildl_default_gamma(int64_t n, int offdiag, double* gamma);

/* Sizes and statistics of a factor. */
typedef struct {
  int n;             /* order                                               */
  int levels;        /* sparse levels (each one parallel step of the solves)*/
  int n_dense;       /* order of the trailing dense block                   */
  int n_2x2;         /* number of 2x2 pivots                                */
  int64_t nnz_L;     /* stored entries of the strictly lower factor L       */
  int64_t nnz_A;     /* stored entries of the input matrix                  */
  double fill;       /* nnz(L D L^T)/nnz(A) = (2 nnz_L + nnz(D))/nnz(A),
                        the measure of Table 5                              */
  double setup_ms;   /* wall time of the construction (host + dense inverse) */
  double match_ms;   /* of which: matchings and scalings                    */
  int relaxed_levels;/* levels where fewer than 0.5% of the rows met kappa and
                        the bound was widened (at most 64 kappa)            */
  double max_abs_L;  /* largest |entry| of L (after the global scaling)     */
  int64_t aggressive_dropped; /* entries removed by aggressive dropping
                        (ildl_params.aggressive; 0 when off)                */
  int apply_shift;   /* autotuned threads per row of the apply: the rule's
                        choice times 2^apply_shift (-1, 0 or 1; 0 untuned) */
  int apply_form;    /* apply kernel in use (ildl_params.apply_form)        */
} ildl_info_t;

/*
 * ildl_setup_csr -- build the preconditioner of a symmetric matrix on the
 * host (no GPU needed).  The matrix is given in CSR with both triangles:
 * rowptr[n+1] (int64), col[nnz] (int32, sorted within each row), val[nnz].
 * The factor is an approximation K = P^T S^{-1} L D L^T S^{-1} P of the
 * matrix (see ildl_export).  Errors: JD_EINVAL, JD_ENOMEM, JD_ESETUP
 * (singular dense block or no usable pivot).
 */
int ildl_setup_csr(int n, const int64_t* rowptr, const int* col, const double* val,
                   const ildl_params* p, ildl_t* out);

/*
 * ildl_matching -- the first setup step on its own (Sections 5.1, 5.2):
 * maximum-product matching of a symmetric CSR matrix (Eqs. (5.1)-(5.2)),
 * the symmetric scaling from its dual potentials, and the split of the
 * matching's cycles into 1x1 and 2x2 groups.  Host only.
 *   match_col[n]  row matched to column j (the permutation sigma)
 *   scale[n]      D with |d_i a_ij d_j| <= 1 and matched entries == 1
 *   partner[n]    2x2 partner of row i within its group, or -1 (1x1)
 * Returns JD_OK, or JD_EINVAL; a structurally singular matrix is matched
 * as far as possible (the leftover rows are paired in index order).
 */
int ildl_matching(int n, const int64_t* rowptr, const int* col, const double* val, int* match_col,
                  double* scale, int* partner);

/*
 * ildl_create -- build the preconditioner of A - sigma I for the lattice h
 * (host construction from the lattice's potential), then upload it to the
 * device of h in binary64 and binary32.  Synchronous.
 */
int ildl_create(anderson_t h, double sigma, const ildl_params* p, ildl_t* out);

/* Statistics of a factor. */
int ildl_info(ildl_t f, ildl_info_t* info);

/*
 * ildl_export -- copy the factor to caller-owned host arrays.  With
 * m = info.n, d = info.n_dense, nl = info.levels, nnz = info.nnz_L:
 *   perm[m]          position p holds original index perm[p]
 *   scale[m]         S
 *   level_ptr[nl+2]  positions of level l are [level_ptr[l], level_ptr[l+1]);
 *                    the dense block is [level_ptr[nl], level_ptr[nl+1]=m)
 *   Lptr[m+1], Lcol[nnz], Lval[nnz]   strictly lower L, CSR by positions
 *   dinv_d[m], dinv_o[m], partner[m]  D^{-1}: for a 1x1 pivot at p,
 *                    (D^{-1} y)_p = dinv_d[p] y_p; for a 2x2 pivot (p, q=partner[p]),
 *                    (D^{-1} y)_p = dinv_d[p] y_p + dinv_o[p] y_q; unused on
 *                    dense positions
 *   dense_inv[d*d]   inverse of the dense block, row-major
 * so that K^{-1} b = P^T S L^{-T} D^{-1} L^{-1} S P b with (P b)[p] = b[perm[p]].
 * Any pointer may be NULL to skip that array.
 */
int ildl_export(ildl_t f, int* perm, double* scale, int* level_ptr, int64_t* Lptr, int* Lcol,
                double* Lval, double* dinv_d, double* dinv_o, int* partner, double* dense_inv);

/*
 * ildl_dataflow_schedule -- the work units of the dataflow apply
 * (ildl_params.apply_form = 1) for this factor with the threads-per-row
 * rule scaled by 2^shift (shift in -1..1), for inspection and tests; host
 * only, also for factors without a device copy.  The units form one
 * sequence in segments, 5 ints per segment in seg[]:
 *   kind        0 level 0 (32 rows per unit), 1 forward level, 2 dense tail
 *               (one row per unit), 3 backward level
 *   lanes       lanes per row G (1..32; 32/G rows per unit of a sparse level)
 *   first, end  the positions [first, end) of the segment's rows
 *   unit0       the first unit of the segment
 * Segments come in the order the units are taken: level 0, forward levels
 * 1..nl (the last one being the dense rows' L part), the dense tail,
 * backward levels nl-1..0 (Section 6's forward and backward sweeps of the
 * level-by-level L; the kernel's correctness rests on every unit reading
 * only values written by earlier units).  cap is seg's capacity in
 * segments; *nseg and *nunits receive the counts (*nseg even when cap is
 * too small, which returns JD_EINVAL).
 */
int ildl_dataflow_schedule(ildl_t f, int shift, int* seg, int cap, int* nseg, int* nunits);

/*
 * ildl_apply -- x = K^{-1} b on the device (created by ildl_create): one
 * gather/scale pass, one parallel step per level of L (forward), the block
 * diagonal and dense solves, one parallel step per level of L^T (backward),
 * and one scatter/scale pass.
 *   b, x       device pointers, n elements each, distinct; binary64 for
 *              JD_FP64 and JD_MIXED (binary32 factor, float-float work
 *              vectors and sums), binary32 for JD_FP32.
 * Errors: JD_EINVAL (no device copy, bad precision), JD_EDEVICE.
 */
int ildl_apply(ildl_t f, const void* b, void* x, int precision, void* stream);

/*
 * ildl_apply_noalloc -- x = K^{-1} b like ildl_apply, for callers that cannot
 * allocate device memory during the call (a fixed memory pool reserved up
 * front, an embedding runtime that owns all device memory).  The paper has no
 * counterpart: this is a deployment variant.
 * It runs the level-counter form of the apply kernel (apply_form 0, whatever
 * form the factor's own applies use; the result agrees with ildl_apply to
 * rounding) and takes its scratch (two work vectors, the status word of its
 * waits and the completion counters of its phases) from
 * one static device array compiled into the library (2 MiB + 16.5 KiB, held
 * by every GPU that loads the library until the process exits) instead of
 * the factor's buffers; it calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *   f          a factor from ildl_create with at most 131072 rows (n = L^3,
 *              L <= 50) and at most 4096 apply phases (two per sparse
 *              level); larger factors are rejected with JD_EINVAL.  The
 *              factor's device must be the current device (JD_EINVAL
 *              otherwise).
 *   b, x       device pointers as for ildl_apply; precision JD_FP64,
 *              JD_FP32 or JD_MIXED.
 * Every call shares the one array (its previous contents are kept; the call
 * clears the words that must start at zero), so calls that overlap on the
 * GPU -- on different streams or threads -- race and must not be issued.
 * The launch is ordered behind the preconditioner applies of jd_server's
 * concurrent solves; it must not overlap an ildl_apply or jd_solve issued
 * on another stream of the same device.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The call waits for the apply to finish and
 * returns JD_EDEVICE if a device-side wait timed out.
 */
int ildl_apply_noalloc(ildl_t f, const void* b, void* x, int precision, void* stream);

/* Release the factor (host and device parts).  NULL is a no-op. */
int ildl_destroy(ildl_t f);

/* ======================================================================== *
 *  Jacobi–Davidson eigensolver (Section 4.2)                                *
 * ======================================================================== */

/* Solver parameters.  Zero fields select the defaults in brackets. */
typedef struct {
  int jmin;           /* search space size kept at a restart [max(2k, 10)]     */
  int jmax;           /* search space size that triggers a restart [jmin+15]   */
  int max_outer;      /* outer (expansion) steps before JD_ENOCONV [3000]      */
  int max_inner;      /* SQMR iterations per correction equation [60]          */
  double inner_decay; /* the correction equation is solved to relative
                         residual max(inner_decay^j, inner_floor), j = outer
                         steps spent on the current Ritz pair [0.7]            */
  double inner_floor; /* [0 = 1e-8 for JD_FP64, 1e-6 for JD_MIXED, 1e-5 for
                         JD_FP32, the level a binary32 solve can still reach] */
  double switch_tol;  /* correction shift: sigma while ||r|| > switch_tol*||A||,
                         the Ritz value theta afterwards [1e-3]                */
  int precision;      /* inner solve: JD_FP64 (all binary64), JD_FP32
                         (stencil, preconditioner and SQMR in binary32) or
                         JD_MIXED (binary32 factor applied with float-float
                         sums; SQMR vectors and stencil in binary64); the
                         outer residual, Ritz
                         projection and orthogonalisation are always
                         binary64 [JD_FP64]                                   */
  uint64_t seed;      /* start vector seed (0 = derived from the lattice seed)*/
  int extraction;     /* 0: harmonic Ritz vectors for targets nearest sigma
                         (robust in the dense interior spectrum); 1: standard
                         Ritz vectors of V^T A V as printed in Section 4.2 [0] */
  int guard;          /* extra pairs computed beyond k; the k nearest of the
                         converged pairs are returned, which protects against
                         a nearer eigenvalue found after a farther one was
                         locked (0 = default 2, < 0 = none)                  */
  ildl_params ildl;   /* preconditioner parameters (zeroed = defaults)       */
  ildl_t precond;     /* optional prebuilt preconditioner of A - sigma I
                         (from ildl_create with the same sigma); NULL = build
                         one inside the call and time it as setup           */
  int gram;           /* first pass of the block Gram-Schmidt that extends
                         the search space (Section 4.2): 1 = binary64 (both
                         passes binary64), 2 = BF16 operands on the tensor
                         cores with FP32 accumulation (second pass
                         binary64); 0 = 2 for JD_MIXED and JD_FP32, 1 for
                         JD_FP64 [0]                                         */
} jd_params;

/* jd_gram_bf16 -- out = BF16(X)^T BF16(t): the first pass of the block
 * Gram-Schmidt of the search-space expansion (Section 4.2) on the tensor
 * cores (tcgen05.mma, BF16 operands, FP32 accumulation per 64-row chunk and
 * CTA, binary64 sum over CTAs), as jd_solve runs it with gram = 2.
 *   X      device, n x c column-major binary64, leading dimension ldx >= n;
 *          c <= 128 columns
 *   t      device, n binary64
 *   out    c binary64 (host or device pointer)
 * Allocates and frees its own BF16 copy of X (c x n x 2 bytes).  JD_EINVAL
 * for bad sizes, JD_EDEVICE on a CUDA error or a tensor-core wait that timed
 * out. */
int jd_gram_bf16(const double* X, int64_t ldx, int c, const double* t, int64_t n, double* out, void* stream);

/* Counters of one solve (the observables of Tables 3-5). */
typedef struct {
  int nconv;           /* eigenpairs that met the tolerance                   */
  int outer_its;       /* Jacobi–Davidson expansion steps                     */
  int inner_its;       /* total SQMR iterations                               */
  int restarts;        /* search space restarts                               */
  double setup_ms;     /* preconditioner construction (host) and upload       */
  double solve_ms;     /* everything after the setup                          */
  double max_residual; /* max ||A x - lambda x||_2 / ||A|| over returned pairs */
  double orth_error;   /* max |X^T X - I| over returned pairs                 */
  ildl_info_t ildl;    /* preconditioner statistics                           */
  int64_t kernel_launches;  /* GPU kernels launched by the solve (incl. setup
                               upload and the final Rayleigh–Ritz)            */
  int precond_calls;   /* preconditioner applications in the inner solves    */
  double precond_ms;   /* their device time (CUDA events on the stream)      */
  int stencil_calls;   /* inner-solve stencil applications                   */
  double stencil_ms;   /* their device time                                  */
  double basis_orth_error; /* max |V^T V - I| over the final search space
                              (jd_solve; 0 for jd_lanczos_solve)             */
} jd_stats;

/* Fill *p with the defaults (all fields zero except ildl = ildl defaults). */
int jd_params_default(jd_params* p);

/*
 * jd_solve -- the k eigenpairs of A (the lattice h) nearest sigma.
 *
 * Jacobi–Davidson (Section 4.2): the search space V is expanded by the
 * approximate solution of the correction equation (4.1),
 *   (I - Q~Q~^T)(A - theta^ I)(I - Q~Q~^T) z = -r,  Q~ = [Q, u],
 * obtained by simplified QMR with the projected preconditioner
 * K^{-1} - W (Q~^T W)^{-1} W^T, W = K^{-1} Q~, K ~ A - sigma I the
 * multilevel ILDL^T; each new vector is orthogonalised against [Q, V]
 * (classical Gram–Schmidt, twice), the target pair is extracted from span(V)
 * (harmonic Ritz by default, standard Ritz on request; the eigenvalue is
 * the Rayleigh quotient), and it is locked into Q once
 * ||A u - theta u|| <= tol*||A||
 * (||A|| = 6 + max|eps|).  A final Rayleigh–Ritz step on Q returns the
 * eigenvalues.
 *
 *   sigma   target shift (finite).
 *   k       number of eigenpairs, 1 <= k <= 64 and k < n.
 *   tol     relative residual tolerance, > 0 (e.g. 1e-8).
 *   p       parameters or NULL for defaults.
 *   evals   caller buffer of k doubles (host or device pointer).
 *   evecs   caller buffer of n*k doubles, column-major (host or device
 *           pointer), or NULL to skip the eigenvectors.
 *   st      optional statistics.
 *   stream  cudaStream_t or NULL.  The call is synchronous.
 * Results are ordered by |lambda - sigma| ascending (ties: lambda
 * ascending); each eigenvector has unit 2-norm and its largest-modulus
 * component (lowest index on ties) positive.
 * Errors: JD_EINVAL, JD_ENOMEM, JD_EDEVICE, JD_ESETUP; JD_ENOCONV when
 * max_outer steps did not converge all k pairs -- evals/evecs then hold the
 * st->nconv converged pairs first.
 */
int jd_solve(anderson_t h, double sigma, int k, double tol, const jd_params* p, double* evals,
             double* evecs, jd_stats* st, void* stream);

/*
 * jd_lanczos_solve -- the same problem as jd_solve by the paper's other
 * method (Section 4.1): shift-and-invert Lanczos, the Lanczos vectors of
 * (A - sigma I)^{-1} (Eq. (4.2)), each product a preconditioned SQMR solve
 * with the same multilevel ILDL^T (Section 7: stopped at relative residual
 * 1e-10).  Full reorthogonalisation replaces implicit restarts: at most
 * p->jmax (<= 64; 0 = 64) Lanczos vectors.  k + guard Ritz pairs with the
 * largest |nu| (lambda = sigma + 1/nu) are taken once their residual
 * estimates fall below tol ||A||, then pass the final Rayleigh-Ritz and the
 * explicit residual check of jd_solve; outputs, ordering and conventions as
 * jd_solve (k <= 60).  Uses from *p: precision (of the inner solve), seed,
 * guard, jmax, max_inner (at least 2000 here), inner_floor (the inner
 * relative tolerance; 0 = 1e-10), ildl, precond.  jd_stats: outer_its =
 * Lanczos steps, inner_its = SQMR iterations.  With JD_FP32 the inner
 * tolerance defaults to 1e-6 (binary32 SQMR stalls there), which bounds the
 * attainable accuracy; use JD_FP64 or JD_MIXED.  JD_ENOCONV when the Ritz
 * estimates did not converge within jmax steps (outputs hold the best
 * pairs).
 */
int jd_lanczos_solve(anderson_t h, double sigma, int k, double tol, const jd_params* p, double* evals,
                     double* evecs, jd_stats* st, void* stream);

/*
 * jd_solve_batch -- jd_solve for nprob independent problems (disorder
 * realisations, shifts, k; the paper's physics needs "many realizations",
 * Section 3), pipelined: `setup_threads` host threads build the
 * preconditioners of later problems (the host part of the setup, each with
 * its share of the OpenMP threads, and the device part on its own stream)
 * while the calling thread solves earlier problems on `stream`.  At most
 * setup_threads + 1 factors are alive at once.
 *   hs[nprob], sigma[nprob], k[nprob]   the problems (each as for jd_solve);
 *   evals[i]   caller buffer of k[i] doubles; evecs NULL or evecs[i] a buffer
 *              of n_i * k[i] doubles (host or device pointers);
 *   stats      NULL or nprob entries; setup_ms is each problem's build time.
 *   setup_threads  concurrent builds (0 = 2).
 * p->precond must be NULL.  Returns JD_OK, JD_ENOCONV if some problem did
 * not converge (its stats say how far it got; the others complete), or the
 * first fatal error (the remaining problems are abandoned).
 */
int jd_solve_batch(const anderson_t* hs, int nprob, const double* sigma, const int* k, double tol,
                   const jd_params* p, double* const* evals, double* const* evecs, jd_stats* stats,
                   int setup_threads, void* stream);

/* ------------------------------------------------------------------ serving
 * A request loop for many independent eigensolves of different sizes (the
 * paper's physics needs many lattices, disorder strengths and energies,
 * Sections 3 and 8; it has no serving layer of its own).  Requests are
 * admitted in arrival order while the device memory they are estimated to
 * need fits the budget; `setup_threads` host threads build their potentials
 * and preconditioners, and `slots` host threads solve admitted problems
 * concurrently, each on its own CUDA stream, so that the device work of
 * several requests overlaps (continuous batching: a request starts as soon
 * as a build finishes and a slot is free, not when a batch fills).  The
 * grid-wide preconditioner applies of concurrent solves are ordered on the
 * device one after another; all other kernels overlap.  Each request is the
 * computation jd_solve does for (anderson_create(L, W, seed, bc), sigma, k,
 * tol) with the server's jd_params, so its result does not depend on what
 * else is running.
 */
typedef struct jd_server_s* jd_server_t;

typedef struct {
  size_t hbm_budget;  /* bytes of device memory the requests may hold at once
                         (estimated per request, see jd_server_estimate);
                         0 = 80% of the free device memory at creation */
  int slots;          /* concurrent solves, 1..64 (0 = 4) */
  int setup_threads;  /* concurrent preconditioner builds, 1..64 (0 = 2) */
  jd_params solve;    /* parameters of every solve; solve.precond must be NULL */
} jd_server_params;

#define JD_SUBMIT_VECTORS 1 /* keep the eigenvectors for jd_poll */

typedef struct {
  int64_t submitted, completed, failed; /* requests */
  int queued, building, ready, solving; /* requests in each state now */
  int peak_solving;                     /* most solves that ran at once */
  size_t hbm_budget, reserved_bytes, peak_reserved_bytes;
} jd_server_info;

/* Defaults as documented above (solve = jd_params_default). */
int jd_server_params_default(jd_server_params* p);

/* Device-memory estimate that admission charges a request of an L^3 lattice
 * with k eigenpairs: potential, the three device copies of a factor of
 * typical fill (and its dense tail), and the solver's search space.  */
int jd_server_estimate(int L, int k, size_t* bytes);

/* Start the worker threads on the current device.  Errors: JD_EINVAL (bad
 * parameters), JD_EDEVICE. */
int jd_server_create(const jd_server_params* p, jd_server_t* out);

/* Queue a request; *ticket identifies it in jd_poll/jd_wait.  Arguments are
 * checked as by anderson_create and jd_solve (JD_EINVAL); a request whose
 * estimate exceeds the whole budget is rejected with JD_ENOMEM. */
int jd_submit(jd_server_t srv, int L, double W, uint64_t seed, int bc, double sigma, int k, double tol, int flags,
              uint64_t* ticket);

/* JD_EAGAIN while the request is queued, building or solving.  Otherwise
 * the request's own status (JD_OK, JD_ENOCONV with the converged prefix,
 * or an error) is returned, evals[k] (caller buffer, may be NULL), evecs
 * (n x k column-major, caller buffer, only with JD_SUBMIT_VECTORS, may be
 * NULL), *st and *latency_ms (submission to completion, may be NULL) are
 * filled, and the ticket is retired.  Unknown ticket: JD_EINVAL. */
int jd_poll(jd_server_t srv, uint64_t ticket, double* evals, double* evecs, jd_stats* st, double* latency_ms);

/* jd_poll that blocks until the request completes or timeout_s seconds
 * pass (JD_EAGAIN then); timeout_s < 0 waits without limit. */
int jd_wait(jd_server_t srv, uint64_t ticket, double* evals, double* evecs, jd_stats* st, double* latency_ms,
            double timeout_s);

int jd_server_info_get(jd_server_t srv, jd_server_info* info);

/* Stop: queued requests are dropped, solves in flight finish, every handle
 * and buffer of the server is released.  NULL is a no-op. */
int jd_server_destroy(jd_server_t srv);

#ifdef __cplusplus
}
#endif
#endif /* ANDERSON_JD_H */
