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

/* ---- boundary conditions and precisions -------------------------------- */
#define JD_PERIODIC 0 /* x_{M+1} = x_1 (the default of every table)           */
#define JD_HARDWALL 1 /* x_0 = x_{M+1} = 0 (Section 7, Table 6)               */

#define JD_FP64 0  /* arithmetic in binary64                                  */
#define JD_FP32 1  /* arithmetic in binary32 (vectors and potential in FP32)  */

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

#ifdef __cplusplus
}
#endif
#endif /* ANDERSON_JD_H */
