// Entry points of the Jacobi–Davidson solver for other translation units.
#pragma once
#include "anderson_impl.cuh"
#include "ildl_impl.cuh"

namespace ajd {

// jd_params with defaults filled in and checked (JD_EINVAL on bad values).
int normalize_jd_params(const jd_params* p, jd_params& prm);

// One solve of (h, sigma, k, tol) with the prebuilt preconditioner pc on
// stream s; prm must be normalised.  Arguments as for jd_solve.
int solve_problem(anderson_s* h, ildl_s* pc, const jd_params& prm, double sigma, int k, double tol, double* evals,
                  double* evecs, jd_stats* st, cudaStream_t s);

// Serialise the persistent preconditioner applies launched by the calling
// thread with those of every other thread that set it (a device-side chain
// of events): used by threads that solve concurrently on their own streams.
void set_apply_serialization(bool on);
bool apply_serialization();

}  // namespace ajd
