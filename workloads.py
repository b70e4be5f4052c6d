"""Seeded synthetic workloads shared by the tests and ``bench.py``.

This module holds only recipes and seeded random inputs (lattice sizes,
disorder strengths, shifts, seeds, random test vectors).  It contains none
of the method's arithmetic: the disorder potential itself is generated by
the library on the device and, independently, by the oracle.

Workloads (all synthetic 3D Anderson lattices, the paper's own problem
class; there is no external dataset):

* ``tiny``   L = 10, W = 16.5, periodic, sigma = 0, k = 5, seed 1.
* ``mid``    L = 50, W = 16.5, periodic, sigma = 0, k = 5, seeds 1..3.
* ``large``  L = 100, W = 16.5, periodic, sigma = 0, k = 5, seeds 1..3:
             the headline size of Table 4 (M = 100, w = w_c = 16.5,
             five eigenvalues closest to 0).
* ``batch``  256 problems, L in {20,30,40,50}, W in {12,16.5,20},
             sigma in {-1,0,1}, k = 5, problem p has seed 1000 + p; the
             choices are drawn from numpy's PCG64 seeded 42.
* ``serve``  4096 requests with Poisson arrivals, L in [16,120],
             W in [8,24], sigma in [-2,2], k in {1,5,10}; request r has
             seed 10**6 + r; driver seed 7.
"""
import numpy as np

W_CRITICAL = 16.5

TINY = dict(name="anderson-L10-W16.5-periodic-k5", L=10, W=16.5, bc=0, sigma=0.0, k=5, seeds=(1,))
MID = dict(name="anderson-L50-W16.5-periodic-k5", L=50, W=16.5, bc=0, sigma=0.0, k=5, seeds=(1, 2, 3))
LARGE = dict(name="anderson-L100-W16.5-periodic-k5", L=100, W=16.5, bc=0, sigma=0.0, k=5, seeds=(1, 2, 3))


def random_vector(n, seed, dtype=np.float64):
    """Standard-normal test vector of length n from PCG64(seed)."""
    return np.random.default_rng(seed).standard_normal(n).astype(dtype)


def random_block(n, m, seed, dtype=np.float64):
    """n x m column-major-friendly block (returned C-contiguous as m x n,
    i.e. one row per column vector)."""
    return np.random.default_rng(seed).standard_normal((m, n)).astype(dtype)


def batch_recipe(nprob=256, seed=42):
    """Problem list of the batched workload: dicts with L, W, sigma, k,
    seed, bc."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice([20, 30, 40, 50], size=nprob)
    Ws = rng.choice([12.0, 16.5, 20.0], size=nprob)
    ss = rng.choice([-1.0, 0.0, 1.0], size=nprob)
    return [dict(L=int(Ls[p]), W=float(Ws[p]), sigma=float(ss[p]), k=5,
                 seed=1000 + p, bc=0) for p in range(nprob)]


def serve_recipe(nreq=4096, rate_per_s=1.0, seed=7, lmax=120):
    """Request stream of the serving workload: dicts with arrival time
    (seconds, Poisson process of the given rate), L, W, sigma, k, seed.
    ``lmax`` < 120 gives a bounded sample (L uniform in 16..lmax)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=nreq)
    t = np.cumsum(gaps)
    Ls = rng.integers(16, lmax + 1, size=nreq)
    Ws = rng.uniform(8.0, 24.0, size=nreq)
    ss = rng.uniform(-2.0, 2.0, size=nreq)
    ks = rng.choice([1, 5, 10], size=nreq)
    return [dict(t=float(t[r]), L=int(Ls[r]), W=float(Ws[r]), sigma=float(ss[r]),
                 k=int(ks[r]), seed=10 ** 6 + r, bc=0) for r in range(nreq)]
