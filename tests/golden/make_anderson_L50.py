#!/usr/bin/env python3
"""Writes the stored oracle eigenpairs of the mid-size workload.

Workload: L = 50 (n = 125,000) periodic Anderson lattices, W = 16.5, the
eigenvalues nearest sigma = 0 (the problem of Section 3 and Table 4 at
M = 50), disorder seeds 1, 2, 3.  For each seed it writes
``anderson_L50_W16.5_sigma0_seed<s>.txt`` with the k + 1 = 6 eigenvalues of
A nearest sigma (five asked for plus one guard, so that the gap behind the
fifth is known), ||A|| = 6 + max|eps| and the oracle's own explicit
residuals; with ``--vectors`` also ``..._seed<s>_vectors.npz``, the five
nearest eigenvectors rounded to binary32 (normalised, largest-modulus entry
positive), for subspace-angle checks.  Only ``oracle/`` is called: the
potential by ``oracle.rng``, the matrix by ``oracle.lattice`` and the
eigenpairs by the shift-and-invert Lanczos of ``oracle.lanczos``
(Section 4.1), run for its full 300 steps (residuals near 1e-12 ||A||,
recorded in the file).

Usage: python tests/golden/make_anderson_L50.py [--seeds 1 2 3] [--vectors]
(about 10 minutes per seed on an 8-core host).
"""
import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import lanczos, lattice, rng  # noqa: E402

L, W, SIGMA, K_STORED, K_VECTORS = 50, 16.5, 0.0, 6, 5


def path(seed, vectors=False):
    stem = os.path.join(HERE, "anderson_L%d_W%g_sigma0_seed%d" % (L, W, seed))
    return stem + ("_vectors.npz" if vectors else ".txt")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, nargs="+", default=[1, 2, 3])
    ap.add_argument("--vectors", action="store_true")
    args = ap.parse_args()
    for seed in args.seeds:
        eps = rng.potential(L, W, seed)
        A = lattice.assemble(L, eps)
        nA = lattice.norm_bound(eps)
        t0 = time.perf_counter()
        ev, X, info = lanczos.shift_invert_nearest(A, SIGMA, K_STORED, tol=1e-13, norm_a=nA)
        dt = time.perf_counter() - t0
        res = np.asarray(info["residuals"]) / nA
        print("seed %d: %.1f s, %d Lanczos steps, max residual %.2e" % (seed, dt, info["steps"], res.max()),
              flush=True)
        lines = [
            "# Eigenvalues of the 3D Anderson matrix nearest sigma = 0, written by",
            "# tests/golden/make_anderson_L50.py from the oracle alone (shift-and-invert",
            "# Lanczos over a sparse LU, Section 4.1).",
            "# Lattice: L = 50 periodic, W = 16.5, disorder seed %d (box distribution of" % seed,
            "# Section 3, SplitMix64 stream of the seed), hopping -1.",
            "norm_A %r" % float(nA),
            "# lambda (ordered by |lambda - sigma|; 5 asked for + 1 guard) and the oracle's",
            "# relative residual ||A x - lambda x|| / ||A||",
        ]
        lines += ["%r %.3e" % (float(v), r) for v, r in zip(ev, res)]
        with open(path(seed), "w") as f:
            f.write("\n".join(lines) + "\n")
        if args.vectors:
            np.savez_compressed(path(seed, True), X=X[:, :K_VECTORS].astype(np.float32),
                                evals=ev[:K_VECTORS])


if __name__ == "__main__":
    main()
