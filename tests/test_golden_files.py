"""The stored oracle eigenpairs of the L = 50 workload (tests/golden/
anderson_L50_*) belong to their lattices and are eigenpairs of them: checks
that need no GPU and do not rerun the oracle's Lanczos."""
import os

import numpy as np
import pytest

from oracle import lattice, rng

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
L, W = 50, 16.5


def _load(seed):
    from pairs import load_golden_L50
    return load_golden_L50(seed)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_stored_eigenvalues_consistent(seed):
    nA, ev, res = _load(seed)
    eps = rng.potential(L, W, seed)
    assert nA == lattice.norm_bound(eps)        # the file belongs to this lattice
    assert len(ev) == 6
    assert np.all(np.diff(np.abs(ev)) >= 0)      # ordered by distance to sigma = 0
    assert np.abs(ev).max() <= 6 + W / 2         # Gershgorin (Section 3)
    assert res.max() <= 1e-11                    # the oracle's residuals


def test_stored_vectors_are_eigenvectors():
    """Seed 1's stored binary32 eigenvectors: Rayleigh quotients equal the
    stored eigenvalues to rounding, residuals at the binary32 level,
    orthonormal to binary32 rounding."""
    nA, ev, _ = _load(1)
    d = np.load(os.path.join(GOLDEN, "anderson_L50_W16.5_sigma0_seed1_vectors.npz"))
    X = d["X"].astype(np.float64)
    assert X.shape == (L ** 3, 5)
    assert np.array_equal(d["evals"], ev[:5])
    A = lattice.assemble(L, rng.potential(L, W, 1))
    AX = A @ X
    nrm2 = np.einsum("ij,ij->j", X, X)
    rq = np.einsum("ij,ij->j", X, AX) / nrm2
    assert np.abs(rq - ev[:5]).max() <= 1e-11 * nA
    assert (np.linalg.norm(AX - X * rq, axis=0) / np.sqrt(nrm2)).max() <= 1e-6 * nA
    G = X.T @ X
    assert np.abs(G - np.eye(5)).max() <= 1e-6
