"""Checks of computed eigenpairs against the oracle, shared by the GPU tests."""
import numpy as np

from oracle import eig, lanczos, lattice, rng


def check_pairs(L, W, seed, bc, sigma, k, ev, X, st, tol, oracle="dense"):
    eps = rng.potential(L, W, seed)
    A = lattice.assemble(L, eps, bc)
    nA = lattice.norm_bound(eps)
    if oracle == "dense":
        w_all, V_all = np.linalg.eigh(A.toarray())
        o = eig.order_nearest(w_all, sigma)
        wl, Vl = w_all[o[:k]], eig.normalize_sign(V_all[:, o[:k]])
        dist = np.sort(np.abs(w_all - sigma))
    else:
        wl, Vl, _ = lanczos.shift_invert_nearest(A, sigma, k + 1, norm_a=nA)
        dist = np.sort(np.abs(wl - sigma))
        wl, Vl = wl[:k], Vl[:, :k]
    assert st["nconv"] == k and st["status"] == 0
    # eigenvalues: |dlambda| <= 1e-10 ||A||
    assert np.abs(ev - wl).max() <= 1e-10 * nA, (ev, wl)
    # residuals measured by the oracle's matrix
    res = np.linalg.norm(A @ X - X * ev, axis=0) / nA
    assert res.max() <= 2 * tol
    assert st["max_residual"] <= 2 * tol
    # orthonormality
    assert np.abs(X.T @ X - np.eye(k)).max() <= 1e-12
    # eigenvectors: angle to the oracle's, bounded by max(1e-6, 2 ||r|| / gap)
    full = np.sort(np.abs(np.concatenate([dist])))
    for j in range(k):
        gaps = np.abs(wl - wl[j])
        gaps[j] = np.inf
        gap = min(gaps.min(), abs(dist[k] - dist[k - 1]) if len(dist) > k else np.inf)
        cosang = min(1.0, abs(X[:, j] @ Vl[:, j]))
        sinang = np.sqrt(max(0.0, 1 - cosang * cosang))
        assert sinang <= max(1e-6, 2 * res[j] * nA / gap), (j, sinang)
    # sign convention
    for j in range(k):
        i = int(np.argmax(np.abs(X[:, j])))
        assert X[i, j] > 0
    assert np.all(np.diff(np.abs(ev - sigma)) >= 0)
    return full
