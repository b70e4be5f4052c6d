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


def check_pairs_certified(L, W, seed, bc, sigma, k, ev, X, st, tol):
    """Pairs of an inexact solve (a binary32 inner solve whose operator is
    only about 1e-6 accurate), checked against the dense oracle with bounds
    derived from each pair's own explicit residual r_j = A x_j - lambda_j x_j
    and the oracle's gap g_j between lambda_j's eigenvalue and the rest of
    the spectrum:
      |lambda_j - lambda_j(oracle)| <= 2 ||r_j||^2 / g_j + 1e-12 ||A||
        (Kato-Temple: a Rayleigh quotient's error is quadratic in ||r||),
      sin angle(x_j, oracle eigenvector) <= 2 ||r_j|| / g_j  (Davis-Kahan),
      ||r_j|| <= 2 tol ||A||, orthonormality, ordering and signs."""
    eps = rng.potential(L, W, seed)
    A = lattice.assemble(L, eps, bc)
    nA = lattice.norm_bound(eps)
    w_all, V_all = np.linalg.eigh(A.toarray())
    o = eig.order_nearest(w_all, sigma)
    wl, Vl = w_all[o[:k]], eig.normalize_sign(V_all[:, o[:k]])
    assert st["nconv"] == k and st["status"] == 0
    res = np.linalg.norm(A @ X - X * ev, axis=0)
    assert res.max() <= 2 * tol * nA, (res / nA, tol)
    assert np.abs(X.T @ X - np.eye(k)).max() <= 1e-12
    for j in range(k):
        others = np.delete(w_all, o[j])
        gap = np.abs(others - wl[j]).min()
        assert abs(ev[j] - wl[j]) <= 2 * res[j] ** 2 / gap + 1e-12 * nA, (j, ev[j] - wl[j], res[j], gap)
        cosang = min(1.0, abs(X[:, j] @ Vl[:, j]))
        assert np.sqrt(max(0.0, 1 - cosang * cosang)) <= max(1e-6, 2 * res[j] / gap), j
        i = int(np.argmax(np.abs(X[:, j])))
        assert X[i, j] > 0
    assert np.all(np.diff(np.abs(ev - sigma)) >= 0)


def load_golden_L50(seed):
    """(||A||, eigenvalues, oracle residuals) of the stored L = 50 oracle
    eigenpairs of one disorder seed (tests/golden/make_anderson_L50.py)."""
    import os
    nA, ev, res = None, [], []
    name = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "anderson_L50_W16.5_sigma0_seed%d.txt" % seed)
    with open(name) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == "norm_A":
                nA = float(parts[1])
            else:
                ev.append(float(parts[0]))
                res.append(float(parts[1]))
    return nA, np.array(ev), np.array(res)
