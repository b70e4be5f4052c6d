"""Shift-and-invert Lanczos with full reorthogonalisation (oracle side).

Section 4.1 applies Lanczos to (A - sigma I)^{-1} instead of A: the
eigenvalues of A nearest sigma become the largest-modulus eigenvalues
nu = 1/(lambda - sigma) of the inverse, which Lanczos finds first.  The
paper's production code (implicitly restarted ARPACK over PARDISO) is a
comparison system and is not restated here; this is the plain method:

* (A - sigma I) is factored once by a sparse direct LU (SuperLU through
  scipy, a library routine), with a symmetric fill-reducing ordering and
  no pivoting so that the same factor also yields the inertia;
* the three-term recurrence beta_{j+1} v_{j+1} = Op v_j - alpha_j v_j -
  beta_j v_{j-1} (the recursion of Eq. (3.1) applied to Op = (A - sigma
  I)^{-1}) is run with two passes of full Gram–Schmidt against all previous
  Lanczos vectors, so no spurious copies arise;
* every few steps the tridiagonal T_j is diagonalised, the Ritz vectors of
  the k + guard largest |nu| are formed and their explicit residuals
  ||A x - lambda x|| with lambda = x^T A x are checked against tol*||A||.
"""
import numpy as np
import scipy.sparse.linalg as spl

from .eig import order_nearest, normalize_sign


def factor_shifted(A, sigma):
    """Sparse LU of A - sigma I without pivoting and with a symmetric
    ordering, so that P (A - sigma I) P^T = L U with U = D L^T."""
    n = A.shape[0]
    import scipy.sparse as sp
    M = (A - sigma * sp.identity(n, format="csr")).tocsc()
    return spl.splu(M, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                    options=dict(SymmetricMode=True))


def shift_invert_nearest(A, sigma, k, tol=1e-12, norm_a=None, seed=12345,
                         max_steps=None, guard=4, factor=None):
    """k eigenpairs of the sparse symmetric A nearest sigma.

    Returns (evals, evecs, info) with evals ordered by |lambda - sigma|
    (ties by lambda) and evecs normalised as in :mod:`oracle.eig`.
    ``info`` holds the Lanczos step count and the explicit residuals.
    """
    n = A.shape[0]
    if norm_a is None:
        norm_a = float(abs(A).sum(axis=1).max())
    lu = factor if factor is not None else factor_shifted(A, sigma)
    if max_steps is None:
        max_steps = min(n, max(300, 20 * k + 100))
    rng = np.random.default_rng(seed)
    Q = np.zeros((n, max_steps + 1))
    q = rng.standard_normal(n)
    Q[:, 0] = q / np.linalg.norm(q)
    alpha = np.zeros(max_steps)
    beta = np.zeros(max_steps)
    want = min(k + guard, n)
    result = None
    for j in range(max_steps):
        w = lu.solve(Q[:, j])
        alpha[j] = Q[:, j] @ w
        w -= alpha[j] * Q[:, j]
        if j > 0:
            w -= beta[j - 1] * Q[:, j - 1]
        for _ in range(2):
            w -= Q[:, :j + 1] @ (Q[:, :j + 1].T @ w)
        beta[j] = np.linalg.norm(w)
        steps = j + 1
        done_space = beta[j] <= 1e-300 or steps == n
        if not done_space:
            Q[:, j + 1] = w / beta[j]
        if steps >= want and (steps % 5 == 0 or done_space or steps == max_steps):
            T = np.diag(alpha[:steps]) + np.diag(beta[:steps - 1], 1) + np.diag(beta[:steps - 1], -1)
            nu, S = np.linalg.eigh(T)
            pick = np.argsort(-np.abs(nu))[:want]
            X = Q[:, :steps] @ S[:, pick]
            AX = A @ X
            lam = np.einsum("ij,ij->j", X, AX) / np.einsum("ij,ij->j", X, X)
            res = np.linalg.norm(AX - X * lam, axis=0) / np.linalg.norm(X, axis=0)
            order = order_nearest(lam, sigma)[:k]
            if np.all(res[order] <= tol * norm_a) or done_space or steps == max_steps:
                result = (lam[order], X[:, order], res[order], steps)
                break
    lam, X, res, steps = result
    return lam, normalize_sign(X), {"steps": steps, "residuals": res}
