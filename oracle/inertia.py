"""Sylvester inertia counts (oracle side).

For a symmetric A and a real c, write P (A - c I) P^T = L D L^T with L
unit lower triangular.  By Sylvester's law of inertia the number of
negative entries of D equals the number of eigenvalues of A below c.  The
factor is SuperLU's LU with a symmetric ordering and pivoting switched off
(U = D L^T, so D = diag(U)).  Counting at c = sigma - d and c = sigma + d
gives the number of eigenvalues in [sigma - d, sigma + d), which proves
that no eigenvalue nearer sigma than d was missed by an iterative solver.
"""
import numpy as np

from .lanczos import factor_shifted


def count_below(A, c):
    """Number of eigenvalues of the sparse symmetric A strictly below c."""
    lu = factor_shifted(A, c)
    if not np.array_equal(lu.perm_r, lu.perm_c):
        raise RuntimeError("factor is not a symmetric permutation; inertia undefined")
    d = lu.U.diagonal()
    if np.any(d == 0.0):
        raise RuntimeError("zero pivot: c is (numerically) an eigenvalue")
    return int(np.sum(d < 0.0))


def count_in_window(A, lo, hi):
    """Number of eigenvalues in [lo, hi)."""
    return count_below(A, hi) - count_below(A, lo)
