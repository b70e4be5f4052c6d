"""Dense eigensolvers and the "k eigenpairs nearest sigma" selection.

The method's result is defined by the problem statement: the few
eigenvalues of A closest to a shift (lambda = 0 in every table; Sections 3
and 7) and their eigenvectors.  Readings used project-wide:

* order by |lambda - sigma| ascending, ties by lambda ascending;
* each eigenvector has unit 2-norm and its largest-modulus component is
  positive (lowest index among equal moduli).
"""
import numpy as np


def jacobi_eigh(A, tol=1e-14, max_sweeps=60):
    """Cyclic-by-row Jacobi eigenvalue algorithm on a dense symmetric matrix.

    Each (p, q) step applies the 2x2 symmetric Schur rotation that zeroes
    a_pq: with tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| +
    sqrt(1 + tau^2)), c = 1/sqrt(1+t^2), s = t c, A <- J^T A J and V <- V J.
    Sweeps repeat until off(A) <= tol * ||A||_F.  Returns (w, V), unsorted
    eigenvalues and the accumulated orthogonal V.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    fro = np.linalg.norm(A)
    if n <= 1 or fro == 0.0:
        return np.diag(A).copy(), V
    for _ in range(max_sweeps):
        off = np.sqrt(max(np.sum(A * A) - np.sum(np.diag(A) ** 2), 0.0))
        if off <= tol * fro:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if abs(apq) <= 1e-300 * max(1.0, abs(A[p, p]), abs(A[q, q])):
                    continue
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                if abs(tau) > 1e150:
                    t = 0.5 / tau
                elif tau >= 0.0:
                    t = 1.0 / (tau + np.sqrt(1.0 + tau * tau))
                else:
                    t = -1.0 / (-tau + np.sqrt(1.0 + tau * tau))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                cp = A[:, p].copy()
                cq = A[:, q].copy()
                A[:, p] = c * cp - s * cq
                A[:, q] = s * cp + c * cq
                rp = A[p, :].copy()
                rq = A[q, :].copy()
                A[p, :] = c * rp - s * rq
                A[q, :] = s * rp + c * rq
                vp = V[:, p].copy()
                vq = V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
    return np.diag(A).copy(), V


def order_nearest(evals, sigma):
    """Indices sorting eigenvalues by |lambda - sigma|, ties by lambda."""
    evals = np.asarray(evals, dtype=np.float64)
    return np.lexsort((evals, np.abs(evals - sigma)))


def normalize_sign(X):
    """Unit columns whose largest-|x_i| entry (first such index) is positive."""
    X = np.array(X, dtype=np.float64, copy=True)
    if X.ndim == 1:
        X = X[:, None]
    for j in range(X.shape[1]):
        X[:, j] /= np.linalg.norm(X[:, j])
        i = int(np.argmax(np.abs(X[:, j])))
        if X[i, j] < 0:
            X[:, j] = -X[:, j]
    return X


def nearest_dense(A, sigma, k, solver="lapack"):
    """The k eigenpairs of the dense symmetric A nearest sigma.

    ``solver='lapack'`` uses numpy.linalg.eigh (a library routine);
    ``solver='jacobi'`` uses :func:`jacobi_eigh` above.
    """
    if solver == "jacobi":
        w, V = jacobi_eigh(A)
    else:
        w, V = np.linalg.eigh(np.asarray(A, dtype=np.float64))
    order = order_nearest(w, sigma)[:k]
    return w[order], normalize_sign(V[:, order])
