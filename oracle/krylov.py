"""Plain restatements of the Krylov pieces of the Jacobi–Davidson hot path.

* :func:`sqmr` -- the simplified (symmetric) QMR method of Freund and
  Nachtigal / Freund and Jarre that Section 4.2 uses for the correction
  equation: it needs a symmetric system matrix and a symmetric (possibly
  indefinite) preconditioner and runs the coupled two-term recurrences
      t = A q, sigma = q^T t, alpha = rho / sigma, r -= alpha t,
      theta_k = ||r|| / tau_{k-1}, c = 1/sqrt(1 + theta_k^2),
      tau_k = tau_{k-1} theta_k c,
      d = c^2 theta_{k-1}^2 d + c^2 alpha q, x += d,
      u = M r, rho' = r^T u, beta = rho'/rho, q = u + beta q,
  with the quasi-residual bound ||b - A x_k|| <= sqrt(k + 1) tau_k.
* :func:`projected_operators` -- the projected system matrix
  (I - Q Q^T)(A - theta I)(I - Q Q^T) of Eq. (4.1) (with Q = [Q_locked, u])
  and the projected preconditioner K^{-1} - W (Q^T W)^{-1} W^T, W = K^{-1} Q
  (Section 4.2; the symmetric form, see the readings in the design notes).
* :func:`cgs2` -- classical Gram–Schmidt run twice against an orthonormal
  basis, then normalisation.
* :func:`rayleigh_ritz` -- Ritz pairs of A on span(V): eigenpairs of V^T A V
  ordered by distance to a target.
"""
import numpy as np

from .eig import order_nearest


def sqmr(Aop, Mop, b, tol, maxit, x0=None):
    """Solve A x = b approximately; stop when sqrt(k+1) tau_k <= tol ||b||.

    Returns (x, iterations, tau_history)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - Aop(x) if x0 is not None else b.copy()
    tau = np.linalg.norm(r)
    q = Mop(r)
    theta = 0.0
    rho = r @ q
    d = np.zeros_like(b)
    nb = np.linalg.norm(b)
    hist = [tau]
    if nb == 0.0:
        return x, 0, hist
    for k in range(1, maxit + 1):
        t = Aop(q)
        sigma = q @ t
        if sigma == 0.0 or rho == 0.0:
            return x, k - 1, hist
        alpha = rho / sigma
        r = r - alpha * t
        theta_old = theta
        theta = np.linalg.norm(r) / tau
        c = 1.0 / np.sqrt(1.0 + theta * theta)
        tau = tau * theta * c
        d = (c * c * theta_old * theta_old) * d + (c * c * alpha) * q
        x = x + d
        hist.append(tau)
        if np.sqrt(k + 1.0) * tau <= tol * nb:
            return x, k, hist
        u = Mop(r)
        rho_new = r @ u
        beta = rho_new / rho
        rho = rho_new
        q = u + beta * q
    return x, maxit, hist


def projected_operators(A_shift_op, Kinv_op, Qt):
    """(Aop, Mop) of the projected correction equation for the orthonormal
    columns Qt = [Q_locked, u]."""
    Qt = np.asarray(Qt, dtype=np.float64)
    if Qt.ndim == 1:
        Qt = Qt[:, None]
    W = np.column_stack([Kinv_op(Qt[:, j]) for j in range(Qt.shape[1])])
    M = Qt.T @ W

    def proj(v):
        return v - Qt @ (Qt.T @ v)

    def Aop(v):
        return proj(A_shift_op(proj(v)))

    def Mop(v):
        y = Kinv_op(v)
        return y - W @ np.linalg.solve(M, Qt.T @ y)

    return Aop, Mop


def cgs2(V, t):
    """Orthogonalise t against the orthonormal columns of V twice (classical
    Gram–Schmidt) and normalise.  Returns (v, norm_after, h_total)."""
    V = np.asarray(V, dtype=np.float64)
    t = np.array(t, dtype=np.float64)
    h_total = np.zeros(V.shape[1])
    for _ in range(2):
        h = V.T @ t
        t = t - V @ h
        h_total += h
    nrm = np.linalg.norm(t)
    return t / nrm, nrm, h_total


def rayleigh_ritz(V, AV, sigma):
    """Ritz values/vectors of A on span(V) (orthonormal V, AV = A V), ordered
    by |theta - sigma| then theta."""
    H = V.T @ AV
    H = 0.5 * (H + H.T)
    w, Y = np.linalg.eigh(H)
    o = order_nearest(w, sigma)
    return w[o], Y[:, o]
