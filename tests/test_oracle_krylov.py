"""Pins for the oracle's SQMR, projections, CGS2 and Rayleigh–Ritz."""
import numpy as np
import pytest

from oracle import krylov, lattice, rng


def _sym_indefinite(n, seed):
    g = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((n, n)))
    w = np.concatenate([g.uniform(-3, -0.5, n // 2), g.uniform(0.5, 3, n - n // 2)])
    return (Q * w) @ Q.T


def test_sqmr_exact_preconditioner_one_step():
    A = _sym_indefinite(30, 1)
    b = np.random.default_rng(2).standard_normal(30)
    Ainv = np.linalg.inv(A)
    x, k, _ = krylov.sqmr(lambda v: A @ v, lambda v: Ainv @ v, b, 1e-12, 10)
    assert k <= 2
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-10)


def test_sqmr_unpreconditioned_converges_and_bound_holds():
    n = 40
    A = _sym_indefinite(n, 3)
    b = np.random.default_rng(4).standard_normal(n)
    x, k, hist = krylov.sqmr(lambda v: A @ v, lambda v: v, b, 1e-11, 200)
    assert np.linalg.norm(A @ x - b) <= 1e-9 * np.linalg.norm(b)
    # quasi-residual bound ||b - A x_j|| <= sqrt(j+1) tau_j at every step
    for j in range(1, min(k, 15)):
        xj, _, h = krylov.sqmr(lambda v: A @ v, lambda v: v, b, 0.0, j)
        assert np.linalg.norm(b - A @ xj) <= np.sqrt(j + 1) * h[-1] * (1 + 1e-10)


def test_sqmr_indefinite_preconditioner_on_anderson():
    """A symmetric indefinite preconditioner (exact inverse of a perturbed
    shifted matrix) on an Anderson system."""
    L = 5
    eps = rng.potential(L, 16.5, 2)
    A = lattice.dense(L, eps)
    M = np.linalg.inv(A + 0.05 * np.diag(np.random.default_rng(1).standard_normal(L ** 3)))
    b = np.random.default_rng(9).standard_normal(L ** 3)
    x, k, _ = krylov.sqmr(lambda v: A @ v, lambda v: M @ v, b, 1e-10, 300)
    assert np.linalg.norm(A @ x - b) <= 1e-8 * np.linalg.norm(b)


def test_projected_operators():
    L = 4
    eps = rng.potential(L, 16.5, 5)
    A = lattice.dense(L, eps)
    n = L ** 3
    g = np.random.default_rng(0)
    Qt, _ = np.linalg.qr(g.standard_normal((n, 3)))
    K = np.linalg.inv(A + 0.3 * np.eye(n))
    Aop, Mop = krylov.projected_operators(lambda v: A @ v - 0.1 * v, lambda v: K @ v, Qt)
    y = Mop(g.standard_normal(n))
    assert np.abs(Qt.T @ y).max() < 1e-12
    a, b = g.standard_normal(n), g.standard_normal(n)
    assert a @ Aop(b) == pytest.approx(b @ Aop(a), rel=1e-12)
    assert a @ Mop(b) == pytest.approx(b @ Mop(a), rel=1e-10)


def test_cgs2_orthogonality():
    g = np.random.default_rng(1)
    V, _ = np.linalg.qr(g.standard_normal((200, 20)))
    t = V @ g.standard_normal(20) + 1e-6 * g.standard_normal(200)
    v, nrm, h = krylov.cgs2(V, t)
    assert np.abs(V.T @ v).max() < 1e-14
    assert np.linalg.norm(v) == pytest.approx(1.0)


def test_rayleigh_ritz_exact_and_interlacing():
    L = 4
    eps = rng.potential(L, 12.0, 8)
    A = lattice.dense(L, eps)
    w, X = np.linalg.eigh(A)
    th, Y = krylov.rayleigh_ritz(X[:, 10:15], A @ X[:, 10:15], 0.0)
    assert np.allclose(np.sort(th), w[10:15], atol=1e-12)
    g = np.random.default_rng(3)
    V, _ = np.linalg.qr(g.standard_normal((L ** 3, 8)))
    th, _ = krylov.rayleigh_ritz(V, A @ V, 0.0)
    th = np.sort(th)
    n, m = L ** 3, 8
    for i in range(m):  # Cauchy interlacing
        assert w[i] - 1e-12 <= th[i] <= w[n - m + i] + 1e-12
