"""Pins for the oracle's eigensolvers: Jacobi vs LAPACK, shift-invert Lanczos
vs dense, and inertia counts proving completeness."""
import numpy as np
import pytest

from oracle import eig, inertia, lanczos, lattice, rng
from oracle.lattice import HARDWALL, PERIODIC


@pytest.mark.parametrize("L,bc", [(3, PERIODIC), (4, PERIODIC), (5, HARDWALL), (5, PERIODIC)])
def test_jacobi_matches_lapack_full_spectrum(L, bc):
    eps = rng.potential(L, 16.5, L)
    A = lattice.dense(L, eps, bc)
    w, V = eig.jacobi_eigh(A)
    assert np.allclose(np.sort(w), np.linalg.eigvalsh(A), atol=1e-12 * lattice.norm_bound(eps))
    assert np.linalg.norm(A @ V - V * w) < 1e-11 * lattice.norm_bound(eps)
    assert np.linalg.norm(V.T @ V - np.eye(len(w))) < 1e-12


def test_jacobi_closed_form_degenerate():
    """W = 0 has large degenerate clusters; Jacobi still returns them."""
    L = 4
    A = lattice.dense(L, np.zeros(L ** 3))
    w, _ = eig.jacobi_eigh(A)
    assert np.allclose(np.sort(w), lattice.closed_form_spectrum(L), atol=1e-12)


def test_brute_force_nearest_L6():
    """Brute force at L = 6: own Jacobi and LAPACK agree on the 5 eigenpairs
    nearest 0, including eigenvector signs."""
    L = 6
    eps = rng.potential(L, 16.5, 1)
    A = lattice.dense(L, eps)
    wj, Vj = eig.nearest_dense(A, 0.0, 5, solver="jacobi")
    wl, Vl = eig.nearest_dense(A, 0.0, 5, solver="lapack")
    assert np.allclose(wj, wl, atol=1e-12)
    assert np.allclose(Vj, Vl, atol=1e-9)
    assert np.all(np.diff(np.abs(wl)) >= 0)


def test_order_nearest_ties():
    w = np.array([1.0, -1.0, 0.5, -0.25, 0.25, 3.0])
    o = eig.order_nearest(w, 0.0)
    assert list(w[o]) == [-0.25, 0.25, 0.5, -1.0, 1.0, 3.0]
    o = eig.order_nearest(w, 0.75)
    assert list(w[o][:3]) == [0.5, 1.0, 0.25]


def test_normalize_sign():
    X = np.array([[0.1, -3.0], [-2.0, 3.0], [0.5, 1.0]])
    Y = eig.normalize_sign(X)
    assert Y[1, 0] > 0 and Y[0, 1] > 0
    assert np.allclose(np.linalg.norm(Y, axis=0), 1.0)


@pytest.mark.parametrize("L,sigma,bc", [(8, 0.0, PERIODIC), (10, 0.0, PERIODIC), (9, 1.0, HARDWALL), (8, -1.0, PERIODIC)])
def test_shift_invert_matches_dense(L, sigma, bc):
    eps = rng.potential(L, 16.5, 1)
    A = lattice.assemble(L, eps, bc)
    nA = lattice.norm_bound(eps)
    wl, Vl = eig.nearest_dense(A.toarray(), sigma, 5)
    ws, Vs, info = lanczos.shift_invert_nearest(A, sigma, 5, tol=1e-12, norm_a=nA)
    assert np.allclose(ws, wl, atol=1e-12 * nA)
    assert np.allclose(Vs, Vl, atol=1e-8)
    assert np.all(info["residuals"] <= 1e-12 * nA)


@pytest.mark.parametrize("L,bc", [(5, PERIODIC), (6, HARDWALL)])
def test_inertia_matches_dense(L, bc):
    eps = rng.potential(L, 12.0, 2)
    A = lattice.assemble(L, eps, bc)
    w = np.linalg.eigvalsh(A.toarray())
    for c in [-3.3, -0.01, 0.0137, 2.5]:
        assert inertia.count_below(A, c) == int(np.sum(w < c))


def test_shift_invert_complete_L20():
    """At L = 20 (n = 8000), the 5 Lanczos eigenvalues are exactly the
    eigenvalues in the window they span (inertia count), so none nearer
    sigma was missed."""
    L, sigma, k = 20, 0.0, 5
    eps = rng.potential(L, 16.5, 1)
    A = lattice.assemble(L, eps)
    nA = lattice.norm_bound(eps)
    ws, Vs, info = lanczos.shift_invert_nearest(A, sigma, k, tol=1e-12, norm_a=nA)
    d = np.max(np.abs(ws - sigma))
    # window [sigma - d', sigma + d') slightly beyond the k-th eigenvalue
    gap = 1e-9
    assert inertia.count_in_window(A, sigma - d - gap, sigma + d + gap) == k
    assert np.all(np.linalg.norm(A @ Vs - Vs * ws, axis=0) <= 1e-12 * nA)
