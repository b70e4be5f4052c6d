"""Pins for the oracle's assembly of the Anderson matrix (Eq. (1))."""
import numpy as np
import pytest

from oracle import lattice, rng
from oracle.lattice import HARDWALL, PERIODIC


@pytest.mark.parametrize("L", [3, 4, 5, 6])
@pytest.mark.parametrize("bc", [PERIODIC, HARDWALL])
@pytest.mark.parametrize("t", [-1.0, 1.0])
def test_zero_disorder_closed_form(L, bc, t):
    """W = 0: the spectrum is the Kronecker sum of three 1D chains."""
    A = lattice.dense(L, np.zeros(L ** 3), bc, t)
    w = np.linalg.eigvalsh(A)
    assert np.allclose(w, lattice.closed_form_spectrum(L, bc, t), atol=1e-12)


def test_hopping_sign_matters_on_odd_periodic_lattice():
    """On L = 5 periodic (not bipartite) the two hopping signs differ, so the
    closed-form pin above distinguishes them."""
    a = lattice.closed_form_spectrum(5, PERIODIC, -1.0)
    b = lattice.closed_form_spectrum(5, PERIODIC, +1.0)
    assert not np.allclose(a, b)
    assert a[0] == pytest.approx(-6.0)


@pytest.mark.parametrize("bc", [PERIODIC, HARDWALL])
def test_plane_waves_are_eigenvectors(bc):
    L = 7
    A = lattice.assemble(L, np.zeros(L ** 3), bc)
    for m in [(1, 0, 0), (2, 3, 1), (3, 3, 3)] if bc == PERIODIC else [(1, 1, 1), (2, 5, 3)]:
        v = lattice.plane_wave(L, m, bc)
        lam = lattice.plane_wave_eigenvalue(L, m, bc)
        assert np.linalg.norm(A @ v - lam * v) < 1e-12


@pytest.mark.parametrize("bc", [PERIODIC, HARDWALL])
def test_trace_frobenius_symmetry(bc):
    L, W = 6, 16.5
    eps = rng.potential(L, W, 11)
    A = lattice.assemble(L, eps, bc)
    assert abs(A - A.T).max() == 0.0
    assert A.diagonal().sum() == pytest.approx(eps.sum(), abs=1e-12)
    nbond_entries = 6 * L ** 3 if bc == PERIODIC else 6 * L * L * (L - 1)
    assert (A.multiply(A)).sum() == pytest.approx((eps ** 2).sum() + nbond_entries, rel=1e-14)
    # every off-diagonal entry is the hopping -1
    off = A.toarray() - np.diag(eps)
    offd = off[~np.eye(L ** 3, dtype=bool)]
    assert set(np.unique(offd)) <= {0.0, -1.0}


def test_neighbour_structure():
    L = 5
    A = lattice.assemble(L, np.zeros(L ** 3), PERIODIC)
    assert np.all(np.diff(A.indptr) == 7)  # 6 neighbours + diagonal
    H = lattice.assemble(L, np.zeros(L ** 3), HARDWALL)
    deg = np.diff(H.indptr) - 1
    # corners 3, edges 4, faces 5, interior 6
    counts = {d: int(np.sum(deg == d)) for d in range(3, 7)}
    assert counts == {3: 8, 4: 12 * (L - 2), 5: 6 * (L - 2) ** 2, 6: (L - 2) ** 3}
    # site (x, y, z) = (1, 0, 0) has index 1; (0, 1, 0) has index L
    row = A[0].toarray().ravel()
    assert row[1] == -1 and row[L] == -1 and row[L * L] == -1
    assert row[L - 1] == -1 and row[L * (L - 1)] == -1 and row[L * L * (L - 1)] == -1


def test_gershgorin_interval():
    for seed in range(3):
        L, W = 6, 16.5
        eps = rng.potential(L, W, seed)
        w = np.linalg.eigvalsh(lattice.dense(L, eps))
        assert np.all(np.abs(w) <= 6 + W / 2)
        assert np.all(np.abs(w) <= lattice.norm_bound(eps) + 1e-12)


def test_sign_identity():
    """H_{-1}(eps) = -H_{+1}(-eps) entry by entry."""
    L = 5
    eps = rng.potential(L, 12.0, 4)
    a = lattice.assemble(L, eps, PERIODIC, -1.0)
    b = lattice.assemble(L, -eps, PERIODIC, +1.0)
    assert abs(a + b).max() == 0.0


def test_rejects_tiny_periodic():
    with pytest.raises(ValueError):
        lattice.assemble(2, np.zeros(8), PERIODIC)
    lattice.assemble(1, np.zeros(1), HARDWALL)


def test_matvec_block_and_shift():
    L = 4
    eps = rng.potential(L, 16.5, 9)
    X = np.random.default_rng(0).standard_normal((L ** 3, 3))
    Y = lattice.matvec(L, eps, X, shift=0.7)
    D = lattice.dense(L, eps) - 0.7 * np.eye(L ** 3)
    assert np.allclose(Y, D @ X, atol=1e-13)


# ---- off-diagonal Anderson model (Section 7, Table 6) ----

@pytest.mark.parametrize("L,bc", [(3, 0), (4, 1), (5, 0), (6, 1)])
def test_offdiag_constant_hopping_is_eq1(L, bc):
    """Equal hopping on every bond and the potential on the diagonal give
    exactly the matrix of Eq. (1) (assemble, pinned by the closed form)."""
    eps = rng.potential(L, 16.5, 4)
    for t in (-1.0, 0.7):
        A = lattice.assemble(L, eps, bc, t=t, shift=0.3)
        B = lattice.assemble_offdiag(L, eps, np.full((L ** 3, 3), t), bc, shift=0.3)
        assert abs(A - B).max() == 0.0


def test_offdiag_hard_wall_ignores_outer_bonds():
    L = 5
    hop = rng.hoppings(L, 3)
    A = lattice.assemble_offdiag(L, 1.28, hop, lattice.HARDWALL)
    _, x, y, z = np.arange(L ** 3), *(np.arange(L ** 3) % L, (np.arange(L ** 3) // L) % L, np.arange(L ** 3) // L ** 2)
    hop2 = hop.copy()
    hop2[x == L - 1, 0] = 99.0
    hop2[y == L - 1, 1] = 99.0
    hop2[z == L - 1, 2] = 99.0
    assert abs(A - lattice.assemble_offdiag(L, 1.28, hop2, lattice.HARDWALL)).max() == 0.0
    # ... while a periodic lattice uses them
    assert abs(lattice.assemble_offdiag(L, 1.28, hop, 0) - lattice.assemble_offdiag(L, 1.28, hop2, 0)).max() > 1.0


@pytest.mark.parametrize("L,bc", [(4, 0), (5, 1)])
def test_offdiag_invariants(L, bc):
    """Symmetry, trace, Frobenius norm (every kept bond twice) and the
    Gershgorin bound of the spectrum."""
    n = L ** 3
    hop = rng.hoppings(L, 9)
    A = lattice.assemble_offdiag(L, 1.28, hop, bc)
    Ad = A.toarray()
    assert np.array_equal(Ad, Ad.T)
    assert np.trace(Ad) == pytest.approx(1.28 * n)
    nbonds = 3 * n if bc == 0 else 3 * L * L * (L - 1)
    assert A.nnz == n + 2 * nbonds
    off = Ad - np.diag(np.diag(Ad))
    assert np.sum(off ** 2) == pytest.approx(2 * (np.sum(hop ** 2) if bc == 0 else np.sum(off[np.triu_indices(n, 1)] ** 2)))
    w = np.linalg.eigvalsh(Ad)
    r = lattice.norm_bound_offdiag(1.28, hop)
    assert w.min() >= 1.28 - 6 * np.abs(hop).max() - 1e-12 and w.max() <= r + 1e-12


def test_hoppings_range_and_stream():
    L = 6
    h = rng.hoppings(L, 11, width=1.0)
    assert h.shape == (L ** 3, 3)
    assert h.min() >= -0.5 and h.max() < 0.5
    # the same stream as the potential, read at 3s + d
    assert np.array_equal(h.ravel(), rng.uniform01(11, 3 * L ** 3) - 0.5)
