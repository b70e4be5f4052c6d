"""The levels' Schur complements formed on the GPU (ildl_params.setup_device
= 1) give the factor of the host threads bit for bit: every exported array
(permutation, scaling, level pointers, L, the pivot inverses, the dense
tail) is compared element by element.  The host factor itself is pinned
against the oracle's block elimination (one and two levels), exactness
without dropping and the matching's optimality in tests/test_setup_host.py,
so those pins carry over to the device-built factor."""
import numpy as np
import pytest

from oracle import lattice, rng

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KEYS = ["perm", "scale", "level_ptr", "Lptr", "Lcol", "Lval", "dinv_d", "dinv_o", "partner", "dense_inv"]


@pytest.fixture(scope="module")
def ajd():
    import paper_math_0508111_gb300 as ajd
    assert torch.cuda.is_available()
    return ajd


def _same(F0, F1):
    for key in KEYS:
        a, b = np.asarray(F0[key]), np.asarray(F1[key])
        assert a.shape == b.shape, key
        if a.dtype.kind == "f":
            assert np.array_equal(a.view(np.int64), b.view(np.int64)), key  # bit for bit
        else:
            assert np.array_equal(a, b), key
    for key in ["levels", "n_dense", "n_2x2", "nnz_L", "relaxed_levels"]:
        assert F0[key] == F1[key], key


@pytest.mark.parametrize("L,W,seed,bc,sigma,extra", [
    (12, 16.5, 1, 0, 0.0, {}),
    (20, 16.5, 2, 0, 0.3, {"n_dense": 500}),
    (16, 12.0, 3, 1, -0.5, {"n_dense": 300}),
    (18, 8.0, 4, 0, 1.0, {"n_dense": 400}),
    (24, 16.5, 5, 0, 0.0, {"n_dense": 300, "aggressive": 0.1}),
    (33, 16.5, 6, 0, 0.0, {}),
])
def test_device_schur_equals_host_lattice(ajd, L, W, seed, bc, sigma, extra):
    with ajd.Anderson(L, W, seed, bc) as h:
        P0 = ajd.Preconditioner.from_lattice(h, sigma, setup_device=0, **extra)
        P1 = ajd.Preconditioner.from_lattice(h, sigma, setup_device=1, **extra)
        F0, F1 = P0.export(), P1.export()
        assert F0["levels"] >= 2
        _same(F0, F1)
        P0.close()
        P1.close()


def test_device_schur_equals_host_offdiag(ajd):
    with ajd.Anderson.offdiag(14, 3, diag=1.28, width=1.0) as h:
        P0 = ajd.Preconditioner.from_lattice(h, 0.0, setup_device=0, n_dense=200)
        P1 = ajd.Preconditioner.from_lattice(h, 0.0, setup_device=1, n_dense=200)
        _same(P0.export(), P1.export())
        P0.close()
        P1.close()


def _random_symmetric(n, seed, per_row=6):
    import scipy.sparse as sparse
    g = np.random.default_rng(seed)
    r, c = g.integers(0, n, n * per_row), g.integers(0, n, n * per_row)
    v = g.choice([-1.0, 1.0], n * per_row) * 10.0 ** g.uniform(-4, 0, n * per_row)
    M = sparse.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    M = (M + M.T + sparse.diags(g.choice([-1.0, 1.0], n) * 10.0 ** g.uniform(-1, 0.5, n))).tocsr()
    M.sort_indices()
    M.eliminate_zeros()
    return M


@pytest.mark.parametrize("case", [("random", 600, 1, {"n_dense": 100}), ("random", 2000, 3, {"n_dense": 100}),
                                  ("lattice", 10, 0.4, {"max_levels": 2, "n_dense": 100}),
                                  ("lattice", 14, 0.0, {"drop": 0.0, "kappa": 1e300, "gamma": 0.0, "n_dense": 200})])
def test_device_schur_equals_host_csr(ajd, case):
    """ildl_setup_csr on the host and with the GPU Schur complements: random
    sparse matrices with entries over four decades (many drops, 2x2
    pivots), a two-level lattice factor (the oracle's two-level pin case)
    and an exact factor without dropping."""
    if case[0] == "random":
        A = _random_symmetric(case[1], case[2])
    else:
        L = case[1]
        A = lattice.assemble(L, rng.potential(L, 16.5, 3), shift=case[2]).tocsr()
        A.sort_indices()
    kw = case[3]
    F0 = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, setup_device=0, **kw).export()
    F1 = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, setup_device=1, **kw).export()
    assert F0["levels"] >= 1
    _same(F0, F1)


def test_device_setup_solves(ajd):
    """A Jacobi-Davidson solve with the (default) device-built factor reaches
    the dense oracle's pairs."""
    from pairs import check_pairs
    L, W, seed, sigma, k, tol = 12, 16.5, 9, 0.0, 4, 1e-10
    with ajd.Anderson(L, W, seed) as h:
        ev, X, st = ajd.solve(h, sigma, k, tol, precision=ajd.JD_MIXED, ildl={"setup_device": 1})
    check_pairs(L, W, seed, 0, sigma, k, ev, X, st, tol)
