"""The library's host-side preconditioner construction (Sections 5-6), run on
the CPU and checked against the oracle."""
import numpy as np
import pytest

from oracle import krylov, lattice, matching, rng
from oracle.lattice import HARDWALL, PERIODIC


@pytest.fixture(scope="module")
def ajd():
    from paper_math_0508111_gb300 import build
    build.build()
    import paper_math_0508111_gb300 as ajd
    return ajd


def _csr(L, W, seed, bc, sigma):
    eps = rng.potential(L, W, seed)
    A = lattice.assemble(L, eps, bc, shift=sigma).tocsr()
    A.sort_indices()
    return A, eps


@pytest.mark.parametrize("L,bc,sigma,match", [(6, PERIODIC, 0.0, 1), (6, HARDWALL, 0.7, 1), (7, PERIODIC, -1.0, 1),
                                              (6, PERIODIC, 0.0, 0)])
def test_exact_without_dropping(ajd, L, bc, sigma, match):
    """With no dropping, no weak couplings ignored and kappa = inf the
    multilevel LDL^T is a complete factorization: K = A - sigma I."""
    A, _ = _csr(L, 16.5, 2, bc, sigma)
    P = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, drop=0.0, kappa=1e300, gamma=0.0,
                                    n_dense=20, matching=match)
    F = P.export()
    assert F["levels"] >= 2
    g = np.random.default_rng(0)
    for _ in range(3):
        x = g.standard_normal(A.shape[0])
        assert np.linalg.norm(matching.apply_factor(F, A @ x) - x) <= 1e-9 * np.linalg.norm(x)


def test_factor_structure(ajd):
    A, _ = _csr(12, 16.5, 1, PERIODIC, 0.0)
    F = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, n_dense=100).export()
    n = A.shape[0]
    assert sorted(F["perm"]) == list(range(n))
    lp = F["level_ptr"]
    assert lp[0] == 0 and lp[-1] == n and np.all(np.diff(lp) >= 0)
    assert lp[-1] - lp[-2] == F["n_dense"]
    # each row only references earlier levels (one parallel step per level)
    lev = np.searchsorted(lp, np.arange(n), side="right") - 1
    for p in range(n):
        cols = F["Lcol"][F["Lptr"][p]:F["Lptr"][p + 1]]
        assert np.all(cols < lp[lev[p]])
    # 2x2 partners sit in the same level and point at each other
    pt = F["partner"]
    for p in range(lp[-2]):
        if pt[p] >= 0:
            assert pt[pt[p]] == p and lev[pt[p]] == lev[p]
    # dense inverse is symmetric
    Dn = F["dense_inv"]
    assert np.allclose(Dn, Dn.T)


def test_default_gamma_factor(ajd):
    """gamma < 0 selects min(0.02, 5/sqrt(n)) for a general symmetric matrix:
    the default factor equals the one built with that value given
    explicitly, array for array (L = 15: 5/sqrt(3375) = 0.086, capped at
    0.02; L = 40: 5/sqrt(64000) = 0.0198)."""
    for L in (15, 40):
        A, _ = _csr(L, 16.5, 3, PERIODIC, 0.0)
        n = A.shape[0]
        F0 = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, n_dense=300).export()
        F1 = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, n_dense=300,
                                         gamma=min(0.02, 5.0 / np.sqrt(n))).export()
        for key in ["perm", "scale", "level_ptr", "Lptr", "Lcol", "Lval", "dinv_d", "dinv_o", "partner",
                    "dense_inv"]:
            assert np.array_equal(F0[key], F1[key]), (L, key)


def test_preconditioner_quality_default(ajd):
    """Default parameters: SQMR (oracle) preconditioned by the library's K
    solves (A - sigma I) x = b at L = 12 in few iterations, versus
    thousands unpreconditioned."""
    A, _ = _csr(12, 16.5, 1, PERIODIC, 0.0)
    F = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, n_dense=200).export()
    b = np.random.default_rng(3).standard_normal(A.shape[0])
    x, k, _ = krylov.sqmr(lambda v: A @ v, lambda v: matching.apply_factor(F, v), b, 1e-8, 400)
    assert k < 80
    assert np.linalg.norm(A @ x - b) <= 1e-7 * np.linalg.norm(b)


def test_symmetry_of_K(ajd):
    A, _ = _csr(5, 16.5, 4, PERIODIC, 0.2)
    F = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, n_dense=10).export()
    g = np.random.default_rng(1)
    a, b = g.standard_normal(125), g.standard_normal(125)
    assert a @ matching.apply_factor(F, b) == pytest.approx(b @ matching.apply_factor(F, a), rel=1e-11)


@pytest.mark.parametrize("L,W,sigma", [(6, 16.5, 0.0), (8, 12.0, 0.5), (5, 2.0, 0.0)])
def test_matching_optimal_and_scaled(ajd, L, W, sigma):
    """The library's matching has the optimal product (unique even when the
    permutation is not), its scaling puts every entry in [-1, 1], and its
    1x1/2x2 groups are matched pairs."""
    A, _ = _csr(L, W, 5, PERIODIC, sigma)
    mc, sc, pt = ajd.matching(A.indptr, A.indices, A.data)
    n = A.shape[0]
    assert sorted(mc) == list(range(n))
    Ad = A.toarray()
    vals = np.abs(Ad[mc, np.arange(n)])
    assert np.all(vals > 0)
    _, _, _, total = matching.max_product_assignment(Ad)
    c = matching.costs(Ad)
    assert c[mc, np.arange(n)].sum() == pytest.approx(total, abs=1e-9)
    S = sc[:, None] * Ad * sc[None, :]
    assert np.abs(S).max() <= 1 + 1e-12
    for i in range(n):
        if pt[i] >= 0:
            j = pt[i]
            assert pt[j] == i
            assert mc[i] == j or mc[j] == i


def test_matching_fig4_structure(ajd):
    """A 6x6 symmetric matrix whose largest entries follow the matching of
    Figure 3 (rows 4,1,5,2,3,6 on the diagonal of P_M A) and whose
    diagonal inside the 3-cycle is largest at row 1: the library returns the
    cycle form and split of Figure 4."""
    n = 6
    A = np.full((n, n), 0.0)
    pm = [3, 0, 4, 1, 2, 5]  # 0-based rows matched to columns 0..5
    for col, row in enumerate(pm):
        A[row, col] = A[col, row] = 4.0
    A[0, 0], A[1, 1], A[3, 3] = 0.5, 0.1, 0.2
    A[2, 2], A[4, 4] = 0.1, 0.1
    A[5, 5] = 3.0
    import scipy.sparse as sp
    C = sp.csr_matrix(A)
    C.sort_indices()
    mc, sc, pt = ajd.matching(C.indptr, C.indices, C.data)
    cyc = sorted(sorted(c) for c in matching.cycles(mc))
    assert cyc == [[0, 1, 3], [2, 4], [5]]
    assert pt[0] == -1 and pt[1] == 3 and pt[3] == 1 and pt[2] == 4 and pt[5] == -1


def test_setup_rejects_bad_input(ajd):
    with pytest.raises(ajd.JDError):
        ajd.Preconditioner.from_csr(np.array([0, 1]), np.array([0]), np.array([1.0]), kappa=0.5)
    with pytest.raises(ajd.JDError):
        ajd.Preconditioner.from_csr(np.array([0, 2, 3]), np.array([1, 0, 1]), np.array([1.0, 2.0, 1.0]))


@pytest.mark.parametrize("aggressive", [0.0, 0.1])
def test_setup_independent_of_thread_count(ajd, aggressive):
    """The parallel setup (matching searches in batches, parallel scatters,
    per-chunk rows) gives the same factor, bit for bit, with 1 and 4 host
    threads.  L = 24 is large enough that the scatters and the Schur mirror
    split their work into several thread groups (at least 16384 entries
    per group)."""
    import ctypes
    import ctypes.util
    gomp = ctypes.CDLL(ctypes.util.find_library("gomp") or "libgomp.so.1")
    A, _ = _csr(24, 12.0, 6, PERIODIC, 0.2)
    out = []
    try:
        for t in (1, 4):
            gomp.omp_set_num_threads(t)
            out.append(ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, n_dense=300,
                                                   aggressive=aggressive).export())
    finally:
        gomp.omp_set_num_threads(max(1, __import__("os").cpu_count() or 1))
    assert out[0]["levels"] >= 3
    for key in out[0]:
        if key.endswith("_ms"):  # timings
            continue
        a, b = np.asarray(out[0][key]), np.asarray(out[1][key])
        assert a.shape == b.shape and np.array_equal(a, b), key


def test_aggressive_dropping_rule(ajd):
    """Section 6.3's aggressive dropping on a one-level factor (the rest of
    the matrix goes to the dense block), where the exported L is exactly the
    level's scaled column block: an entry l_ij of the default factor is
    removed iff |l_ij| <= tau / #(entries of column j); the pivots,
    ordering, scaling and D are unchanged and the kept entries are the same
    numbers.  tau = 0 gives the default factor bit for bit.  (The first
    level's entries are large, so a large tau is taken to make it drop.)"""
    A, _ = _csr(10, 16.5, 5, PERIODIC, 0.0)
    kw = dict(max_levels=1, n_dense=100)
    F0 = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, **kw).export()
    Fz = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, aggressive=0.0, **kw).export()
    tau = 0.9
    Fa = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, aggressive=tau, **kw).export()
    for key in F0:
        if not key.endswith("_ms"):
            assert np.array_equal(np.asarray(F0[key]), np.asarray(Fz[key])), key
    assert F0["levels"] == Fa["levels"] == 1 and F0["aggressive_dropped"] == 0
    for key in ("perm", "scale", "level_ptr", "dinv_d", "dinv_o", "partner"):
        assert np.array_equal(F0[key], Fa[key]), key
    n = A.shape[0]
    L0 = [(r, c, v) for r in range(n) for c, v in zip(F0["Lcol"][F0["Lptr"][r]:F0["Lptr"][r + 1]],
                                                        F0["Lval"][F0["Lptr"][r]:F0["Lptr"][r + 1]])]
    count = np.bincount([c for _, c, _ in L0], minlength=n)
    want = {(r, c): v for r, c, v in L0 if abs(v) > tau / count[c]}
    got = {(r, c): v for r in range(n) for c, v in zip(Fa["Lcol"][Fa["Lptr"][r]:Fa["Lptr"][r + 1]],
                                                         Fa["Lval"][Fa["Lptr"][r]:Fa["Lptr"][r + 1]])}
    assert got == want
    assert Fa["aggressive_dropped"] == len(L0) - len(want) > 0


def test_aggressive_dropping_quality(ajd):
    """A multilevel factor with aggressive dropping (tau = 0.1, the value the
    paper suggests) is sparser and still a good preconditioner: oracle SQMR
    on (A - sigma I) x = b needs at most twice the default factor's
    iterations."""
    A, _ = _csr(14, 16.5, 1, PERIODIC, 0.0)
    b = np.random.default_rng(4).standard_normal(A.shape[0])
    its = {}
    nnz = {}
    for tau in (0.0, 0.1):
        F = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, n_dense=300, aggressive=tau).export()
        assert F["levels"] >= 3
        x, its[tau], _ = krylov.sqmr(lambda v: A @ v, lambda v: matching.apply_factor(F, v), b, 1e-8, 400)
        assert np.linalg.norm(A @ x - b) <= 1e-7 * np.linalg.norm(b)
        nnz[tau] = F["nnz_L"]
    assert nnz[0.1] < nnz[0.0]
    assert its[0.1] <= 2 * its[0.0]


def test_aggressive_dropping_rejects_bad_tau(ajd):
    A, _ = _csr(6, 16.5, 1, PERIODIC, 0.0)
    for tau in (-0.1, 1.0, float("nan")):
        with pytest.raises(ajd.JDError):
            ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, aggressive=tau)


def _random_symmetric(n, seed, per_row=6):
    """Sparse symmetric test matrix with entries over four decades (so that
    the drop rule and 2x2 pivots come into play)."""
    import scipy.sparse as sparse
    g = np.random.default_rng(seed)
    r, c = g.integers(0, n, n * per_row), g.integers(0, n, n * per_row)
    v = g.choice([-1.0, 1.0], n * per_row) * 10.0 ** g.uniform(-4, 0, n * per_row)
    M = sparse.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    M = (M + M.T + sparse.diags(g.choice([-1.0, 1.0], n) * 10.0 ** g.uniform(-1, 0.5, n))).tocsr()
    M.sort_indices()
    M.eliminate_zeros()
    return M


@pytest.mark.parametrize("case", [("lattice", 8, 16.5, 3, 0.0), ("lattice", 9, 12.0, 4, 0.4),
                                  ("lattice", 8, 21.0, 6, -0.7), ("lattice", 8, 1.0, 3, 0.0),
                                  ("random", 500, 1), ("random", 400, 3)])
def test_one_level_factor_matches_oracle(ajd, case):
    """A factor with one sparse level (the rest goes to the dense block),
    element by element against the oracle's block elimination (Sections
    6.2-6.3) on the same scaled matrix and pivots: D_B^{-1}, the column
    block L_F of L with its drops, and the dense block's inverse against the
    oracle's Schur complement.  The library's pivot choice is checked against
    its rules: every 1x1 pivot meets 1 + d1 <= kappa, every 2x2 pivot
    d2 < d1 and 1 + (largest column sum of its L block) <= kappa, and pivots
    of the level are coupled by at most gamma.  Lattices (one with many 2x2
    pivots and a relaxed level) and random sparse matrices whose entries span
    four decades (many drops in L_F)."""
    from oracle import ildl
    if case[0] == "lattice":
        A, _ = _csr(*case[1:3], case[3], PERIODIC, case[4])
    else:
        A = _random_symmetric(case[1], case[2])
    n = A.shape[0]
    F = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, max_levels=1, n_dense=100).export()
    assert F["levels"] == 1
    perm, lp, pt = F["perm"], F["level_ptr"], F["partner"]
    nb = int(lp[1])
    s = np.empty(n)
    s[perm] = F["scale"]
    As = s[:, None] * A.toarray() * s[None, :]
    blocks, p = [], 0
    while p < nb:  # the pivot blocks in elimination order
        if pt[p] >= 0:
            assert pt[p] == p + 1 and pt[p + 1] == p
            blocks.append([int(perm[p]), int(perm[p + 1])])
            p += 2
        else:
            blocks.append([int(perm[p])])
            p += 1
    tau = 1.0 / (5.0 * np.sqrt(n))  # epsilon / kappa, epsilon = 1/sqrt(n)
    B, C, D, LF, S = ildl.eliminate_level(As, blocks, tau)
    assert list(perm[:nb]) == B and list(perm[nb:]) == C
    # no entry within rounding of the drop threshold (so both sides must
    # take the same drop decisions)
    _, _, _, LF0, _ = ildl.eliminate_level(As, blocks, 0.0)
    assert not np.any(np.abs(np.abs(LF0) - tau) <= 1e-9 * tau)
    # D^{-1} per position
    Dinv = np.linalg.inv(D)
    for q in range(nb):
        assert abs(F["dinv_d"][q] - Dinv[q, q]) <= 1e-12 * abs(Dinv[q, q])
        if pt[q] >= 0:
            assert abs(F["dinv_o"][q] - Dinv[q, pt[q]]) <= 1e-12 * np.abs(Dinv).max()
    # L: only the block (C rows, B columns), same pattern and values
    import scipy.sparse as sparse
    Lx = sparse.csr_matrix((F["Lval"], F["Lcol"], F["Lptr"]), shape=(n, n)).toarray()
    assert not Lx[:nb].any() and not Lx[nb:, nb:].any()
    got = Lx[nb:, :nb]
    assert np.array_equal(got != 0, LF != 0)
    assert np.abs(got - LF).max() <= 1e-12 * np.abs(LF).max()
    # dense block: the inverse of the oracle's Schur complement
    Sd = S[np.ix_(range(len(C)), range(len(C)))]
    off = ~np.eye(len(C), dtype=bool)
    S0 = As[np.ix_(C, C)] - LF @ D @ LF.T
    assert not np.any(off & (np.abs(np.abs(S0) - tau) <= 1e-9 * tau))
    assert np.abs(F["dense_inv"] @ Sd - np.eye(len(C))).max() <= 1e-8
    # the pivot rules
    # a relaxed level widens the bound step by step, at most to 64 kappa
    kappa, gamma = (5.0 if F["relaxed_levels"] == 0 else 320.0), min(0.02, 5.0 / np.sqrt(n))
    absA = np.abs(As)
    d1 = (absA.sum(axis=0) - np.diag(absA)) / np.abs(np.diag(As))
    owner = {i: k for k, b in enumerate(blocks) for i in b}
    _, _, pt0 = ajd.matching(A.indptr, A.indices, A.data)  # the level's matched pairs
    for b in blocks:
        if len(b) == 1:
            assert 1.0 + d1[b[0]] <= kappa * (1 + 1e-12)
            x, y = b[0], pt0[b[0]]
            if y >= 0:  # a matched pair taken apart: its 2x2 form was not better (d2 >= d1)
                Bxy = As[np.ix_([x, y], [x, y])]
                if abs(np.linalg.det(Bxy)) > 1e-300:
                    R = As[:, [x, y]] @ np.linalg.inv(Bxy)
                    R[[x, y]] = 0.0
                    assert np.abs(R).sum() >= min(d1[x], d1[y]) * (1 - 1e-12)
        else:
            i, j = b
            R = As[:, b] @ np.linalg.inv(As[np.ix_(b, b)])
            R[b] = 0.0
            cs = np.abs(R).sum(axis=0)
            assert cs.sum() < min(d1[i], d1[j])
            assert 1.0 + cs.max() <= kappa * (1 + 1e-12)
    for x in B:
        for y in B:
            if owner[x] != owner[y]:
                assert absA[x, y] <= gamma


def _pivot_blocks(F, lo, hi):
    """Pivot blocks (lists of positions) of the positions [lo, hi)."""
    pt, blocks, p = F["partner"], [], lo
    while p < hi:
        if pt[p] >= 0:
            assert pt[p] == p + 1 and pt[p + 1] == p
            blocks.append([p, p + 1])
            p += 2
        else:
            blocks.append([p])
            p += 1
    return blocks


@pytest.mark.parametrize("case", [("lattice", 8, 16.5, 3, 0.0), ("lattice", 9, 12.0, 5, 0.3), ("random", 500, 2)])
def test_two_level_factor_matches_oracle(ajd, case):
    """The composition of levels, element by element: a factor with two
    sparse levels against the oracle's block elimination applied twice.
    Level 1 works on the oracle's Schur complement of level 0, scaled by the
    library's matching of that matrix (``ildl_matching``); the stored scaling
    of a level-1 node is the product of its two scalings, a level-0 column of
    L seen from a later row carries that row's second scaling, and the dense
    block inverts the oracle's second Schur complement."""
    import scipy.sparse as sparse
    from oracle import ildl
    if case[0] == "lattice":
        A, _ = _csr(*case[1:3], case[3], PERIODIC, case[4])
    else:
        A = _random_symmetric(case[1], case[2])
    n = A.shape[0]
    tau = 1.0 / (5.0 * np.sqrt(n))
    F = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, max_levels=2, n_dense=100).export()
    assert F["levels"] == 2
    perm, lp, sc = F["perm"], F["level_ptr"], F["scale"]
    n0, n1 = int(lp[1]), int(lp[2])
    # level 0 on the library's scaling of A
    _, s1, _ = ajd.matching(A.indptr, A.indices, A.data)
    assert np.array_equal(sc[:n0], s1[perm[:n0]])
    As1 = s1[:, None] * A.toarray() * s1[None, :]
    blocks0 = [[int(perm[q]) for q in b] for b in _pivot_blocks(F, 0, n0)]
    B0, C0, D0, LF0, S1 = ildl.eliminate_level(As1, blocks0, tau)
    assert list(perm[:n0]) == B0
    # level 1 on the oracle's Schur complement, scaled by the library's matching of it
    S1c = sparse.csr_matrix(S1)
    S1c.sort_indices()
    assert all(S1c[i, i] != 0 for i in range(S1.shape[0]))
    _, s2, _ = ajd.matching(S1c.indptr, S1c.indices, S1c.data)
    loc = {g: k for k, g in enumerate(C0)}
    later = np.array([loc[int(g)] for g in perm[n0:]])  # local index in level 1 of positions n0..n-1
    assert np.allclose(sc[n0:], s1[perm[n0:]] * s2[later], rtol=1e-12, atol=0)
    As2 = s2[:, None] * S1 * s2[None, :]
    blocks1 = [[int(later[q - n0]) for q in b] for b in _pivot_blocks(F, n0, n1)]
    B1, C1, D1, LF1, S2 = ildl.eliminate_level(As2, blocks1, tau)
    assert list(later[:n1 - n0]) == B1 and list(later[n1 - n0:]) == C1
    for As_, blocks_ in ((As1, blocks0), (As2, blocks1)):  # no entry within rounding of the drop threshold
        _, _, _, LFx, _ = ildl.eliminate_level(As_, blocks_, 0.0)
        assert not np.any(np.abs(np.abs(LFx) - tau) <= 1e-9 * tau)
    # D^{-1} of both levels
    Dinv = np.zeros(n)
    Dinv[:n0] = np.diag(np.linalg.inv(D0))
    Dinv[n0:n1] = np.diag(np.linalg.inv(D1))
    assert np.allclose(F["dinv_d"][:n1], Dinv[:n1], rtol=1e-11, atol=0)
    # L: level-0 columns (rows n0.., times the row's level-1 scaling), level-1 columns (dense rows)
    Lx = sparse.csr_matrix((F["Lval"], F["Lcol"], F["Lptr"]), shape=(n, n)).toarray()
    want = np.zeros((n, n))
    want[n0:, :n0] = LF0[later] * s2[later][:, None]
    want[n1:, n0:n1] = LF1
    assert np.array_equal(Lx != 0, want != 0)
    assert np.abs(Lx - want).max() <= 1e-11 * np.abs(want).max()
    # dense block: inverse of the second Schur complement
    assert np.abs(F["dense_inv"] @ S2 - np.eye(S2.shape[0])).max() <= 1e-8


def _off_diagonal_dominant(n, seed):
    """Sparse symmetric matrix with tiny diagonal: the matching goes off the
    diagonal, mostly in 2-cycles, with a few long cycles."""
    import scipy.sparse as sparse
    g = np.random.default_rng(seed)
    r, c = g.integers(0, n, n * 4), g.integers(0, n, n * 4)
    v = g.choice([-1.0, 1.0], n * 4) * 10.0 ** g.uniform(-2, 0, n * 4)
    M = sparse.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    M = (M + M.T + sparse.diags(g.choice([-1.0, 1.0], n) * 10.0 ** g.uniform(-4, -2, n))).tocsr()
    M.sort_indices()
    M.eliminate_zeros()
    return M


@pytest.mark.parametrize("seed", [1, 2, 5, 14])
def test_cycle_split_rules(ajd, seed):
    """The 1x1/2x2 groups of the library's matching follow the cycle-split
    readings of Section 5.2 on matrices with long cycles: an odd cycle keeps
    its member of largest |diagonal| (scaled matrix) as the 1x1 and pairs
    the rest in cycle order; an even cycle takes the split with the larger
    sum of log|off-diagonal| (ties: fewer nonzeros in the merged rows).  The
    seeds give odd cycles of length 3 to 93; even cycles longer than 2 only
    arise from ties (for a symmetric matrix the product along an even cycle
    is the geometric mean of its two splits, so one split is at least as
    good), and the rule for them is checked wherever one appears."""
    A = _off_diagonal_dominant(3000, seed)
    mc, sc, pt = ajd.matching(A.indptr, A.indices, A.data)
    S = (sc[:, None] * A.toarray()) * sc[None, :]
    pattern = [set(A.indices[A.indptr[i]:A.indptr[i + 1]]) for i in range(A.shape[0])]
    long_cycles = 0
    for cyc in matching.cycles(mc):
        m = len(cyc)
        if m == 1:
            want = matching.split_cycle(cyc, 0)
        elif m % 2 == 0:
            def score(s):
                return sum(np.log(abs(S[a, b]) + 1e-300) for a, b in matching.split_cycle(cyc, s))

            def nnz(s):
                return sum(len(pattern[a] | pattern[b]) for a, b in matching.split_cycle(cyc, s))
            s = 1 if (score(1) > score(0) or (score(1) == score(0) and nnz(1) < nnz(0))) else 0
            want = matching.split_cycle(cyc, s)
        else:
            d = np.abs(S[cyc, cyc])
            t = max(range(m), key=lambda k: (d[k], -cyc[k]))
            want = matching.split_cycle(cyc, t)
        long_cycles += m > 2
        for grp in want:
            if len(grp) == 1:
                assert pt[grp[0]] == -1
            else:
                assert pt[grp[0]] == grp[1] and pt[grp[1]] == grp[0]
    assert long_cycles >= 1


def test_dense_only_factor(ajd):
    """Degenerate case: a matrix no larger than the dense block gets no sparse
    level, an empty L, and K = A - sigma I exactly (the dense inverse)."""
    A, _ = _csr(5, 16.5, 2, PERIODIC, 0.3)
    F = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, n_dense=200).export()
    assert F["levels"] == 0 and F["nnz_L"] == 0 and F["n_dense"] == A.shape[0]
    b = np.random.default_rng(0).standard_normal(A.shape[0])
    assert np.abs(matching.apply_factor(F, A @ b) - b).max() <= 1e-12 * np.abs(b).max()


def test_concurrent_setups_match_sequential(ajd):
    """The host setup holds no shared state: two setups running at once on
    two host threads (as in the batch and the server) give the same factors,
    bit for bit, as one after the other."""
    import threading
    mats = [_csr(16, 16.5, s, PERIODIC, 0.1)[0] for s in (7, 8)]

    def build(A):
        return ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, n_dense=200).export()

    seq = [build(A) for A in mats]
    out = [None, None]

    def run(i):
        out[i] = build(mats[i])

    ts = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for a, b in zip(seq, out):
        for key in a:
            if not key.endswith("_ms"):
                assert np.array_equal(np.asarray(a[key]), np.asarray(b[key])), key
