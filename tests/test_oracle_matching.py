"""Pins for the oracle's matching, cycle split, scaling and factor apply."""
import itertools
import os

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from oracle import lattice, matching, rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_sparse(n, density, seed):
    g = np.random.default_rng(seed)
    A = g.standard_normal((n, n)) * (g.random((n, n)) < density)
    A = A + A.T
    A[np.arange(n), np.arange(n)] += g.standard_normal(n) * (g.random(n) < 0.7)
    return A


@pytest.mark.parametrize("seed", range(6))
def test_assignment_matches_brute_force(seed):
    n = 6
    A = _random_sparse(n, 0.6, seed)
    A += np.eye(n) * 1e-3  # keep a perfect matching
    col_of_row, u, v, total = matching.max_product_assignment(A)
    best = -np.inf
    for perm in itertools.permutations(range(n)):
        vals = np.abs(A[np.arange(n), perm])
        if np.all(vals > 0):
            best = max(best, np.sum(np.log(vals)))
    got = np.sum(np.log(np.abs(A[np.arange(n), col_of_row])))
    assert got == pytest.approx(best, abs=1e-12)


def test_assignment_matches_library_and_duals_certify():
    n = 60
    A = _random_sparse(n, 0.15, 7) + np.eye(n) * 0.5
    c = matching.costs(A)
    col_of_row, u, v, total = matching.max_product_assignment(A)
    big = np.where(np.isfinite(c), c, 1e6)
    r, cc = linear_sum_assignment(big)
    assert total == pytest.approx(big[r, cc].sum(), abs=1e-9)
    finite = np.isfinite(c)
    slack = c - u[:, None] - v[None, :]
    assert np.all(slack[finite] >= -1e-10)
    assert np.allclose(slack[np.arange(n), col_of_row], 0.0, atol=1e-10)


def _golden_fig4():
    d = {}
    for line in open(os.path.join(GOLDEN, "fig4_cycles.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, rest = line.split(None, 1)
        d[key] = rest
    return d


def test_fig4_cycle_form_and_split():
    """Section 5.2, Figures 3-4: P_M = (e4;e1;e5;e2;e3;e6) has cycles
    (1 2 4)(3 5)(6); keeping 1 as the 1x1 gives (1)(2 4)(3 5)(6)."""
    g = _golden_fig4()
    pm = [int(x) - 1 for x in g["pm"].split()]
    # row i of P_M is e_{pm[i]}: the diagonal of P_M A holds a_{pm[i], i},
    # so column i is matched to row pm[i]
    match_col = np.array(pm)
    cyc = matching.cycles(match_col)
    want = [sorted(int(x) - 1 for x in part.split()) for part in g["cycles"].split("|")]
    assert sorted(sorted(c) for c in cyc) == sorted(want)
    c3 = [c for c in cyc if len(c) == 3][0]
    split = matching.split_cycle(c3, c3.index(0))
    want_split = [tuple(sorted(int(x) - 1 for x in part.split())) for part in g["split"].split("|")]
    for grp in split:
        assert grp in want_split
    # every 2x2 group holds an entry of the matching
    for grp in split:
        if len(grp) == 2:
            a, b = grp
            assert match_col[a] == b or match_col[b] == a


@pytest.mark.parametrize("L,W,sigma", [(4, 16.5, 0.0), (5, 12.0, 0.3), (4, 2.0, 0.0)])
def test_scaling_invariants_on_anderson(L, W, sigma):
    """Section 4.2: after scaling all entries are <= 1 in modulus and the
    matched entries are exactly 1 in modulus."""
    eps = rng.potential(L, W, 3)
    A = lattice.dense(L, eps, shift=sigma)
    col_of_row, u, v, _ = matching.max_product_assignment(A)
    d = matching.symmetric_scaling(A, u, v)
    S = d[:, None] * A * d[None, :]
    assert np.abs(S).max() <= 1.0 + 1e-12
    # matched entries: the row-column scaling D_r A D_c is exactly 1 there;
    # the symmetric scaling keeps 1x1 matches (diagonal) at exactly 1
    a = np.abs(A).max(axis=1)
    Dr = np.exp(u) / a
    Dc = np.exp(v)
    R = Dr[:, None] * np.abs(A) * Dc[None, :]
    assert np.allclose(R[np.arange(A.shape[0]), col_of_row], 1.0, atol=1e-12)
    diag_matched = col_of_row == np.arange(A.shape[0])
    assert np.allclose(np.abs(np.diag(S))[diag_matched], 1.0, atol=1e-12)


def test_apply_factor_definition():
    """apply_factor inverts K = P^T S^{-1} L D L^T S^{-1} P built by hand."""
    g = np.random.default_rng(5)
    n = 9
    perm = g.permutation(n)
    s = g.uniform(0.5, 2.0, n)
    Lm = np.tril(g.standard_normal((n, n)) * (g.random((n, n)) < 0.4), -1)
    # levels: positions 0-3 level 0, 4-6 level 1, 7-8 dense; L only from earlier levels
    Lm[1:4, :4] = 0.0
    Lm[5:7, 4:7] = 0.0
    Lm[8, 7] = 0.0
    D = np.zeros((n, n))
    D[0, 0], D[3, 3] = 2.0, -1.5
    D[1:3, 1:3] = [[0.3, 1.0], [1.0, -0.2]]
    D[4, 4], D[5:7, 5:7] = 0.7, [[1.1, 0.4], [0.4, -0.9]]
    D[7:9, 7:9] = [[1.0, 0.5], [0.5, 2.0]]
    Dinv = np.linalg.inv(D)
    Ls = Lm.copy()
    import scipy.sparse as sp
    Lc = sp.csr_matrix(Ls)
    F = dict(perm=perm, scale=s, level_ptr=np.array([0, 4, 7, 9]), Lptr=Lc.indptr, Lcol=Lc.indices,
             Lval=Lc.data, dinv_d=np.diag(Dinv).copy(), dinv_o=np.zeros(n),
             partner=-np.ones(n, dtype=int), dense_inv=Dinv[7:, 7:])
    for p, q in [(1, 2), (5, 6)]:
        F["partner"][p], F["partner"][q] = q, p
        F["dinv_o"][p] = F["dinv_o"][q] = Dinv[p, q]
    P = np.zeros((n, n))
    P[np.arange(n), perm] = 1.0
    Lfull = np.eye(n) + Lm
    K = P.T @ np.diag(1 / s) @ Lfull @ D @ Lfull.T @ np.diag(1 / s) @ P
    b = g.standard_normal(n)
    assert np.allclose(matching.apply_factor(F, K @ b), b, atol=1e-12)
