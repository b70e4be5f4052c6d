"""Pins of the oracle's one-level block elimination (Sections 6.2-6.3):
the block LDL^T identity without dropping and hand-worked examples with a
1x1 pivot, a 2x2 pivot and the drop rule."""
import numpy as np

from oracle import ildl


def test_block_ldlt_identity_without_dropping():
    """With tau = 0 and no coupling between different pivots,
    [[I, 0], [L_F, I]] diag(D_B, S') [[I, L_F^T], [0, I]] = As in (B, C) order."""
    g = np.random.default_rng(5)
    n = 12
    As = g.standard_normal((n, n))
    As = As + As.T + 8.0 * np.eye(n)
    blocks = [[0], [3, 4], [7], [9, 10]]
    piv = [i for b in blocks for i in b]
    owner = {i: k for k, b in enumerate(blocks) for i in b}
    for x in piv:  # pivots of one level are not coupled to each other
        for y in piv:
            if owner[x] != owner[y]:
                As[x, y] = 0.0
    B, C, D, LF, S = ildl.eliminate_level(As, blocks, 0.0)
    assert B == piv and C == [i for i in range(n) if i not in piv]
    nb, nc = len(B), len(C)
    Lfull = np.eye(n)
    Lfull[nb:, :nb] = LF
    M = np.zeros((n, n))
    M[:nb, :nb] = D
    M[nb:, nb:] = S
    order = B + C
    assert np.allclose(Lfull @ M @ Lfull.T, As[np.ix_(order, order)], atol=1e-12, rtol=0)


def test_one_by_one_pivot_and_drop_order():
    """Hand-worked: pivot 0 of [[2, 1, .5], [1, 3, .25], [.5, .25, 4]].
    Without dropping L_F = (1/2, 1/4) and S' = [[2.5, 0], [0, 3.875]] (the
    coupling cancels exactly).  With tau = 0.3 the entry 1/4 of L_F is dropped
    first, so S' = [[2.5, .25], [.25, 4]] before its own drop, and the 0.25
    coupling is then dropped too."""
    As = np.array([[2.0, 1.0, 0.5], [1.0, 3.0, 0.25], [0.5, 0.25, 4.0]])
    _, C, D, LF, S = ildl.eliminate_level(As, [[0]], 0.0)
    assert C == [1, 2]
    assert np.allclose(D, [[2.0]]) and np.allclose(LF, [[0.5], [0.25]])
    assert np.allclose(S, [[2.5, 0.0], [0.0, 3.875]], atol=1e-15)
    _, _, _, LF, S = ildl.eliminate_level(As, [[0]], 0.3)
    assert np.array_equal(LF, [[0.5], [0.0]])
    assert np.allclose(S, [[2.5, 0.0], [0.0, 4.0]], atol=1e-15)


def test_two_by_two_pivot():
    """Hand-worked 2x2 pivot [[1, 2], [2, 1]] (inverse [[-1, 2], [2, -1]]/3)
    with rows (1, 0) and (0, 3) below it: L_F = [[-1/3, 2/3], [2, -1]] and
    S' = [[5, 0], [0, 6]] - [[-1/3, 2], [2, -3]] = [[16/3, -2], [-2, 9]]."""
    As = np.array([[1.0, 2.0, 1.0, 0.0],
                   [2.0, 1.0, 0.0, 3.0],
                   [1.0, 0.0, 5.0, 0.0],
                   [0.0, 3.0, 0.0, 6.0]])
    B, C, D, LF, S = ildl.eliminate_level(As, [[0, 1]], 0.0)
    assert B == [0, 1] and C == [2, 3]
    assert np.allclose(LF, [[-1.0 / 3.0, 2.0 / 3.0], [2.0, -1.0]], atol=1e-15)
    assert np.allclose(S, [[16.0 / 3.0, -2.0], [-2.0, 9.0]], atol=1e-14)
