"""One level of the incomplete block LDL^T (oracle side, test infrastructure).

Sections 6.2-6.3: a level eliminates a set of pivots B (1x1 or 2x2 blocks of
the scaled symmetric matrix As) and passes the Schur complement of the rest
C on to the next level.  Written from that definition, densely, for small
matrices:

  D_B   block diagonal matrix of the pivot blocks, As[b, b] for each block b.
        Couplings between different pivots of the same level are not part of
        D_B: the level treats them as dropped (the pivots are chosen so that
        these couplings are weak).
  L_F = As[C, B] D_B^{-1}, entries with |l| < tau set to zero (the drop
        rule of Section 6.2, tau = epsilon / kappa).
  S'  = As[C, C] - L_F D_B L_F^T, off-diagonal entries with |s| < tau set
        to zero; the diagonal is always kept.

C is taken in increasing index order.  With tau = 0 and no coupling between
different pivots, [[I, 0], [L_F, I]] diag(D_B, S') [[I, L_F^T], [0, I]] equals
As permuted to (B, C) order; the tests check that identity.

Imported only by the tests.
"""
import numpy as np


def pivot_block_matrix(As, blocks):
    """D_B for the given pivot blocks (lists of one or two indices), in the
    order of the blocks."""
    idx = [i for b in blocks for i in b]
    D = np.zeros((len(idx), len(idx)))
    o = 0
    for b in blocks:
        k = len(b)
        D[o:o + k, o:o + k] = As[np.ix_(b, b)]
        o += k
    return D


def eliminate_level(As, blocks, tau):
    """(B, C, D_B, L_F, S') of one level; B is the pivot order (blocks
    concatenated), C the remaining indices ascending; L_F has shape
    (len(C), len(B)) and S' shape (len(C), len(C))."""
    As = np.asarray(As, dtype=np.float64)
    n = As.shape[0]
    B = [i for b in blocks for i in b]
    inB = np.zeros(n, dtype=bool)
    inB[B] = True
    C = [i for i in range(n) if not inB[i]]
    D = pivot_block_matrix(As, blocks)
    LF = As[np.ix_(C, B)] @ np.linalg.inv(D)
    LF[np.abs(LF) < tau] = 0.0
    S = As[np.ix_(C, C)] - LF @ D @ LF.T
    S = 0.5 * (S + S.T)  # exactly symmetric; the two triangles agree to rounding
    off = ~np.eye(len(C), dtype=bool)
    S[off & (np.abs(S) < tau)] = 0.0
    return B, C, D, LF, S
