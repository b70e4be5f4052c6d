"""Matching, cycle split, scaling and factor application (oracle side).

* :func:`max_product_assignment` -- Section 5.1: the permutation sigma that
  maximises prod_i |a_{sigma(i) i}| (Eq. (5.1)), found by minimising
  sum_i c_{sigma(i) i} with c_ij = log a_i - log |a_ij|, a_i = max_j |a_ij|
  (Eq. (5.2)).  Dense O(n^3) Kuhn–Munkres (shortest augmenting paths with
  row and column potentials), written out plainly; it returns the duals that
  certify optimality (u_i + v_j <= c_ij everywhere, equality on the
  assignment).
* :func:`cycles` / :func:`split_cycle` -- Section 5.2: the cycle form of the
  matching permutation and its split into 2-cycles plus one 1-cycle for odd
  cycles.
* :func:`symmetric_scaling` -- the scaling of Section 4.2 built from the
  duals: D_i = sqrt(exp(u_i + v_i) / a_i), after which every entry of D A D
  is at most one in modulus and matched entries equal one.
* :func:`apply_factor` -- the plain definition of the preconditioner
  application K^{-1} b = P^T S L^{-T} D^{-1} L^{-1} S P b for a factor given
  in the library's exported layout (two sparse triangular solves and a
  block diagonal solve, by scipy's library routines).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl


def costs(A):
    """Dense cost matrix c[i, j] = log a_i - log|a_ij| (inf where a_ij = 0)."""
    A = np.asarray(A, dtype=np.float64)
    a = np.abs(A).max(axis=1)
    a[a == 0] = 1.0
    with np.errstate(divide="ignore"):
        c = np.log(a)[:, None] - np.log(np.abs(A))
    c[A == 0] = np.inf
    return c


def max_product_assignment(A):
    """Returns (col_of_row, u, v, total_cost): row i is matched to column
    col_of_row[i], i.e. sigma(col) = row with a_{row, col} on the diagonal of
    P_M A.  u (rows) and v (columns) are feasible duals with equality on the
    assignment."""
    c = costs(A)
    n = c.shape[0]
    INF = np.inf
    u = np.zeros(n + 1)
    v = np.zeros(n + 1)
    p = np.zeros(n + 1, dtype=int)      # p[j] = row matched to column j (1-based, 0 = none)
    way = np.zeros(n + 1, dtype=int)
    # 1-based shortest augmenting path algorithm with potentials
    for i in range(1, n + 1):
        p[0] = i
        j0 = 0
        minv = np.full(n + 1, INF)
        used = np.zeros(n + 1, dtype=bool)
        while True:
            used[j0] = True
            i0 = p[j0]
            delta = INF
            j1 = -1
            for j in range(1, n + 1):
                if not used[j]:
                    cur = c[i0 - 1, j - 1] - u[i0] - v[j]
                    if cur < minv[j]:
                        minv[j] = cur
                        way[j] = j0
                    if minv[j] < delta:
                        delta = minv[j]
                        j1 = j
            if j1 < 0 or delta == INF:
                raise ValueError("structurally singular: no perfect matching")
            for j in range(n + 1):
                if used[j]:
                    u[p[j]] += delta
                    v[j] -= delta
                else:
                    minv[j] -= delta
            j0 = j1
            if p[j0] == 0:
                break
        while True:
            j1 = way[j0]
            p[j0] = p[j1]
            j0 = j1
            if j0 == 0:
                break
    col_of_row = np.empty(n, dtype=int)
    for j in range(1, n + 1):
        col_of_row[p[j] - 1] = j - 1
    # In this formulation u_i + v_j <= c_ij with v carrying the negated
    # potential; return duals in the convention u_i + v_j <= c_ij.
    uu = u[1:].copy()
    vv = v[1:].copy()
    total = float(sum(c[i, col_of_row[i]] for i in range(n)))
    return col_of_row, uu, vv, total


def row_of_col(col_of_row):
    r = np.empty_like(col_of_row)
    r[col_of_row] = np.arange(len(col_of_row))
    return r


def cycles(match_col):
    """Cycles of the permutation j -> match_col[j] (match_col[j] = row matched
    to column j), each as a list starting at its smallest member and following
    the permutation."""
    n = len(match_col)
    seen = np.zeros(n, dtype=bool)
    out = []
    for j0 in range(n):
        if seen[j0]:
            continue
        cyc = []
        j = j0
        while not seen[j]:
            seen[j] = True
            cyc.append(int(j))
            j = int(match_col[j])
        out.append(cyc)
    return out


def split_cycle(cyc, singleton_position):
    """Split one cycle into consecutive pairs, leaving the member at
    ``singleton_position`` alone for odd cycles (for even cycles the position
    selects which of the two splits: pairs start at position 0 or 1)."""
    m = len(cyc)
    if m == 1:
        return [(cyc[0],)]
    if m % 2 == 0:
        s = singleton_position % 2
        return [tuple(sorted((cyc[(s + k) % m], cyc[(s + k + 1) % m]))) for k in range(0, m, 2)]
    t = singleton_position
    groups = [(cyc[t],)]
    for k in range(1, m, 2):
        groups.append(tuple(sorted((cyc[(t + k) % m], cyc[(t + k + 1) % m]))))
    return groups


def symmetric_scaling(A, u, v):
    """D_i = sqrt(exp(u_i + v_i) / a_i) with a_i the row maxima of |A|."""
    a = np.abs(np.asarray(A)).max(axis=1)
    a[a == 0] = 1.0
    return np.sqrt(np.exp(u + v) / a)


def apply_factor(F, b):
    """K^{-1} b for an exported factor F (dict of arrays as produced by the
    library's export): (P b)[p] = b[perm[p]], S = diag(scale), unit lower L
    in CSR by positions, D^{-1} given per position (1x1 / 2x2 via partner)
    and the dense trailing block's inverse."""
    perm = np.asarray(F["perm"])
    s = np.asarray(F["scale"])
    n = len(perm)
    lp = np.asarray(F["level_ptr"])
    d0 = int(lp[-2])
    Lfull = sp.csr_matrix((F["Lval"], F["Lcol"], F["Lptr"]), shape=(n, n)) + sp.identity(n, format="csr")
    w = s * np.asarray(b, dtype=np.float64)[perm]
    y = spl.spsolve_triangular(Lfull, w, lower=True)
    z = np.empty(n)
    dd, do, pt = F["dinv_d"], F["dinv_o"], F["partner"]
    for p in range(d0):
        z[p] = dd[p] * y[p] + (do[p] * y[pt[p]] if pt[p] >= 0 else 0.0)
    if n > d0:
        z[d0:] = np.asarray(F["dense_inv"]) @ y[d0:]
    x = spl.spsolve_triangular(Lfull.T.tocsr(), z, lower=False)
    out = np.empty(n)
    out[perm] = s * x
    return out
