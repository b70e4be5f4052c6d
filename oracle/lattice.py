"""The Anderson matrix of Eq. (1), assembled explicitly (oracle side).

Eq. (1) couples every site (i, j, k) of an M x M x M lattice to its six
nearest neighbours with unit hopping and puts the random energy
eps_{i;j;k} on the diagonal.  Readings used here:

* sites are numbered from 0 with x fastest: idx = x + L*(y + L*z);
* the hopping amplitude is ``t`` (default -1, the sign the project's
  configurations use; Eq. (1) prints +1).  For any disorder,
  H_{-1}(eps) = -H_{+1}(-eps), and on a bipartite lattice (even L
  periodic, or any hard wall) the two signs give the same spectrum;
* periodic boundaries (the default of every table) wrap x+1 = L to 0.
  L < 3 is rejected because the +1 and -1 neighbours coincide;
* hard-wall boundaries (Section 7, Table 6) set x_0 = x_{M+1} = 0, i.e.
  drop the couplings that would leave the cube.

The product matrix-vector multiply is the plain sparse product ``A @ x``.
"""
import numpy as np
import scipy.sparse as sp

PERIODIC = 0
HARDWALL = 1


def _coords(L):
    idx = np.arange(L ** 3, dtype=np.int64)
    return idx, idx % L, (idx // L) % L, idx // (L * L)


def bonds(L, bc):
    """Undirected nearest-neighbour bonds as two index arrays (a, b), each
    bond listed once (a -> its +x, +y or +z neighbour b)."""
    if bc == PERIODIC and L < 3:
        raise ValueError("periodic lattice needs L >= 3")
    if bc not in (PERIODIC, HARDWALL):
        raise ValueError("bc must be 0 (periodic) or 1 (hard wall)")
    idx, x, y, z = _coords(L)
    A, B = [], []
    for d in range(3):
        c = (x, y, z)[d]
        if bc == HARDWALL:
            keep = c < L - 1
        else:
            keep = np.ones_like(c, dtype=bool)
        nx, ny, nz = x.copy(), y.copy(), z.copy()
        if d == 0:
            nx = (x + 1) % L
        elif d == 1:
            ny = (y + 1) % L
        else:
            nz = (z + 1) % L
        nb = nx + L * (ny + L * nz)
        A.append(idx[keep])
        B.append(nb[keep])
    return np.concatenate(A), np.concatenate(B)


def assemble(L, eps, bc=PERIODIC, t=-1.0, shift=0.0):
    """Sparse CSR matrix A - shift*I of Eq. (1) with hopping t, FP64."""
    n = L ** 3
    eps = np.asarray(eps, dtype=np.float64)
    assert eps.shape == (n,)
    a, b = bonds(L, bc)
    rows = np.concatenate([a, b, np.arange(n)])
    cols = np.concatenate([b, a, np.arange(n)])
    vals = np.concatenate([np.full(a.size, t), np.full(a.size, t), eps - shift])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def assemble_offdiag(L, diag, hop, bc=PERIODIC, shift=0.0):
    """Sparse CSR matrix A - shift*I of the off-diagonal Anderson model
    (Section 7): diagonal ``diag`` (a scalar or an array of n values) and the
    hopping hop[s, d] on the bond from site s to its +x/+y/+z neighbour
    (d = 0/1/2), the same graph as Eq. (1).  Hard walls drop the bonds that
    would leave the cube (their hop entries are not used).  FP64."""
    n = L ** 3
    if bc == PERIODIC and L < 3:
        raise ValueError("periodic lattice needs L >= 3")
    hop = np.asarray(hop, dtype=np.float64)
    assert hop.shape == (n, 3)
    d_all = np.broadcast_to(np.asarray(diag, dtype=np.float64), (n,))
    idx, x, y, z = _coords(L)
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [d_all - shift]
    for d in range(3):
        c = (x, y, z)[d]
        keep = c < L - 1 if bc == HARDWALL else np.ones(n, dtype=bool)
        step = L ** d
        nb = np.where(c == L - 1, idx - (L - 1) * step, idx + step)  # the +d neighbour, wrapped
        a, b, t = idx[keep], nb[keep], hop[keep, d]
        rows += [a, b]
        cols += [b, a]
        vals += [t, t]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def norm_bound_offdiag(diag, hop):
    """Gershgorin bound max|diag| + 6 max|t| of the off-diagonal model (the
    relative tolerances use it as ||A||; with t = -1 it is norm_bound)."""
    return float(np.max(np.abs(diag))) + 6.0 * float(np.max(np.abs(hop)))


def dense(L, eps, bc=PERIODIC, t=-1.0, shift=0.0):
    return assemble(L, eps, bc, t, shift).toarray()


def matvec(L, eps, x, bc=PERIODIC, t=-1.0, shift=0.0):
    """y = (A - shift*I) x by the assembled sparse matrix (FP64).  ``x`` may
    be a vector or an n x m block."""
    return assemble(L, eps, bc, t, shift) @ np.asarray(x, dtype=np.float64)


def norm_bound(eps):
    """||A|| as used for relative tolerances: 6 + max|eps_i|, the Gershgorin
    radius that gives the spectral interval [-6 - w/2, 6 + w/2] quoted in
    Section 3 (after Eq. (1))."""
    return 6.0 + float(np.max(np.abs(eps))) if len(eps) else 6.0


def closed_form_spectrum(L, bc=PERIODIC, t=-1.0):
    """All eigenvalues of the disorder-free (W = 0) matrix of Eq. (1).

    The hopping part is a Kronecker sum of three 1D chains.  A periodic
    chain of length L has eigenvalues 2t cos(2 pi m / L), m = 0..L-1
    (eigenvectors exp(2 pi i m x / L)); a chain with hard walls has
    2t cos(pi m / (L+1)), m = 1..L (eigenvectors sin(pi m x / (L+1))).
    The 3D eigenvalues are all sums of one value per direction.
    """
    if bc == PERIODIC:
        c = 2.0 * t * np.cos(2.0 * np.pi * np.arange(L) / L)
    else:
        c = 2.0 * t * np.cos(np.pi * np.arange(1, L + 1) / (L + 1))
    s = c[:, None, None] + c[None, :, None] + c[None, None, :]
    return np.sort(s.ravel())


def plane_wave(L, m, bc=PERIODIC):
    """A real eigenvector of the W = 0 matrix for wave numbers m = (mx, my, mz):
    cos(2 pi m.r / L) for periodic boundaries, prod sin(pi m_d (r_d+1)/(L+1))
    for hard walls (r_d 0-based).  Returned normalised."""
    _, x, y, z = _coords(L)
    if bc == PERIODIC:
        v = np.cos(2.0 * np.pi * (m[0] * x + m[1] * y + m[2] * z) / L)
    else:
        v = (np.sin(np.pi * m[0] * (x + 1) / (L + 1))
             * np.sin(np.pi * m[1] * (y + 1) / (L + 1))
             * np.sin(np.pi * m[2] * (z + 1) / (L + 1)))
    return v / np.linalg.norm(v)


def plane_wave_eigenvalue(L, m, bc=PERIODIC, t=-1.0):
    if bc == PERIODIC:
        return 2.0 * t * sum(np.cos(2.0 * np.pi * md / L) for md in m)
    return 2.0 * t * sum(np.cos(np.pi * md / (L + 1)) for md in m)
