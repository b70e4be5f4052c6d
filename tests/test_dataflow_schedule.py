"""The work units of the dataflow preconditioner apply (CPU; the schedule
is built on the host).  The kernel lets every row start as soon as the
values it reads are written and has no other synchronisation, so its
correctness and its freedom from deadlock rest on properties of the unit
sequence that ildl_dataflow_schedule exposes: the units cover every row of
the forward sweep, the dense tail and the backward sweep exactly once, and
every value a unit reads (Section 6: L's entries in the forward sweep, L^T's
and the 2x2 pivots' forward values in the backward sweep, the whole forward
dense block in the dense tail) is written by an earlier unit.  Warps take
units in increasing order and are all resident, so the holder of the
earliest unfinished unit can always proceed."""
import ctypes

import numpy as np
import pytest

from oracle import lattice, rng

GATHER, FWD, DENSE, BWD = 0, 1, 2, 3


@pytest.fixture(scope="module")
def ajd():
    import paper_math_0508111_gb300 as ajd
    return ajd


def schedule(ajd, P, shift):
    nseg, nunits = ctypes.c_int(0), ctypes.c_int(0)
    vp = ctypes.c_void_p
    lib = ajd._ffi.lib()
    # first call sizes the segment list
    rc = lib.ildl_dataflow_schedule(P.handle, shift, None, 0, ctypes.byref(nseg), ctypes.byref(nunits))
    assert rc == ajd.JD_EINVAL and nseg.value > 0
    seg = np.zeros(5 * nseg.value, dtype=np.int32)
    ajd._ffi.call("ildl_dataflow_schedule", P.handle, shift, seg.ctypes.data_as(vp), nseg.value,
                  ctypes.byref(nseg), ctypes.byref(nunits))
    return seg.reshape(-1, 5), nunits.value


def unit_of_rows(kind, G, p0, p1, u0):
    per = 32 if kind == GATHER else (1 if kind == DENSE else 32 // G)
    p = np.arange(p0, p1)
    return p, u0 + (p - p0) // per, (p1 - p0 + per - 1) // per


def check_schedule(F, seg, nunits):
    n = len(F["perm"])
    lp = np.asarray(F["level_ptr"])
    nl = len(lp) - 2
    d0 = int(lp[nl])
    Lptr = np.asarray(F["Lptr"])
    nnz = int(Lptr[-1])
    Lcol = np.asarray(F["Lcol"][:nnz])
    rows = np.repeat(np.arange(n), np.diff(Lptr))
    partner = np.asarray(F["partner"])
    kinds = seg[:, 0]
    # segment order: level 0, forward levels, the dense tail, backward levels
    assert kinds[0] == GATHER and (np.diff(kinds) >= 0).all()
    assert set(kinds.tolist()) <= {GATHER, FWD, DENSE, BWD}
    assert (kinds == DENSE).sum() == (1 if n > d0 else 0)
    wunit = np.full(n, -1)
    zunit = np.full(n, -1)
    nxt = 0
    for kind, G, p0, p1, u0 in seg:
        assert G in (1, 2, 4, 8, 16, 32) and 0 <= p0 < p1 <= n
        assert u0 == nxt, "units are numbered without gaps"
        p, u, cnt = unit_of_rows(kind, G, p0, p1, u0)
        nxt = u0 + cnt
        if kind in (GATHER, FWD):
            assert (wunit[p] < 0).all()
            wunit[p] = u
        else:
            assert (zunit[p] < 0).all()
            zunit[p] = u
        if kind == DENSE:
            assert G == 32 and p0 == d0 and p1 == n
    assert nxt == nunits
    # every row written once in each sweep
    assert (wunit >= 0).all() and (zunit >= 0).all()
    # level 0 rows read nothing in the forward sweep; forward rows read
    # earlier forward values only
    assert (wunit[Lcol] < wunit[rows]).all()
    # backward row p reads z of the rows q > p with L[q, p] != 0 and the
    # forward values of itself and its 2x2 partner
    bwd = rows < d0
    assert (zunit[rows] < zunit[Lcol]).all()
    pos = np.arange(d0)
    assert (wunit[pos] < zunit[pos]).all()
    has = partner[:d0] >= 0
    assert (wunit[partner[:d0][has]] < zunit[pos[has]]).all()
    # the dense tail reads the whole forward dense block
    if n > d0:
        assert wunit[d0:].max() < zunit[d0:].min()
    return bwd.sum()


@pytest.mark.parametrize("L,W,seed,sigma,kw", [
    (12, 16.5, 1, 0.0, {"n_dense": 100}),
    (16, 12.0, 2, 0.7, {"n_dense": 300}),
    (20, 16.5, 3, -0.4, {"n_dense": 200}),
    (14, 16.5, 4, 0.3, {"n_dense": 100, "drop": 0.0}),   # long deep rows
    (10, 8.0, 5, 0.0, {"n_dense": 2000}),                # all dense
])
def test_dataflow_units_cover_and_respect_dependencies(ajd, L, W, seed, sigma, kw):
    A = lattice.assemble(L, rng.potential(L, W, seed), shift=sigma).tocsr()
    A.sort_indices()
    P = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, **kw)
    F = P.export()
    for shift in (-1, 0, 1):
        seg, nunits = schedule(ajd, P, shift)
        check_schedule(F, seg, nunits)


def test_dataflow_schedule_lanes_follow_row_length(ajd):
    """Lanes per row grow with the level's mean row length (about six stored
    entries per lane, at most 32), and the shift scales them by 2^shift."""
    L = 18
    A = lattice.assemble(L, rng.potential(L, 16.5, 6)).tocsr()
    A.sort_indices()
    P = ajd.Preconditioner.from_csr(A.indptr, A.indices, A.data, n_dense=200)
    F = P.export()
    Lptr = np.asarray(F["Lptr"])
    seg0, _ = schedule(ajd, P, 0)
    for kind, G, p0, p1, _ in seg0:
        if kind != FWD:
            continue
        avg = (Lptr[p1] - Lptr[p0]) / (p1 - p0)
        want = 1
        while want < 32 and 2 * want <= avg / 6.0:
            want *= 2
        assert G == want, (p0, p1, avg, G)
    segm, _ = schedule(ajd, P, -1)
    segp, _ = schedule(ajd, P, 1)
    sparse = np.isin(seg0[:, 0], (FWD, BWD))
    assert (segm[sparse, 1] == np.maximum(seg0[sparse, 1] // 2, 1)).all()
    assert (segp[sparse, 1] == np.minimum(seg0[sparse, 1] * 2, 32)).all()
    lib = ajd._ffi.lib()
    n1, n2 = ctypes.c_int(0), ctypes.c_int(0)
    assert lib.ildl_dataflow_schedule(P.handle, 2, None, 0, ctypes.byref(n1),
                                      ctypes.byref(n2)) == ajd.JD_EINVAL
