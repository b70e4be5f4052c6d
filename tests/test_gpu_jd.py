"""GPU parity of the preconditioner apply and of the Jacobi–Davidson
eigenpairs against the CPU oracle."""
import numpy as np
import pytest

from oracle import eig, lanczos, lattice, matching, rng
from pairs import check_pairs as _check_pairs
from pairs import check_pairs_certified

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ajd():
    import paper_math_0508111_gb300 as ajd
    assert torch.cuda.is_available()
    return ajd


# Tolerances of the apply against the oracle, relative to max|x|.  The
# binary32 and mixed applies use the factor's values rounded to binary32
# (the device copy they read); the oracle applies that same rounded factor
# in binary64, so what remains is the kernel's own arithmetic: binary64
# sums, float-float sums (about 48 bits) and binary32 sums (24 bits,
# with b rounded to binary32 as the kernel receives it).
TOL_APPLY = {"fp64": 1e-12, "mixed": 1e-11, "fp32": 1e-5}
# the same kernels against the unrounded binary64 factor: rounding the
# stored values to binary32 is a small change of the preconditioner
TOL_APPLY_UNROUNDED = 2e-5


def rounded32(F):
    """The factor with every stored value rounded to binary32 (scale, L, the
    1x1/2x2 pivot inverses, the dense tail inverse), as on the device."""
    G = dict(F)
    for key in ["scale", "Lval", "dinv_d", "dinv_o", "dense_inv"]:
        G[key] = np.asarray(F[key]).astype(np.float32).astype(np.float64)
    return G


def apply_errors(P, F, b):
    """Relative max errors of the three device applies against the oracle on
    the factor each one reads."""
    want = matching.apply_factor(F, b)
    F32 = rounded32(F)
    want_m = matching.apply_factor(F32, b)
    b32 = b.astype(np.float32)
    want_32 = matching.apply_factor(F32, b32.astype(np.float64))
    x64 = P.apply(torch.tensor(b, device="cuda")).cpu().numpy()
    xm = P.apply(torch.tensor(b, device="cuda"), mixed=True).cpu().numpy()
    x32 = P.apply(torch.tensor(b32, device="cuda")).double().cpu().numpy()
    err = {"fp64": np.abs(x64 - want).max() / np.abs(want).max(),
           "mixed": np.abs(xm - want_m).max() / np.abs(want_m).max(),
           "fp32": np.abs(x32 - want_32).max() / np.abs(want_32).max(),
           "mixed_unrounded": np.abs(xm - want).max() / np.abs(want).max(),
           "fp32_unrounded": np.abs(x32 - want).max() / np.abs(want).max()}
    assert all(np.isfinite(v) for v in err.values()), err
    return err


def check_apply_errors(err):
    for key, tol in TOL_APPLY.items():
        assert err[key] <= tol, (key, err)
    assert err["mixed_unrounded"] <= TOL_APPLY_UNROUNDED, err
    assert err["fp32_unrounded"] <= TOL_APPLY_UNROUNDED, err


FORMS = [0, 1]  # apply kernels: level counters, dataflow


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("L,bc,sigma,nd", [(10, 0, 0.0, 1000), (20, 0, 0.3, 1000), (33, 1, -0.5, 300), (16, 0, 1.0, 50)])
def test_ildl_apply_matches_oracle(ajd, L, bc, sigma, nd, form):
    """x = K^{-1} b on the GPU equals the plain definition applied by the
    oracle to the same factor (binary64, mixed and binary32), in both apply
    forms."""
    with ajd.Anderson(L, 16.5, 1, bc) as h:
        P = ajd.Preconditioner.from_lattice(h, sigma, n_dense=nd, apply_form=form)
        assert P.info()["apply_form"] == form
        F = P.export()
        b = np.random.default_rng(0).standard_normal(h.n)
        check_apply_errors(apply_errors(P, F, b))
        P.close()


def test_ildl_apply_forms_agree(ajd):
    """The level-counter and the dataflow kernels form the same products,
    summed in different orders (their rows are split over different numbers
    of lanes): their binary64 results agree to rounding, and repeated
    dataflow applies of the same vector give the same bits (each row's sum
    is formed by one fixed set of lanes in a fixed order, whatever the
    timing)."""
    with ajd.Anderson(30, 16.5, 7) as h:
        P0 = ajd.Preconditioner.from_lattice(h, 0.1, apply_form=0)
        P1 = ajd.Preconditioner.from_lattice(h, 0.1, apply_form=1)
        b = torch.tensor(np.random.default_rng(9).standard_normal(h.n), device="cuda")
        x0 = P0.apply(b).cpu().numpy()
        x1 = P1.apply(b).cpu().numpy()
        assert np.abs(x0 - x1).max() <= 1e-12 * np.abs(x0).max()
        for mixed in (False, True):
            r1 = P1.apply(b, mixed=mixed).cpu().numpy()
            r2 = P1.apply(b, mixed=mixed).cpu().numpy()
            assert np.array_equal(r1.view(np.int64), r2.view(np.int64))
        P0.close()
        P1.close()


def test_ildl_apply_autotuned(ajd):
    """A factor of more than 200,000 rows has its apply tuned on the device
    (the two kernels, each with the rule's threads per row times 1/2, 1 or
    2, whichever runs fastest); whatever the choice, the apply equals the
    oracle's.  A kernel fixed by the caller is tuned over the threads per
    row only."""
    with ajd.Anderson(60, 16.5, 4) as h:
        P = ajd.Preconditioner.from_lattice(h, 0.2)
        assert P.info()["apply_shift"] in (-1, 0, 1)
        assert P.info()["apply_form"] in (0, 1)
        b = np.random.default_rng(5).standard_normal(h.n)
        check_apply_errors(apply_errors(P, P.export(), b))
        P.close()
        for form in FORMS:
            P1 = ajd.Preconditioner.from_lattice(h, 0.2, apply_form=form)
            assert P1.info()["apply_form"] == form
            check_apply_errors(apply_errors(P1, P1.export(), b))
            P1.close()
        P0 = ajd.Preconditioner.from_lattice(h, 0.2, autotune=0)
        assert P0.info()["apply_shift"] == 0
        P0.close()


@pytest.mark.parametrize("form", FORMS)
def test_ildl_apply_wide_rows(ajd, form):
    """A factor without dropping has few, long rows on its deepest levels:
    those phases run with 64..512 threads per row (CTA-wide rows with a
    shared-memory reduction) in the level-counter kernel and with a warp
    per row and many batches in the dataflow kernel, and must still equal
    the oracle's apply."""
    with ajd.Anderson(22, 16.5, 1) as h:
        P = ajd.Preconditioner.from_lattice(h, 0.3, n_dense=200, drop=0.0, apply_form=form)
        F = P.export()
        assert P.info()["nnz_L"] > 5 * 10 ** 6  # deep rows of several hundred to thousands of entries
        b = np.random.default_rng(3).standard_normal(h.n)
        err = apply_errors(P, F, b)
        # without dropping the deep rows are long and the factor's entries
        # large: rounding the stored values moves K^{-1} b by more than the
        # default factor's 2e-5, but the kernels' own arithmetic (against
        # the rounded factor) stays at the usual bounds
        for key, tol in TOL_APPLY.items():
            assert err[key] <= tol, (key, err)
        assert err["mixed_unrounded"] <= 1e-3 and err["fp32_unrounded"] <= 1e-3, err
        P.close()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("L,bc,sigma,nd", [(12, 1, -1.0, 200), (20, 0, 0.3, 1000)])
def test_ildl_apply_no_read_before_write(ajd, monkeypatch, L, bc, sigma, nd, form):
    """Work vectors filled with NaN before the first apply (AJD_POISON_ALLOC):
    every apply must still equal the oracle's, so no entry of w or z is read
    before this apply wrote it (padding lanes of a row included).  The
    dataflow kernel refills them with its own sentinel before every apply
    and waits on it, so there a read before the write would hang until the
    bounded wait reports JD_EDEVICE instead."""
    monkeypatch.setenv("AJD_POISON_ALLOC", "1")
    with ajd.Anderson(L, 12.0, 12, bc) as h:
        P = ajd.Preconditioner.from_lattice(h, sigma, n_dense=nd, apply_form=form)
        assert P.info()["levels"] >= 2
        b = np.random.default_rng(0).standard_normal(h.n)
        check_apply_errors(apply_errors(P, P.export(), b))
        P.close()


@pytest.mark.parametrize("L,bc,sigma", [(8, 0, 0.0), (9, 1, 0.7)])
def test_dense_tail_inverse_is_exact(ajd, L, bc, sigma):
    """When the whole matrix fits the dense tail, K = A - sigma I exactly: the
    device Gauss-Jordan inverse must reproduce (A - sigma I)^{-1}."""
    with ajd.Anderson(L, 16.5, 2, bc) as h:
        P = ajd.Preconditioner.from_lattice(h, sigma)
        assert P.info()["n_dense"] == h.n
        A = lattice.assemble(L, rng.potential(L, 16.5, 2), bc, shift=sigma)
        x = np.random.default_rng(1).standard_normal(h.n)
        y = P.apply(torch.tensor(A @ x, device="cuda")).cpu().numpy()
        assert np.linalg.norm(y - x) <= 1e-9 * np.linalg.norm(x)
        F = P.export()
        assert np.linalg.norm(matching.apply_factor(F, A @ x) - x) <= 1e-9 * np.linalg.norm(x)
        P.close()


@pytest.mark.parametrize("L,nd", [(10, 200), (12, 1100), (8, 512)])
def test_multilevel_factor_exact_on_device(ajd, L, nd):
    """No dropping, exact independence, kappa = inf: the device apply of the
    multilevel factor (sparse levels + device-inverted dense tail) inverts
    A - sigma I.  The dense tails span one partial panel of the blocked
    Gauss-Jordan inversion (200 rows: 7 panels of 32, the last of 8), many
    panels over all eight row ranges of its cluster (1100 rows), and the
    whole matrix (L = 8: 512 rows, no sparse level)."""
    sigma = 0.3
    with ajd.Anderson(L, 16.5, 3) as h:
        P = ajd.Preconditioner.from_lattice(h, sigma, drop=0.0, kappa=1e300, gamma=0.0, n_dense=nd)
        if nd < h.n:
            assert P.info()["levels"] >= 2
        A = lattice.assemble(L, rng.potential(L, 16.5, 3), 0, shift=sigma)
        x = np.random.default_rng(2).standard_normal(h.n)
        y = P.apply(torch.tensor(A @ x, device="cuda")).cpu().numpy()
        assert np.linalg.norm(y - x) <= 1e-8 * np.linalg.norm(x)
        P.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_jd_tiny_config(ajd, precision):
    """L = 10, W = 16.5, periodic, 5 eigenpairs nearest 0."""
    L, W, seed, sigma, k = 10, 16.5, 1, 0.0, 5
    tol = 1e-11 if precision == 0 else 1e-10  # a binary32 inner solve stalls near 1e-12
    with ajd.Anderson(L, W, seed) as h:
        ev, X, st = ajd.solve(h, sigma, k, tol, precision=precision)
    _check_pairs(L, W, seed, 0, sigma, k, ev, X, st, tol)


@pytest.mark.parametrize("L,W,seed,bc,sigma,k,prec", [
    (8, 16.5, 2, 1, 0.5, 3, 0),
    (12, 12.0, 3, 0, -1.0, 10, 1),
    (9, 21.0, 4, 0, 0.0, 1, 0),
    (11, 16.5, 5, 1, 2.0, 6, 1),
    (6, 8.0, 6, 0, 0.25, 4, 0),
])
def test_jd_dense_oracle_cases(ajd, L, W, seed, bc, sigma, k, prec):
    tol = 1e-11 if prec == 0 else 1e-10
    with ajd.Anderson(L, W, seed, bc) as h:
        ev, X, st = ajd.solve(h, sigma, k, tol, precision=prec)
    _check_pairs(L, W, seed, bc, sigma, k, ev, X, st, tol)


@pytest.mark.parametrize("L,sigma,prec", [(20, 0.0, 1), (24, 1.0, 0), (27, -0.5, 1)])
def test_jd_shift_invert_oracle(ajd, L, sigma, prec):
    """Mid sizes against the shift-and-invert Lanczos oracle."""
    W, seed, k = 16.5, 1, 5
    tol = 1e-11 if prec == 0 else 1e-10
    with ajd.Anderson(L, W, seed) as h:
        ev, X, st = ajd.solve(h, sigma, k, tol, precision=prec)
    _check_pairs(L, W, seed, 0, sigma, k, ev, X, st, tol, oracle="lanczos")


@pytest.mark.parametrize("prec", [0, 2])
def test_jd_with_aggressive_dropping(ajd, prec):
    """Jacobi-Davidson preconditioned by a factor with Section 6.3's
    aggressive dropping (tau = 0.1) reaches the dense oracle's pairs."""
    L, W, seed, sigma, k = 14, 16.5, 3, 0.0, 5
    tol = 1e-11 if prec == 0 else 1e-10
    with ajd.Anderson(L, W, seed) as h:
        ev, X, st = ajd.solve(h, sigma, k, tol, precision=prec, ildl=dict(aggressive=0.1, n_dense=300))
    assert st["ildl"]["aggressive_dropped"] > 0
    _check_pairs(L, W, seed, 0, sigma, k, ev, X, st, tol)


@pytest.mark.parametrize("extraction", [0, 1])
def test_jd_extraction_modes(ajd, extraction):
    """Harmonic (default) and standard Ritz extraction reach the same pairs."""
    L, W, seed, sigma, k, tol = 12, 16.5, 7, 0.0, 5, 1e-11
    with ajd.Anderson(L, W, seed) as h:
        ev, X, st = ajd.solve(h, sigma, k, tol, extraction=extraction)
    _check_pairs(L, W, seed, 0, sigma, k, ev, X, st, tol)


def test_jd_degenerate_zero_disorder(ajd):
    """W = 0: eigenvalues of the closed form, degenerate clusters; compare
    eigenvalues and check the returned vectors are eigenvectors."""
    L, k = 4, 4
    with ajd.Anderson(L, 0.0, 1) as h:
        ev, X, st = ajd.solve(h, 1.0, k, 1e-11)
    A = lattice.assemble(L, np.zeros(L ** 3))
    spec = lattice.closed_form_spectrum(L)
    o = eig.order_nearest(spec, 1.0)
    # the cluster at distance 1 (lambda = 0 and 2) straddles k: compare distances
    assert np.allclose(np.abs(ev - 1.0), np.abs(spec[o[:k]] - 1.0), atol=1e-10)
    assert np.linalg.norm(A @ X - X * ev, axis=0).max() <= 1e-10 * 6


def test_jd_small_lattice_and_errors(ajd):
    with ajd.Anderson(3, 16.5, 1) as h:
        ev, X, st = ajd.solve(h, 0.0, 2, 1e-11)
        _check_pairs(3, 16.5, 1, 0, 0.0, 2, ev, X, st, 1e-11)
        with pytest.raises(ajd.JDError):
            ajd.solve(h, 0.0, 27, 1e-8)
        with pytest.raises(ajd.JDError):
            ajd.solve(h, 0.0, 2, 0.0)
        with pytest.raises(ajd.JDError):
            ajd.solve(h, float("nan"), 2, 1e-8)


def test_jd_noconv_reports_prefix(ajd):
    """A too-small outer budget returns JD_ENOCONV with the converged prefix."""
    with ajd.Anderson(12, 16.5, 1) as h:
        ev, X, st = ajd.solve(h, 0.0, 5, 1e-11, max_outer=12, raise_on_noconv=False)
    assert st["status"] == ajd.JD_ENOCONV
    assert 0 <= st["nconv"] < 5


@pytest.mark.parametrize("threads,prec", [(1, 0), (3, 2)])
def test_jd_batch_matches_single_solves(ajd, threads, prec):
    """The pipelined batch returns, per problem, the pairs of the oracle and
    of a single jd_solve of the same problem."""
    cases = [(10, 16.5, 11, 0, 0.0, 4), (12, 12.0, 12, 1, -1.0, 3), (8, 16.5, 13, 0, 0.5, 5),
             (11, 21.0, 14, 0, 1.5, 2), (9, 16.5, 15, 1, 0.0, 6)]
    tol = 1e-11 if prec == 0 else 1e-10
    hs = [ajd.Anderson(L, W, s, bc) for (L, W, s, bc, _, _) in cases]
    try:
        out = ajd.solve_batch(hs, [c[4] for c in cases], [c[5] for c in cases], tol, precision=prec,
                              setup_threads=threads)
        for (L, W, s, bc, sigma, k), h, (ev, X, st) in zip(cases, hs, out):
            _check_pairs(L, W, s, bc, sigma, k, ev, X, st, tol)
            assert st["setup_ms"] > 0
            ev1, _, _ = ajd.solve(h, sigma, k, tol, precision=prec)
            assert np.abs(ev - ev1).max() <= 1e-10 * (6 + W / 2)
    finally:
        for h in hs:
            h.close()


def test_jd_batch_empty_and_errors(ajd):
    assert ajd.solve_batch([], 0.0, 1, 1e-8) == []
    with ajd.Anderson(4, 16.5, 1) as h:
        with pytest.raises(ajd.JDError):
            ajd.solve_batch([h, h], [0.0, 0.0], [2, 64], 1e-8)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_jd_no_read_before_write(ajd, prec, monkeypatch):
    """Every work buffer of the solver and of the preconditioner apply starts
    as NaN (AJD_POISON_ALLOC): a read before the first write would poison the
    solve, so the pairs coming out right shows none happens."""
    monkeypatch.setenv("AJD_POISON_ALLOC", "1")
    tol = 1e-11 if prec == 0 else 1e-10
    for (L, W, s, bc, sigma, k) in [(12, 12.0, 12, 1, -1.0, 3), (11, 21.0, 14, 0, 1.5, 2), (14, 16.5, 16, 0, 0.0, 4)]:
        with ajd.Anderson(L, W, s, bc) as h:
            ev, X, st = ajd.solve(h, sigma, k, tol, precision=prec, ildl={"n_dense": 200})
        _check_pairs(L, W, s, bc, sigma, k, ev, X, st, tol)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("prec", [0, 2])
def test_jd_apply_forms(ajd, form, prec):
    """Jacobi-Davidson with either apply kernel reaches the dense oracle's
    pairs."""
    L, W, s, bc, sigma, k = 16, 16.5, 31, 0, 0.4, 4
    tol = 1e-11 if prec == 0 else 1e-10
    with ajd.Anderson(L, W, s, bc) as h:
        ev, X, st = ajd.solve(h, sigma, k, tol, precision=prec, ildl={"n_dense": 300, "apply_form": form})
    assert st["ildl"]["apply_form"] == form
    _check_pairs(L, W, s, bc, sigma, k, ev, X, st, tol)


@pytest.mark.parametrize("L", [50, 100])
def test_jd_full_size_certificate(ajd, L):
    """The C2 (L = 50) and C3 (L = 100) workloads at full size, in the
    launch configuration of the benchmark (mixed inner solve, tol 1e-8).
    The shift-invert oracle does not reach these sizes in test time, so the
    pairs are pinned by properties the oracle checks at any size: residuals
    computed with the oracle's own matrix (each within tol ||A|| means an
    eigenvalue of A lies within that distance: Weyl / Krylov-Bogoliubov),
    orthonormality, the ordering and sign conventions, and agreement of the
    eigenvalues with an independent binary64 solve (Kato-Temple: both are
    within ||r||^2 / gap of the same eigenvalues)."""
    W, seed, sigma, k, tol = 16.5, 2, 0.0, 5, 1e-8
    eps = rng.potential(L, W, seed)
    nA = lattice.norm_bound(eps)
    with ajd.Anderson(L, W, seed) as h:
        ev, X, st = ajd.solve(h, sigma, k, tol, precision=ajd.JD_MIXED)
        ev64, _, st64 = ajd.solve(h, sigma, k, tol, precision=ajd.JD_FP64, vectors=False)
    assert st["nconv"] == k and st64["nconv"] == k
    A = lattice.assemble(L, eps)
    res = np.linalg.norm(A @ X - X * ev, axis=0)
    assert res.max() <= 2 * tol * nA
    assert np.abs(X.T @ X - np.eye(k)).max() <= 1e-12
    assert np.all(np.diff(np.abs(ev - sigma)) >= 0)
    for j in range(k):
        i = int(np.argmax(np.abs(X[:, j])))
        assert X[i, j] > 0
    # the two solves find the same eigenvalues (both converged to 1e-8 ||A||)
    assert np.abs(ev - ev64).max() <= 1e-10 * nA


@pytest.mark.parametrize("L,W,seed,bc,sigma,k,prec", [
    (10, 16.5, 1, 0, 0.0, 5, 0),
    (9, 12.0, 3, 1, -0.5, 4, 2),
    (12, 16.5, 8, 0, 1.0, 3, 0),
])
def test_lanczos_matches_dense_oracle(ajd, L, W, seed, bc, sigma, k, prec):
    """Shift-and-invert Lanczos over the preconditioned SQMR (Section 4.1)
    reaches the pairs of the dense oracle."""
    tol = 1e-11 if prec == 0 else 1e-10
    with ajd.Anderson(L, W, seed, bc) as h:
        ev, X, st = ajd.solve(h, sigma, k, tol, precision=prec, method="lanczos", ildl={"n_dense": 300})
    _check_pairs(L, W, seed, bc, sigma, k, ev, X, st, tol)
    assert st["outer_its"] <= 64 and st["inner_its"] > 0


@pytest.mark.parametrize("L,W,seed,bc,sigma,k", [(12, 16.5, 8, 0, 1.0, 3), (9, 12.0, 3, 1, -0.5, 4)])
def test_lanczos_binary32(ajd, L, W, seed, bc, sigma, k):
    """Shift-and-invert Lanczos with a binary32 inner solve: each operator
    application (A - sigma I)^{-1} v is only accurate to the binary32 SQMR
    floor (1e-6 relative), so the pairs reach tol = 1e-5 and no further; the
    eigenvalues are pinned to the dense oracle by the Kato-Temple bound of
    each pair's explicit residual."""
    tol = 1e-5
    with ajd.Anderson(L, W, seed, bc) as h:
        ev, X, st = ajd.solve(h, sigma, k, tol, precision=ajd.JD_FP32, method="lanczos", ildl={"n_dense": 300})
    check_pairs_certified(L, W, seed, bc, sigma, k, ev, X, st, tol)


def test_lanczos_agrees_with_jd_mid_size(ajd):
    """At L = 24 (several levels, dense tail 1000) both methods give the same
    eigenvalues, checked against the shift-invert oracle."""
    L, W, seed, sigma, k, tol = 24, 16.5, 4, 0.0, 5, 1e-10
    with ajd.Anderson(L, W, seed) as h:
        ev_l, X_l, st_l = ajd.solve(h, sigma, k, tol, method="lanczos", precision=2)
        ev_j, _, _ = ajd.solve(h, sigma, k, tol, precision=2, vectors=False)
    _check_pairs(L, W, seed, 0, sigma, k, ev_l, X_l, st_l, tol, oracle="lanczos")
    assert np.abs(ev_l - ev_j).max() <= 1e-10 * (6 + W / 2)
