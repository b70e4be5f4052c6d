"""The first Gram-Schmidt pass on the tensor cores (jd_gram_bf16: BF16
operands, FP32 accumulation, tcgen05.mma) against the same products formed
in binary64 from the BF16-rounded operands, and the orthonormality of the
search space that the BF16 first pass plus the binary64 second pass leave
inside Jacobi-Davidson solves."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ajd():
    import paper_math_0508111_gb300 as ajd
    assert torch.cuda.is_available()
    return ajd


def to_bf16(x):
    """Round binary64 values to the nearest BF16 (8 significant bits, ties to
    even), returned as binary64."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def test_bf16_rounding_helper():
    assert to_bf16(1.0) == 1.0
    assert to_bf16(1.0 + 2.0 ** -9) == 1.0           # tie to even
    assert to_bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7
    assert to_bf16(-3.14159) == -3.140625


@pytest.mark.parametrize("n,c", [(1, 1), (100003, 1), (100003, 5), (65536, 37), (250001, 128), (777, 64)])
def test_gram_bf16_matches_rounded_products(ajd, n, c):
    g = np.random.default_rng(n + c)
    X = g.standard_normal((c, n))             # column j of X is row j (column-major n x c)
    t = g.standard_normal(n)
    Xd = torch.tensor(X, device="cuda")
    td = torch.tensor(t, device="cuda")
    out = np.zeros(c)
    vp = ctypes.c_void_p
    ajd._ffi.call("jd_gram_bf16", vp(Xd.data_ptr()), n, c, vp(td.data_ptr()), n, out.ctypes.data_as(vp), None)
    Xr, tr = to_bf16(X), to_bf16(t)
    want = Xr @ tr
    scale = np.abs(Xr) @ np.abs(tr)
    # FP32 accumulation within a chunk of rows per CTA, binary64 across CTAs
    assert np.all(np.abs(out - want) <= 1e-5 * scale + 1e-30), np.max(np.abs(out - want) / scale)
    # the BF16 products are a close (first-pass) estimate of the binary64 ones
    assert np.all(np.abs(out - X @ t) <= 2e-2 * np.abs(X) @ np.abs(t))


def test_gram_bf16_rejects_bad_sizes(ajd):
    L = ajd._ffi.lib()
    x = torch.zeros(10, device="cuda", dtype=torch.float64)
    out = np.zeros(200)
    vp = ctypes.c_void_p
    assert L.jd_gram_bf16(vp(x.data_ptr()), 10, 129, vp(x.data_ptr()), 10, out.ctypes.data_as(vp), None) \
        == ajd.JD_EINVAL
    assert L.jd_gram_bf16(vp(x.data_ptr()), 5, 1, vp(x.data_ptr()), 10, out.ctypes.data_as(vp), None) == ajd.JD_EINVAL


@pytest.mark.parametrize("gram,prec", [(2, 2), (2, 0), (1, 2), (0, 1)])
def test_search_space_orthonormal(ajd, gram, prec):
    """After every expansion the basis V is orthonormal to binary64 accuracy,
    with the BF16 first pass (gram 2; the default for the mixed and binary32
    inner solves) and with two binary64 passes (gram 1)."""
    from pairs import check_pairs
    L, W, seed, sigma, k = 14, 16.5, 21, 0.0, 5
    tol = 1e-11 if prec == 0 else 1e-10
    with ajd.Anderson(L, W, seed) as h:
        ev, X, st = ajd.solve(h, sigma, k, tol, precision=prec, gram=gram)
    assert st["basis_orth_error"] <= 1e-13, st["basis_orth_error"]
    if prec != 1:
        check_pairs(L, W, seed, 0, sigma, k, ev, X, st, tol)


def test_search_space_orthonormal_full_size(ajd):
    """The L = 50 workload with the default mixed solve (BF16 first pass)."""
    with ajd.Anderson(50, 16.5, 2) as h:
        ev, X, st = ajd.solve(h, 0.0, 5, 1e-8, precision=ajd.JD_MIXED, vectors=False)
    assert st["nconv"] == 5
    assert st["basis_orth_error"] <= 1e-13, st["basis_orth_error"]
