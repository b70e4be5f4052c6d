"""The allocation-free preconditioner application.

``ildl_apply_noalloc`` is for callers that cannot allocate device memory
while they run (a fixed memory pool, an embedding runtime that owns all
device memory, a region that must stay allocation-free).  It runs the same
kernel as ``ildl_apply`` with its scratch taken from a static device array,
so its results must equal ``ildl_apply``'s.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
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


def _noalloc(ajd, P, b, out, precision):
    ajd._ffi.call("ildl_apply_noalloc", P.handle, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                  int(precision), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return out


@pytest.mark.parametrize("L,precision", [(20, 0), (33, 1), (50, 2)])
def test_noalloc_matches_apply_twice(ajd, L, precision):
    with ajd.Anderson(L, 16.5, 5) as h:
        P = ajd.Preconditioner.from_lattice(h, 0.1)
        dt = torch.float32 if precision == ajd.JD_FP32 else torch.float64
        g = torch.Generator(device="cuda").manual_seed(L)
        for call in range(2):  # two calls in a row share the static scratch
            b = torch.randn(h.n, device="cuda", dtype=torch.float64, generator=g).to(dt)
            want = P.apply(b, mixed=(precision == ajd.JD_MIXED))
            got = _noalloc(ajd, P, b, torch.empty_like(b), precision)
            torch.cuda.synchronize()
            w = want.double().cpu().numpy()
            x = got.double().cpu().numpy()
            tol = 1e-12 if precision != ajd.JD_FP32 else 1e-6
            assert np.abs(x - w).max() <= tol * np.abs(w).max(), (L, precision, call)
        P.close()


def test_noalloc_rejects_orders_beyond_the_limit(ajd):
    with ajd.Anderson(51, 16.5, 5) as h:  # 132651 rows > 131072
        P = ajd.Preconditioner.from_lattice(h, 0.0, n_dense=500)
        b = torch.zeros(h.n, device="cuda", dtype=torch.float64)
        with pytest.raises(ajd.JDError) as ei:
            _noalloc(ajd, P, b, torch.empty_like(b), ajd.JD_FP64)
        assert ei.value.code == ajd.JD_EINVAL
        assert "static scratch limit" in str(ei.value)
        P.close()
