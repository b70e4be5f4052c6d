"""GPU parity of the disorder generator and the stencil against the oracle."""
import numpy as np
import pytest

import workloads
from oracle import lattice, rng

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ajd():
    import paper_math_0508111_gb300 as ajd
    assert torch.cuda.is_available()
    return ajd


@pytest.mark.parametrize("L,W,seed,bc", [(3, 16.5, 1, 0), (10, 16.5, 1, 0), (33, 12.0, 7, 0),
                                         (1, 5.0, 3, 1), (2, 5.0, 3, 1), (37, 21.0, 2**63 + 5, 1),
                                         (100, 16.5, 1, 0)])
def test_potential_bit_exact(ajd, L, W, seed, bc):
    with ajd.Anderson(L, W, seed, bc) as h:
        got = h.potential()
        want = rng.potential(L, W, seed)
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
        assert h.norm() == lattice.norm_bound(want)


def test_zero_disorder(ajd):
    with ajd.Anderson(8, 0.0, 5) as h:
        assert np.all(h.potential() == 0.0)
        assert h.norm() == 6.0


def _check_stencil(ajd, L, W, seed, bc, shift, m, dtype):
    with ajd.Anderson(L, W, seed, bc) as h:
        n = L ** 3
        X = workloads.random_block(n, m, seed=100 + L)
        x = torch.tensor(X, device="cuda", dtype=dtype)
        y = h.apply(x if m > 1 else x[0].contiguous(), shift=shift)
        torch.cuda.synchronize()
        eps = rng.potential(L, W, seed)
        want = lattice.matvec(L, eps, X.T, bc=bc, shift=shift).T
        got = y.double().cpu().numpy().reshape(m, n)
        scale = (lattice.norm_bound(eps) + abs(shift)) * np.abs(X).max()
        tol = 1e-14 if dtype == torch.float64 else 2e-6
        err = np.abs(got - want).max() / scale
        assert err <= tol, (L, bc, err)


@pytest.mark.parametrize("L,bc", [(3, 0), (4, 0), (5, 1), (10, 0), (10, 1), (33, 0), (37, 1), (64, 0),
                                  # L >= 16 with 16-byte rows runs the plane-tile kernel: tiles past L
                                  # (L % 8 != 0), hard walls, several x-segments per row (L > 128 binary32,
                                  # > 64 binary64); L = 8, 12 exercise the row-marching kernel
                                  (8, 0), (12, 1), (20, 1), (24, 0), (132, 1), (136, 0)])
@pytest.mark.parametrize("dtype_name", ["float64", "float32"])
def test_stencil_matches_oracle(ajd, L, bc, dtype_name):
    _check_stencil(ajd, L, 16.5, 3, bc, 0.37, 1, getattr(torch, dtype_name))


@pytest.mark.parametrize("dtype_name", ["float64", "float32"])
def test_stencil_block_and_edge_sizes(ajd, dtype_name):
    dt = getattr(torch, dtype_name)
    _check_stencil(ajd, 1, 16.5, 3, 1, 0.0, 2, dt)  # single site, no neighbours
    _check_stencil(ajd, 2, 16.5, 3, 1, -1.0, 3, dt)
    _check_stencil(ajd, 21, 12.0, 4, 0, 1.5, 4, dt)
    _check_stencil(ajd, 12, 12.0, 4, 1, 0.7, 3, dt)  # several vectors on the plane-tile kernel
    _check_stencil(ajd, 16, 12.0, 5, 0, -0.3, 2, dt)


def test_stencil_full_size_L100(ajd):
    """The headline lattice (L = 100, n = 10^6), in both precisions."""
    _check_stencil(ajd, 100, 16.5, 1, 0, 0.0, 1, torch.float64)
    _check_stencil(ajd, 100, 16.5, 1, 0, 0.0, 1, torch.float32)


def test_stencil_rejects_bad_args(ajd):
    with ajd.Anderson(5, 1.0, 1) as h:
        x = torch.zeros(h.n, device="cuda", dtype=torch.float16)
        with pytest.raises(TypeError):
            h.apply(x)
        with pytest.raises(ajd.JDError):
            from paper_math_0508111_gb300 import _ffi
            import ctypes
            _ffi.call("anderson_apply", h.handle, 0.0, ctypes.c_void_p(0), ctypes.c_void_p(0), 1, 0, None)
