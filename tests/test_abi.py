"""The C ABI library loads and exports every function the headers declare
(no GPU needed: only argument validation runs, no compute)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_math_0508111_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_core_api():
    names = declared_functions()
    for core in ["anderson_create", "anderson_destroy", "anderson_apply", "jd_last_error"]:
        assert core in names


def test_every_declared_symbol_is_exported(built_lib):
    missing = [n for n in declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_math_0508111_gb300 import _ffi
    bound = {s[0] for s in _ffi.SIGNATURES}
    assert set(declared_functions()) <= bound, set(declared_functions()) - bound


def test_argument_validation_without_gpu(built_lib):
    from paper_math_0508111_gb300 import _ffi
    L = _ffi.lib()
    h = ctypes.c_void_p()
    assert L.anderson_create(2, 16.5, 1, _ffi.JD_PERIODIC, ctypes.byref(h)) == _ffi.JD_EINVAL
    assert b"L >= 3" in L.jd_last_error()
    assert L.anderson_create(10, -1.0, 1, _ffi.JD_PERIODIC, ctypes.byref(h)) == _ffi.JD_EINVAL
    assert L.anderson_create(10, 1.0, 1, 7, ctypes.byref(h)) == _ffi.JD_EINVAL
    assert L.anderson_create(0, 1.0, 1, _ffi.JD_HARDWALL, ctypes.byref(h)) == _ffi.JD_EINVAL
    assert L.anderson_create(1300, 1.0, 1, _ffi.JD_HARDWALL, ctypes.byref(h)) == _ffi.JD_EINVAL
    assert L.anderson_destroy(None) == _ffi.JD_OK
    assert L.jd_version() >= 100


def test_batch_argument_validation_without_gpu(built_lib):
    """jd_solve_batch rejects bad arguments before touching a device."""
    from paper_math_0508111_gb300 import _ffi
    L = _ffi.lib()
    assert L.jd_solve_batch(None, 0, None, None, 1e-8, None, None, None, None, 0, None) == _ffi.JD_OK
    assert L.jd_solve_batch(None, 2, None, None, 1e-8, None, None, None, None, 0, None) == _ffi.JD_EINVAL
    assert L.jd_solve_batch(None, -1, None, None, 1e-8, None, None, None, None, 0, None) == _ffi.JD_EINVAL
    hs = (ctypes.c_void_p * 1)(None)
    sig = (ctypes.c_double * 1)(0.0)
    kk = (ctypes.c_int * 1)(1)
    ev = (ctypes.c_void_p * 1)(None)
    assert L.jd_solve_batch(hs, 1, sig, kk, 1e-8, None, ev, None, None, 0, None) == _ffi.JD_EINVAL
    assert b"problem 0" in L.jd_last_error()
