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


def test_server_argument_validation_without_gpu(built_lib):
    """The request loop rejects bad arguments before touching a device."""
    from paper_math_0508111_gb300 import _ffi
    L = _ffi.lib()
    p = _ffi.JdServerParams()
    assert L.jd_server_params_default(ctypes.byref(p)) == _ffi.JD_OK
    assert p.slots == 4 and p.setup_threads == 2 and p.hbm_budget == 0
    h = ctypes.c_void_p()
    p.slots = 100
    assert L.jd_server_create(ctypes.byref(p), ctypes.byref(h)) == _ffi.JD_EINVAL
    t = ctypes.c_uint64()
    assert L.jd_submit(None, 10, 16.5, 1, 0, 0.0, 5, 1e-8, 0, ctypes.byref(t)) == _ffi.JD_EINVAL
    assert L.jd_poll(None, 1, None, None, None, None) == _ffi.JD_EINVAL
    assert L.jd_server_destroy(None) == _ffi.JD_OK
    # the admission estimate grows with the lattice and covers the factor
    b = [ctypes.c_size_t() for _ in range(3)]
    for x, Lx in zip(b, [10, 50, 100]):
        assert L.jd_server_estimate(Lx, 5, ctypes.byref(x)) == _ffi.JD_OK
    assert b[0].value < b[1].value < b[2].value
    assert b[2].value > 56 * 56 * 10 ** 6  # three copies of ~57 entries per row at L = 100


def test_binding_struct_layout_matches_header(tmp_path):
    """Every parameter and statistics struct of the binding has the size and
    field offsets that a C compiler gives the header's struct (a C program
    built against include/ prints sizeof and offsetof)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_math_0508111_gb300 import _ffi
    structs = {"ildl_params": _ffi.IldlParams, "ildl_info_t": _ffi.IldlInfo, "jd_params": _ffi.JdParams,
               "jd_stats": _ffi.JdStats, "jd_server_params": _ffi.JdServerParams,
               "jd_server_info": _ffi.JdServerInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "anderson_jd.h"', "int main(void) {"]
    want = []
    for cname, py in structs.items():
        lines.append('  printf("%%zu\\n", sizeof(%s));' % cname)
        want.append(ctypes.sizeof(py))
        for field, _ in py._fields_:
            lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (cname, field))
            want.append(getattr(py, field).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == want


def test_default_gamma(built_lib):
    """gamma < 0 selects min(0.02, 5/sqrt(n)), and min(0.02, 1/sqrt(n)) for
    the off-diagonal model (Section 7): at L = 33 the two defaults are 0.02
    and 1/sqrt(35937); from L = 40 on the off-diagonal one is five times
    smaller."""
    from paper_math_0508111_gb300 import _ffi
    L = _ffi.lib()
    g = ctypes.c_double()
    for n, off, want in [(33 ** 3, 0, 0.02), (33 ** 3, 1, 1 / 35937 ** 0.5), (100 ** 3, 0, 0.005),
                         (100 ** 3, 1, 0.001), (50 ** 3, 1, 1 / 125000 ** 0.5), (10, 1, 0.02)]:
        assert L.ildl_default_gamma(n, off, ctypes.byref(g)) == _ffi.JD_OK
        assert abs(g.value - want) <= 1e-15 * want, (n, off, g.value)
    assert L.ildl_default_gamma(0, 0, ctypes.byref(g)) == _ffi.JD_EINVAL
    assert L.ildl_default_gamma(10, 0, None) == _ffi.JD_EINVAL
