"""ctypes declarations of the C ABI in ``include/anderson_jd.h``.

Loading fails loudly when the shared library has not been built: there is no
fallback implementation.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libanderson_jd.so")

c_int, c_double, c_void_p, c_int64, c_uint64 = (ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                                ctypes.c_int64, ctypes.c_uint64)
P = ctypes.POINTER

JD_OK, JD_EINVAL, JD_ENOMEM, JD_ENOCONV, JD_EBREAKDOWN, JD_EDEVICE, JD_ESETUP = 0, -1, -2, -3, -4, -5, -6
JD_EAGAIN = -7
JD_SUBMIT_VECTORS = 1
JD_PERIODIC, JD_HARDWALL = 0, 1
JD_FP64, JD_FP32, JD_MIXED = 0, 1, 2

ERROR_NAMES = {JD_EINVAL: "JD_EINVAL", JD_ENOMEM: "JD_ENOMEM", JD_ENOCONV: "JD_ENOCONV",
               JD_EBREAKDOWN: "JD_EBREAKDOWN", JD_EDEVICE: "JD_EDEVICE", JD_ESETUP: "JD_ESETUP",
               JD_EAGAIN: "JD_EAGAIN"}


class JDError(RuntimeError):
    def __init__(self, code, func, msg):
        super().__init__("%s failed with %s: %s" % (func, ERROR_NAMES.get(code, str(code)), msg))
        self.code = code


class IldlParams(ctypes.Structure):
    _fields_ = [("kappa", c_double), ("drop", c_double), ("gamma", c_double), ("max_levels", c_int),
                ("n_dense", c_int), ("matching", c_int), ("aggressive", c_double), ("setup_device", c_int),
                ("autotune", c_int), ("apply_form", c_int)]


class IldlInfo(ctypes.Structure):
    _fields_ = [("n", c_int), ("levels", c_int), ("n_dense", c_int), ("n_2x2", c_int), ("nnz_L", c_int64),
                ("nnz_A", c_int64), ("fill", c_double), ("setup_ms", c_double), ("match_ms", c_double),
                ("relaxed_levels", c_int), ("max_abs_L", c_double), ("aggressive_dropped", c_int64),
                ("apply_shift", c_int), ("apply_form", c_int)]


class JdParams(ctypes.Structure):
    _fields_ = [("jmin", c_int), ("jmax", c_int), ("max_outer", c_int), ("max_inner", c_int),
                ("inner_decay", c_double), ("inner_floor", c_double), ("switch_tol", c_double),
                ("precision", c_int), ("seed", c_uint64), ("extraction", c_int), ("guard", c_int), ("ildl", IldlParams),
                ("precond", c_void_p), ("gram", c_int)]


class JdStats(ctypes.Structure):
    _fields_ = [("nconv", c_int), ("outer_its", c_int), ("inner_its", c_int), ("restarts", c_int),
                ("setup_ms", c_double), ("solve_ms", c_double), ("max_residual", c_double),
                ("orth_error", c_double), ("ildl", IldlInfo), ("kernel_launches", c_int64),
                ("precond_calls", c_int), ("precond_ms", c_double), ("stencil_calls", c_int), ("stencil_ms", c_double),
                ("basis_orth_error", c_double)]


class JdServerParams(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("slots", c_int), ("setup_threads", c_int), ("solve", JdParams)]


class JdServerInfo(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("failed", c_int64), ("queued", c_int),
                ("building", c_int), ("ready", c_int), ("solving", c_int), ("peak_solving", c_int),
                ("hbm_budget", ctypes.c_size_t), ("reserved_bytes", ctypes.c_size_t),
                ("peak_reserved_bytes", ctypes.c_size_t)]


# (name, restype, argtypes) of every exported function
SIGNATURES = [
    ("jd_last_error", ctypes.c_char_p, []),
    ("jd_version", c_int, []),
    ("anderson_create", c_int, [c_int, c_double, c_uint64, c_int, P(c_void_p)]),
    ("anderson_create_from_potential", c_int, [c_int, c_void_p, c_int, P(c_void_p)]),
    ("anderson_create_offdiag", c_int, [c_int, c_double, c_double, c_uint64, c_int, P(c_void_p)]),
    ("anderson_bonds", c_int, [c_void_p, c_void_p]),
    ("anderson_destroy", c_int, [c_void_p]),
    ("anderson_size", c_int, [c_void_p, P(c_int64)]),
    ("anderson_potential", c_int, [c_void_p, c_void_p]),
    ("anderson_norm", c_int, [c_void_p, P(c_double)]),
    ("anderson_apply", c_int, [c_void_p, c_double, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    ("ildl_params_default", c_int, [P(IldlParams)]),
    ("ildl_default_gamma", c_int, [c_int64, c_int, P(c_double)]),
    ("ildl_setup_csr", c_int, [c_int, c_void_p, c_void_p, c_void_p, P(IldlParams), P(c_void_p)]),
    ("ildl_matching", c_int, [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("ildl_create", c_int, [c_void_p, c_double, P(IldlParams), P(c_void_p)]),
    ("ildl_info", c_int, [c_void_p, P(IldlInfo)]),
    ("ildl_export", c_int, [c_void_p] + [c_void_p] * 10),
    ("ildl_dataflow_schedule", c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p]),
    ("ildl_apply", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    ("ildl_apply_noalloc", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    ("ildl_destroy", c_int, [c_void_p]),
    ("jd_params_default", c_int, [P(JdParams)]),
    ("jd_solve", c_int, [c_void_p, c_double, c_int, c_double, P(JdParams), c_void_p, c_void_p, P(JdStats),
                         c_void_p]),
    ("jd_gram_bf16", c_int, [c_void_p, c_int64, c_int, c_void_p, c_int64, c_void_p, c_void_p]),
    ("jd_lanczos_solve", c_int, [c_void_p, c_double, c_int, c_double, P(JdParams), c_void_p, c_void_p, P(JdStats),
                                 c_void_p]),
    ("jd_server_params_default", c_int, [P(JdServerParams)]),
    ("jd_server_estimate", c_int, [c_int, c_int, P(ctypes.c_size_t)]),
    ("jd_server_create", c_int, [P(JdServerParams), P(c_void_p)]),
    ("jd_submit", c_int, [c_void_p, c_int, c_double, c_uint64, c_int, c_double, c_int, c_double, c_int,
                          P(c_uint64)]),
    ("jd_poll", c_int, [c_void_p, c_uint64, c_void_p, c_void_p, P(JdStats), P(c_double)]),
    ("jd_wait", c_int, [c_void_p, c_uint64, c_void_p, c_void_p, P(JdStats), P(c_double), c_double]),
    ("jd_server_info_get", c_int, [c_void_p, P(JdServerInfo)]),
    ("jd_server_destroy", c_int, [c_void_p]),
    ("jd_solve_batch", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double, P(JdParams), c_void_p, c_void_p,
                               c_void_p, c_int, c_void_p]),
]

_lib = None


def lib():
    """The loaded library (loaded on first use)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libanderson_jd.so is not built; run `python -m paper_math_0508111_gb300.build` "
                              "(or __graft_entry__.build()).  There is no non-CUDA fallback.")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code, func):
    if code != JD_OK:
        msg = lib().jd_last_error().decode(errors="replace")
        raise JDError(code, func, msg)
    return code


def call(name, *args):
    return check(getattr(lib(), name)(*args), name)
