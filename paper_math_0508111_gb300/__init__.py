"""GB300 Jacobi–Davidson eigensolver for the 3D Anderson model of localization.

Python binding of the C ABI declared in ``include/anderson_jd.h``.  The
binding only marshals arguments: every step of the computation runs in the
library's CUDA kernels (and its native host setup code).  PyTorch supplies
device memory and streams; tensors passed in must live on the CUDA device
that was current when the handle was created.
"""
import ctypes

import numpy as np

from . import _ffi
from ._ffi import (JD_EAGAIN, JD_EBREAKDOWN, JD_EDEVICE, JD_EINVAL, JD_ENOCONV, JD_ENOMEM, JD_ESETUP, JD_FP32,
                   JD_FP64, JD_HARDWALL, JD_MIXED, JD_OK, JD_PERIODIC, JD_SUBMIT_VECTORS, JDError)

__all__ = ["Anderson", "Preconditioner", "Server", "ildl_params", "jd_params", "solve", "solve_batch", "JDError",
           "JD_PERIODIC", "JD_HARDWALL", "JD_FP64", "JD_FP32", "JD_MIXED", "library_path"]


def library_path():
    return _ffi.LIB_PATH


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _precision_of(t):
    import torch
    if t.dtype == torch.float64:
        return JD_FP64
    if t.dtype == torch.float32:
        return JD_FP32
    raise TypeError("only float64 and float32 tensors are supported, got %s" % t.dtype)


def _dev_ptr(t, what):
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    return ctypes.c_void_p(t.data_ptr())


class Anderson:
    """An L^3 Anderson lattice (Eq. (1)) with box disorder of width W.

    The potential is generated on the current CUDA device from ``seed``, or
    copied from ``potential`` (host array of L**3 energies) when given.
    """

    def __init__(self, L, W, seed, bc=JD_PERIODIC, potential=None):
        h = ctypes.c_void_p()
        if potential is None:
            _ffi.call("anderson_create", int(L), float(W), ctypes.c_uint64(int(seed) & (2 ** 64 - 1)), int(bc),
                      ctypes.byref(h))
        else:
            eps = np.ascontiguousarray(potential, dtype=np.float64)
            if eps.shape != (int(L) ** 3,):
                raise ValueError("potential must have L**3 entries")
            _ffi.call("anderson_create_from_potential", int(L), eps.ctypes.data_as(ctypes.c_void_p), int(bc),
                      ctypes.byref(h))
        self._h = h
        self.L, self.W, self.seed, self.bc = int(L), float(W), int(seed), int(bc)
        n = ctypes.c_int64()
        _ffi.call("anderson_size", self._h, ctypes.byref(n))
        self.n = n.value

    @classmethod
    def offdiag(cls, L, seed, diag=1.28, width=1.0, bc=JD_PERIODIC):
        """The off-diagonal Anderson model of Section 7 (anderson_create_offdiag):
        constant diagonal ``diag``, bond hoppings uniform on
        [-width/2, width/2)."""
        self = cls.__new__(cls)
        h = ctypes.c_void_p()
        _ffi.call("anderson_create_offdiag", int(L), float(diag), float(width),
                  ctypes.c_uint64(int(seed) & (2 ** 64 - 1)), int(bc), ctypes.byref(h))
        self._h = h
        self.L, self.W, self.seed, self.bc = int(L), float(width), int(seed), int(bc)
        n = ctypes.c_int64()
        _ffi.call("anderson_size", self._h, ctypes.byref(n))
        self.n = n.value
        return self

    def bonds(self):
        """Hoppings t[s, d] of an off-diagonal lattice, shape (n, 3)."""
        out = np.empty(3 * self.n, dtype=np.float64)
        _ffi.call("anderson_bonds", self.handle, out.ctypes.data_as(ctypes.c_void_p))
        return out.reshape(self.n, 3)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("handle is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _ffi.lib().anderson_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def norm(self):
        v = ctypes.c_double()
        _ffi.call("anderson_norm", self.handle, ctypes.byref(v))
        return v.value

    def potential(self):
        out = np.empty(self.n, dtype=np.float64)
        _ffi.call("anderson_potential", self.handle, out.ctypes.data_as(ctypes.c_void_p))
        return out

    def apply(self, x, shift=0.0, out=None, stream=None):
        """y = (A - shift I) x.  ``x`` is a CUDA tensor of shape (n,) or
        (m, n) (m vectors, one per row, i.e. an n x m column-major block),
        float64 or float32."""
        import torch
        if x.shape[-1] != self.n:
            raise ValueError("last dimension must be n = %d" % self.n)
        m = 1 if x.dim() == 1 else x.shape[0]
        if out is None:
            out = torch.empty_like(x)
        prec = _precision_of(x)
        if out.dtype != x.dtype or out.shape != x.shape:
            raise ValueError("out must match x in dtype and shape")
        _ffi.call("anderson_apply", self.handle, float(shift), _dev_ptr(x, "x"), _dev_ptr(out, "out"), int(m),
                  prec, _stream_handle(stream))
        return out


def ildl_params(**kw):
    """Preconditioner parameters (defaults of ildl_params_default) with
    keyword overrides: kappa, drop, gamma, max_levels, n_dense, matching,
    aggressive (tau of the aggressive dropping of Section 6.3; 0 = off)."""
    p = _ffi.IldlParams()
    _ffi.call("ildl_params_default", ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError("unknown preconditioner parameter %r" % k)
        setattr(p, k, v)
    return p


def matching(indptr, indices, data):
    """Sections 5.1-5.2 on a symmetric CSR matrix (host): returns
    (match_col, scale, partner) as numpy arrays."""
    indptr = np.ascontiguousarray(indptr, dtype=np.int64)
    indices = np.ascontiguousarray(indices, dtype=np.int32)
    data = np.ascontiguousarray(data, dtype=np.float64)
    n = len(indptr) - 1
    mc = np.empty(n, np.int32)
    sc = np.empty(n)
    pt = np.empty(n, np.int32)
    vp = ctypes.c_void_p
    _ffi.call("ildl_matching", int(n), indptr.ctypes.data_as(vp), indices.ctypes.data_as(vp),
              data.ctypes.data_as(vp), mc.ctypes.data_as(vp), sc.ctypes.data_as(vp), pt.ctypes.data_as(vp))
    return mc, sc, pt


class Preconditioner:
    """Multilevel incomplete LDL^T K ~ A - sigma I (Sections 5-6).

    ``Preconditioner.from_lattice(h, sigma)`` builds it for a lattice and
    uploads it to the device; ``Preconditioner.from_csr(...)`` builds the
    host factor of any symmetric CSR matrix (no GPU needed)."""

    def __init__(self, handle):
        self._h = handle

    @classmethod
    def from_lattice(cls, lattice, sigma, **params):
        h = ctypes.c_void_p()
        p = ildl_params(**params)
        _ffi.call("ildl_create", lattice.handle, float(sigma), ctypes.byref(p), ctypes.byref(h))
        return cls(h)

    @classmethod
    def from_csr(cls, indptr, indices, data, **params):
        indptr = np.ascontiguousarray(indptr, dtype=np.int64)
        indices = np.ascontiguousarray(indices, dtype=np.int32)
        data = np.ascontiguousarray(data, dtype=np.float64)
        n = len(indptr) - 1
        h = ctypes.c_void_p()
        p = ildl_params(**params)
        _ffi.call("ildl_setup_csr", int(n), indptr.ctypes.data_as(ctypes.c_void_p),
                  indices.ctypes.data_as(ctypes.c_void_p), data.ctypes.data_as(ctypes.c_void_p),
                  ctypes.byref(p), ctypes.byref(h))
        return cls(h)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("handle is closed")
        return self._h

    def info(self):
        i = _ffi.IldlInfo()
        _ffi.call("ildl_info", self.handle, ctypes.byref(i))
        return {f: getattr(i, f) for f, _ in i._fields_}

    def export(self):
        """The factor as numpy arrays (see ildl_export in the header)."""
        inf = self.info()
        n, nl, nd, nnz = inf["n"], inf["levels"], inf["n_dense"], inf["nnz_L"]
        out = dict(perm=np.empty(n, np.int32), scale=np.empty(n), level_ptr=np.empty(nl + 2, np.int32),
                   Lptr=np.empty(n + 1, np.int64), Lcol=np.empty(max(nnz, 1), np.int32),
                   Lval=np.empty(max(nnz, 1)), dinv_d=np.empty(n), dinv_o=np.empty(n),
                   partner=np.empty(n, np.int32), dense_inv=np.empty(max(nd * nd, 1)))
        ptrs = [out[k].ctypes.data_as(ctypes.c_void_p) for k in
                ["perm", "scale", "level_ptr", "Lptr", "Lcol", "Lval", "dinv_d", "dinv_o", "partner", "dense_inv"]]
        _ffi.call("ildl_export", self.handle, *ptrs)
        out["Lcol"], out["Lval"] = out["Lcol"][:nnz], out["Lval"][:nnz]
        out["dense_inv"] = out["dense_inv"][:nd * nd].reshape(nd, nd)
        out.update(inf)
        return out

    def apply(self, b, out=None, stream=None, mixed=False):
        """x = K^{-1} b for a CUDA tensor b (float64 or float32, length n).
        ``mixed=True`` (float64 b) applies the binary32 factor with
        float-float (about 48-bit) work vectors and sums."""
        import torch
        if out is None:
            out = torch.empty_like(b)
        prec = _precision_of(b)
        if mixed:
            if prec != JD_FP64:
                raise TypeError("mixed apply takes float64 vectors")
            prec = JD_MIXED
        _ffi.call("ildl_apply", self.handle, _dev_ptr(b, "b"), _dev_ptr(out, "out"), prec, _stream_handle(stream))
        return out

    def close(self):
        if getattr(self, "_h", None) is not None:
            _ffi.lib().ildl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def jd_params(precision=JD_FP64, precond=None, ildl=None, **kw):
    """Solver parameters: defaults of jd_params_default with keyword
    overrides (jmin, jmax, max_outer, max_inner, inner_decay, inner_floor,
    switch_tol, seed); ``ildl`` is a dict of preconditioner overrides and
    ``precond`` an optional prebuilt :class:`Preconditioner`."""
    p = _ffi.JdParams()
    _ffi.call("jd_params_default", ctypes.byref(p))
    p.precision = int(precision)
    for k, v in kw.items():
        if not hasattr(p, k) or k in ("ildl", "precond", "precision"):
            raise TypeError("unknown solver parameter %r" % k)
        setattr(p, k, v)
    if ildl:
        for k, v in ildl.items():
            setattr(p.ildl, k, v)
    if precond is not None:
        p.precond = precond.handle
    return p


def _stats_dict(st):
    d = {f: getattr(st, f) for f, _ in st._fields_ if f != "ildl"}
    d["ildl"] = {f: getattr(st.ildl, f) for f, _ in st.ildl._fields_}
    return d


def solve(lattice, sigma, k, tol, precision=JD_FP64, vectors=True, stream=None, raise_on_noconv=True,
          method="jd", **params):
    """The k eigenpairs of the lattice's matrix nearest sigma: by
    Jacobi-Davidson (jd_solve, ``method="jd"``) or by shift-and-invert
    Lanczos over the same preconditioned SQMR (jd_lanczos_solve,
    ``method="lanczos"``).

    Returns (evals, evecs, stats): evals has shape (k,), evecs shape (n, k)
    (numpy, host), stats a dict of the solver counters.  Extra keyword
    arguments go to :func:`jd_params`."""
    p = jd_params(precision=precision, **params)
    ev = np.zeros(int(k))
    X = np.zeros((int(k), lattice.n)) if vectors else None
    st = _ffi.JdStats()
    vp = ctypes.c_void_p
    fn = {"jd": "jd_solve", "lanczos": "jd_lanczos_solve"}[method]
    rc = getattr(_ffi.lib(), fn)(lattice.handle, float(sigma), int(k), float(tol), ctypes.byref(p),
                             ev.ctypes.data_as(vp), X.ctypes.data_as(vp) if vectors else None, ctypes.byref(st),
                             _stream_handle(stream) if stream is not None else None)
    if rc != JD_OK and (rc != JD_ENOCONV or raise_on_noconv):
        _ffi.check(rc, fn)
    stats = _stats_dict(st)
    stats["status"] = rc
    return ev, (X.T if vectors else None), stats


def solve_batch(lattices, sigmas, ks, tol, precision=JD_FP64, vectors=True, setup_threads=2, stream=None,
                raise_on_noconv=True, **params):
    """Independent problems through jd_solve_batch: later problems'
    preconditioners are built on host threads while earlier ones solve.

    ``sigmas`` and ``ks`` are scalars or one entry per lattice.  Returns a
    list of (evals, evecs, stats) like :func:`solve`."""
    m = len(lattices)
    sig = np.broadcast_to(np.asarray(sigmas, dtype=np.float64), (m,)).copy()
    kk = np.broadcast_to(np.asarray(ks, dtype=np.int32), (m,)).copy()
    p = jd_params(precision=precision, **params)
    evs = [np.zeros(int(kk[i])) for i in range(m)]
    Xs = [np.zeros((int(kk[i]), lat.n)) for i, lat in enumerate(lattices)] if vectors else None
    vp = ctypes.c_void_p
    hs = (vp * max(m, 1))(*[lat.handle for lat in lattices])
    ep = (vp * max(m, 1))(*[e.ctypes.data for e in evs])
    xp = (vp * max(m, 1))(*[x.ctypes.data for x in Xs]) if vectors else None
    sts = (_ffi.JdStats * max(m, 1))()
    rc = _ffi.lib().jd_solve_batch(hs, m, sig.ctypes.data_as(vp), kk.ctypes.data_as(vp), float(tol),
                                   ctypes.byref(p), ep, xp, sts, int(setup_threads),
                                   _stream_handle(stream) if stream is not None else None)
    if rc != JD_OK and (rc != JD_ENOCONV or raise_on_noconv):
        _ffi.check(rc, "jd_solve_batch")
    out = []
    for i in range(m):
        stats = _stats_dict(sts[i])
        stats["status"] = JD_OK if stats["nconv"] >= kk[i] else JD_ENOCONV
        out.append((evs[i], (Xs[i].T if vectors else None), stats))
    return out


class Server:
    """The request loop of ``jd_server_*``: submit eigensolves of any size,
    poll or wait for each result.  ``slots`` solves run concurrently on
    their own CUDA streams, ``setup_threads`` host threads build the
    preconditioners, and requests are admitted while their estimated device
    memory fits ``hbm_budget`` bytes (0: 80% of the free memory).  Keyword
    arguments other than these go to :func:`jd_params` (for every solve)."""

    def __init__(self, hbm_budget=0, slots=4, setup_threads=2, precision=JD_FP64, **params):
        p = _ffi.JdServerParams()
        _ffi.call("jd_server_params_default", ctypes.byref(p))
        p.hbm_budget = int(hbm_budget)
        p.slots = int(slots)
        p.setup_threads = int(setup_threads)
        p.solve = jd_params(precision=precision, **params)
        h = ctypes.c_void_p()
        _ffi.call("jd_server_create", ctypes.byref(p), ctypes.byref(h))
        self._h = h
        self._meta = {}

    @staticmethod
    def estimate(L, k):
        b = ctypes.c_size_t()
        _ffi.call("jd_server_estimate", int(L), int(k), ctypes.byref(b))
        return b.value

    def submit(self, L, W, seed, sigma, k, tol, bc=JD_PERIODIC, vectors=False):
        t = ctypes.c_uint64()
        _ffi.call("jd_submit", self._h, int(L), float(W), int(seed), int(bc), float(sigma), int(k), float(tol),
                  JD_SUBMIT_VECTORS if vectors else 0, ctypes.byref(t))
        self._meta[t.value] = (int(L) ** 3, int(k), bool(vectors))
        return t.value

    def _result(self, fn, ticket, *extra, raise_on_error=True):
        n, k, vec = self._meta[ticket]
        ev = np.zeros(k)
        X = np.zeros((k, n)) if vec else None
        st = _ffi.JdStats()
        lat = ctypes.c_double()
        vp = ctypes.c_void_p
        rc = getattr(_ffi.lib(), fn)(self._h, ticket, ev.ctypes.data_as(vp), X.ctypes.data_as(vp) if vec else None,
                                     ctypes.byref(st), ctypes.byref(lat), *extra)
        if rc == JD_EAGAIN:
            return None
        del self._meta[ticket]
        if rc != JD_OK and (rc != JD_ENOCONV or raise_on_error):
            _ffi.check(rc, fn)
        stats = _stats_dict(st)
        stats["status"] = rc
        stats["latency_ms"] = lat.value
        return ev, (X.T if vec else None), stats

    def poll(self, ticket, raise_on_error=True):
        """(evals, evecs or None, stats) once done, else None."""
        return self._result("jd_poll", ticket, raise_on_error=raise_on_error)

    def wait(self, ticket, timeout=-1.0, raise_on_error=True):
        return self._result("jd_wait", ticket, ctypes.c_double(timeout), raise_on_error=raise_on_error)

    def info(self):
        i = _ffi.JdServerInfo()
        _ffi.call("jd_server_info_get", self._h, ctypes.byref(i))
        return {f: getattr(i, f) for f, _ in i._fields_}

    def close(self):
        if self._h is not None:
            _ffi.lib().jd_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
