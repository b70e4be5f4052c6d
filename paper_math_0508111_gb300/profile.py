"""Small, repeatable workloads for timing and profiling single kernels.

    python -m paper_math_0508111_gb300.profile apply   [--L 70] [--reps 5] [--only fp32|fp64|mixed]
    python -m paper_math_0508111_gb300.profile stencil [--L 256] [--reps 20] [--vectors 1]
    python -m paper_math_0508111_gb300.profile setup   [--L 100] [--threads 16,8] [--schur gpu,host]
    python -m paper_math_0508111_gb300.profile gram    [--n 1000000] [--cols 40] [--reps 10]

``apply`` builds the preconditioner of A - 0 I for an L^3 lattice (W = 16.5,
seed 1) and times its application in binary32, binary64 and the mixed form
(binary32 factor values, float-float work vectors and sums): 3 warm-up
applications each, then ``reps`` timed ones, CUDA events on the current
stream.  ``stencil`` times y = A x in binary64
and binary32 with the L2 flushed before every repetition.  Both print one
JSON line per case.  Run them under ncu with ``-k regex:persistent`` or
``-k regex:stencil`` to capture the kernel of interest.  ``setup`` times the
whole construction of the preconditioner of A - 0 I for an L^3 lattice
(host setup, dense-tail inversion on the device, upload) once per host
thread count and per place of the levels' Schur complements (GPU or host
threads), with the OpenMP thread count set through libgomp.
"""
import argparse
import json

import torch

import paper_math_0508111_gb300 as ajd


def _time(fn, reps, flush=None):
    s = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ts.sort()
    return ts[len(ts) // 2]


def apply_case(L, reps, only=None, forms=(-1,)):
    """The apply of the L-lattice's factor (sigma = 0), per apply form
    (-1: the autotuner's choice; 0: level counters; 1: dataflow)."""
    h = ajd.Anderson(L, 16.5, 1)
    for form in forms:
        P = ajd.Preconditioner.from_lattice(h, 0.0, apply_form=form)
        info = P.info()
        print(json.dumps({"case": "setup", "L": L, "form_requested": form, **info}), flush=True)
        for name, dt, mixed in [("fp32", torch.float32, False), ("fp64", torch.float64, False),
                                ("mixed", torch.float64, True)]:
            if only and name != only:
                continue
            b = torch.randn(h.n, device="cuda", dtype=dt)
            x = torch.empty_like(b)
            for _ in range(3):
                P.apply(b, out=x, mixed=mixed)
            ms = _time(lambda: P.apply(b, out=x, mixed=mixed), reps)
            print(json.dumps({"case": "apply", "precision": name, "L": L, "form": info["apply_form"],
                              "shift": info["apply_shift"], "ms": ms}), flush=True)
        P.close()


def stencil_case(L, reps, m=1):
    h = ajd.Anderson(L, 16.5, 1)
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda", dtype=torch.float32)
    for name, dt, nbytes in [("fp64", torch.float64, 24), ("fp32", torch.float32, 12)]:
        # m vectors in one launch (a block of m columns) amortise the launch
        # and event overhead of a ~40 us kernel; the potential is read once
        # per vector in the byte count (an upper bound on the reuse)
        x = torch.randn((m, h.n) if m > 1 else (h.n,), device="cuda", dtype=dt)
        y = torch.empty_like(x)
        for _ in range(3):
            h.apply(x, out=y)
        ms = _time(lambda: h.apply(x, out=y), reps, flush)
        print(json.dumps({"case": "stencil", "precision": name, "L": L, "vectors": m, "ms": ms,
                          "GBps": nbytes * h.n * m / (ms * 1e-3) / 1e9}), flush=True)


def gram_case(n, c, reps):
    """The BF16 tensor-core projection (jd_gram_bf16: conversion of the
    columns to BF16, the tcgen05 kernel, the cross-CTA sum) on n x c
    columns; CUDA events around the whole call."""
    import ctypes
    X = torch.randn((c, n), device="cuda", dtype=torch.float64)
    t = torch.randn(n, device="cuda", dtype=torch.float64)
    out = torch.empty(c, device="cuda", dtype=torch.float64)
    vp = ctypes.c_void_p

    def call():
        ajd._ffi.call("jd_gram_bf16", vp(X.data_ptr()), n, c, vp(t.data_ptr()), n, vp(out.data_ptr()),
                      vp(torch.cuda.current_stream().cuda_stream))
    for _ in range(3):
        call()
    ms = _time(call, reps)
    print(json.dumps({"case": "gram_bf16", "n": n, "columns": c, "ms": ms,
                      "bf16_GBps": 2 * n * c / (ms * 1e-3) / 1e9}), flush=True)


def setup_case(L, threads, where):
    import ctypes
    import ctypes.util
    import time
    gomp = ctypes.CDLL(ctypes.util.find_library("gomp") or "libgomp.so.1")
    with ajd.Anderson(L, 16.5, 1) as h:
        for t in threads:
            for dev in where:
                gomp.omp_set_num_threads(int(t))
                t0 = time.perf_counter()
                P = ajd.Preconditioner.from_lattice(h, 0.0, setup_device=dev)
                wall = time.perf_counter() - t0
                inf = P.info()
                print(json.dumps({"case": "setup", "L": L, "threads": int(t),
                                  "schur": {0: "host", 1: "gpu"}[dev], "wall_s": wall,
                                  "setup_ms": inf["setup_ms"], "match_ms": inf["match_ms"], "levels": inf["levels"],
                                  "nnz_L": inf["nnz_L"]}), flush=True)
                P.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["apply", "stencil", "setup", "gram"])
    ap.add_argument("--n", type=int, default=1000000, help="gram: rows")
    ap.add_argument("--cols", type=int, default=40, help="gram: columns")
    ap.add_argument("--L", type=int, default=None)
    ap.add_argument("--reps", type=int, default=None)
    ap.add_argument("--only", choices=["fp32", "fp64", "mixed"], default=None)
    ap.add_argument("--forms", default="-1", help="apply: apply forms, comma separated (-1 = autotuned)")
    ap.add_argument("--vectors", type=int, default=1, help="stencil: vectors per launch")
    ap.add_argument("--threads", default="16,8", help="setup: host thread counts, comma separated")
    ap.add_argument("--schur", default="gpu,host", help="setup: where the Schur complements are formed")
    a = ap.parse_args()
    if a.what == "apply":
        apply_case(a.L or 70, a.reps or 5, a.only, [int(x) for x in a.forms.split(",")])
    elif a.what == "gram":
        gram_case(a.n, a.cols, a.reps or 10)
    elif a.what == "setup":
        setup_case(a.L or 100, [int(t) for t in a.threads.split(",")],
                   [{"host": 0, "gpu": 1}[w] for w in a.schur.split(",")])
    else:
        stencil_case(a.L or 256, a.reps or 20, a.vectors)


if __name__ == "__main__":
    main()
