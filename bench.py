#!/usr/bin/env python3
"""Benchmark of the GPU Jacobi–Davidson solver for the 3D Anderson model.

Metric: converged eigenpairs per second (residual <= 1e-8 ||A||) on the
L = 100, W = 16.5 periodic lattice, k = 5 eigenpairs nearest sigma = 0 (the
configuration of Table 4's headline row M = 100, w = 16.5).  One step is one
disorder realisation solved completely: preconditioner construction
(matching, ordering, multilevel ILDL^T and its upload) plus the
Jacobi–Davidson iteration, with the potential already resident on the
device.  The headline (batched) form runs the K timed realisations through
one ``jd_solve_batch``: host threads build the preconditioners of later
realisations while the GPU solves earlier ones, with the mixed inner solve
(binary32 preconditioner inside binary64 vectors and outer iteration).  The
plain form -- one binary64 ``jd_solve`` after another -- is timed on the same
realisations for comparison.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run; every rank solves its own
realisations (independent problems, no collective on the data path) and the
JSON line reports the whole-job rate (weak scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "eigenpairs/s at resid≤1e-8, L=100 W=16.5; batched/served vs plain FP64; p99"
UNIT = "eigenpairs/s"
PAPER_EIGENPAIRS_PER_S = 5.0 / 978.0  # Table 4, M = 100, w = 16.5, one Itanium2 core
# Table 6 (M = 100, five eigenvalues nearest 0): periodic 980 s, hard wall
# 969 s, off-diagonal ("inverse") problem 2075 s
PAPER_TABLE6_S = {("diagonal", "periodic"): 980.0, ("diagonal", "hardwall"): 969.0, ("offdiag", "periodic"): 2075.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=100)
    ap.add_argument("--W", type=float, default=16.5)
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--sigma", type=float, default=0.0)
    ap.add_argument("--model", default="diagonal", choices=["diagonal", "offdiag"],
                    help="diagonal disorder of Eq. (1), or the off-diagonal model of Section 7 (diagonal 1.28, "
                         "hoppings uniform on [-1/2, 1/2])")
    ap.add_argument("--bc", default="periodic", choices=["periodic", "hardwall"])
    ap.add_argument("--method", default="jd", choices=["jd", "lanczos"],
                    help="jd: pipelined jd_solve_batch; lanczos: shift-and-invert Lanczos (jd_lanczos_solve), "
                         "one realisation after another")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32", "fp64"],
                    help="inner-solve precision of the headline form")
    ap.add_argument("--no-fp64", action="store_true", help="skip the binary64 comparison arms")
    ap.add_argument("--fp64-steps", type=int, default=8,
                    help="realisations of the binary64 comparison arms (the first of the timed ones)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--workload", default="headline", choices=["headline", "batch"],
                    help="headline: the L = 100 realisations; batch: the 256-problem batch through jd_server")
    ap.add_argument("--batch-problems", type=int, default=256)
    ap.add_argument("--batch-sample", type=int, default=32,
                    help="problems of the bounded batch sample reported beside the headline (0 skips it)")
    ap.add_argument("--serve-requests", type=int, default=8,
                    help="requests per arrival rate of the serving sweep (0 skips it)")
    ap.add_argument("--serve-max-outer", type=int, default=400,
                    help="Jacobi-Davidson outer steps per served request before it returns its converged prefix "
                         "(bounds the sample's run time; the weak-disorder requests of the stream converge slowly)")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[0.5, 1.0, 2.0],
                    help="arrival rates of the serving sweep, as multiples of the measured capacity")
    ap.add_argument("--serve-budget-s", type=float, default=240.0,
                    help="no further rate of the serving sweep is started once the sweep has run this long")
    ap.add_argument("--serve-lmax", type=int, default=120, help="largest lattice of the serving stream")
    ap.add_argument("--cpu-L", type=int, default=30, help="lattice of the CPU oracle baseline sample")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-setup-threads", type=int, default=3)
    ap.add_argument("--setup-threads", type=int, default=4,
                    help="concurrent preconditioner builds in the pipelined batch")
    ap.add_argument("--n-dense", type=int, default=0,
                    help="rows of the preconditioner's dense tail (0: the library's default)")
    return ap.parse_args()


_T0 = time.perf_counter()


def progress(msg):
    """One line on stderr per stage (wall time since start), so a slow stage
    shows in the log even when the run is cut short."""
    sys.stderr.write("[bench %7.1f s] %s\n" % (time.perf_counter() - _T0, msg))
    sys.stderr.flush()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def apply_bytes(info, val, vec):
    """Algorithmic bytes of one preconditioner application x = K^{-1} b with
    `val`-byte factor values and `vec`-byte vectors: every stored entry of L
    read once in the forward and once in the backward sweep (value + int32
    column), both row-pointer arrays, and per position the gather/scatter
    data (perm twice, scale twice, b, out), the work vectors w and z
    (written once, read once), the 2x2 pivot data (diagonal, off-diagonal,
    partner) and the dense trailing inverse.  Gathers of earlier solution
    entries through the column indices are cache traffic and not counted."""
    n, nnz, nd = info["n"], info["nnz_L"], info["n_dense"]
    idx = 4
    return (2 * nnz * (val + idx) + 2 * (n + 1) * idx
            + n * (2 * idx + 2 * val + 2 * vec)       # perm x2, scale x2, b, out
            + n * (4 * vec)                           # w write/read, z write/read
            + (n - nd) * (2 * val + idx)              # D^{-1} diagonal, off-diagonal, partner
            + nd * nd * val)


APPLY_SOURCES = {0: ["ildl_apply_kernel.cuh"], 1: ["ildl_apply_kernel.cuh", "ildl_apply_dataflow.cuh"]}
APPLY_KERNELS = {0: "ildl_apply_persistent_kernel (one cooperative launch; level sweeps with per-level completion "
                    "counters: gather, forward levels, dense tail, backward levels)",
                 1: "ildl_apply_dataflow_kernel (one cooperative launch; every row starts once the entries it "
                    "reads are written: gather, forward levels, dense tail, backward levels)"}


def kernel_source_hash(files):
    """SHA-1 of the apply kernel's sources (csrc/<files>, concatenated):
    DRAM counters recorded for an older source no longer describe the kernel
    that runs."""
    import hashlib
    h = hashlib.sha1()
    for name in files:
        with open(os.path.join(ROOT, "paper_math_0508111_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(precision, info, form):
    """DRAM bytes per apply from the committed ncu summary of the apply form
    in use (profiles/ildl_apply_<precision>_traffic.json for the level-counter
    kernel, profiles/ildl_apply_dataflow_<precision>_traffic.json for the
    dataflow kernel), scaled from the captured lattice to this factor by the
    ratio of algorithmic bytes; None when no capture exists or the kernel
    source changed since it was taken."""
    name = "ildl_apply_%s_traffic.json" % precision if form == 0 else "ildl_apply_dataflow_%s_traffic.json" % precision
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            d = json.load(f)
    except Exception:
        return None
    files = d.get("source_files") or [os.path.basename(d.get("source_file", ""))]
    if files != APPLY_SOURCES[form] or d.get("source_sha1") != kernel_source_hash(files):
        return None
    return d["dram_bytes_per_apply"] * apply_bytes(info, *d["val_vec_bytes"]) / d["algorithmic_bytes_per_apply"]


def run_requests(ajd, args, precision, reqs, slots, setup_threads):
    """Submit each request to a jd_server at its arrival time ("t", seconds
    from the start) and poll until all are done.  Returns eigenpairs/s over
    the whole run and the latency percentiles (submission to completion)."""
    lat, pairs, failed, per = [], 0, 0, []
    with ajd.Server(slots=slots, setup_threads=setup_threads, precision=precision,
                    max_outer=args.serve_max_outer) as srv:
        start = time.perf_counter()
        pending, i = {}, 0
        while i < len(reqs) or pending:
            now = time.perf_counter() - start
            while i < len(reqs) and reqs[i]["t"] <= now:
                r = reqs[i]
                pending[srv.submit(r["L"], r["W"], r["seed"], r["sigma"], r["k"], args.tol, bc=r["bc"])] = r
                i += 1
            for tk in list(pending):
                out = srv.poll(tk, raise_on_error=False)
                if out is not None:
                    st, r = out[2], pending.pop(tk)
                    lat.append(st["latency_ms"])
                    pairs += st["nconv"]
                    failed += st["status"] not in (0, ajd.JD_ENOCONV)
                    per.append([r["L"], round(r["W"], 2), round(r["sigma"], 3), r["k"], round(st["latency_ms"]),
                                round(st["setup_ms"]), round(st["solve_ms"]), st["outer_its"], st["inner_its"],
                                st["nconv"]])
            time.sleep(0.002)
        elapsed = time.perf_counter() - start
        info = srv.info()
    out = summarize_requests(lat, pairs, failed, elapsed, info["peak_solving"], slots, setup_threads)
    out["per_request"] = {"fields": ["L", "W", "sigma", "k", "latency_ms", "setup_ms", "solve_ms", "outer", "inner",
                                     "nconv"], "rows": per}
    out["unconverged"] = sum(1 for r in per if r[9] < r[3])
    out["max_outer"] = args.serve_max_outer
    return out


def summarize_requests(lat, pairs, failed, elapsed, peak, slots, setup_threads):
    """Throughput and latency percentiles of one request run; with several
    ranks (each serving its balanced share of the requests) the eigenpairs
    are summed, the time is the slowest rank's and the percentiles are over
    every rank's latencies."""
    import numpy as np
    from paper_math_0508111_gb300 import replicas
    parts = replicas.gather_to_root(list(lat))
    allat = [x for part in parts for x in part] if parts is not None else list(lat)
    pairs = int(replicas.sum_over_ranks(pairs))
    failed = int(replicas.sum_over_ranks(failed))
    elapsed = replicas.max_over_ranks(elapsed)
    lat = np.sort(np.array(allat)) if allat else np.zeros(1)
    return {"value": pairs / elapsed, "unit": UNIT, "requests": len(allat), "failed": failed, "eigenpairs": pairs,
            "p50_latency_ms": float(np.percentile(lat, 50)), "p99_latency_ms": float(np.percentile(lat, 99)),
            "max_latency_ms": float(lat[-1]), "seconds": elapsed, "peak_concurrent_solves": peak,
            "slots": slots, "setup_threads": setup_threads}


def rank_share(ajd, reqs, rank, world):
    """This rank's balanced share of independent requests (greedy by work,
    under the HBM estimate of each solve); all of them on one GPU."""
    if world == 1:
        return reqs
    from paper_math_0508111_gb300 import replicas
    work = [replicas.problem_work(r["L"], r["k"]) for r in reqs]
    mem = [ajd.Server.estimate(r["L"], r["k"]) for r in reqs]
    return [reqs[i] for i in replicas.balanced_shard(work, mem, world)[rank]]


def serving_sweep(ajd, args, precision, rank=0, world=1):
    """The serving workload (workloads.serve_recipe: L uniform in
    16..serve_lmax, W in [8, 24], sigma in [-2, 2], k in {1, 5, 10}, request
    r on disorder seed 10^6 + r): first the capacity, the completion rate
    of serve_requests requests all submitted at t = 0, then Poisson streams
    of serve_requests requests at each rate of serve_rates times that
    capacity, with p50/p99 latency (submission to completion) per rate."""
    import workloads
    t_start = time.perf_counter()
    base = workloads.serve_recipe(args.serve_requests, 1.0, seed=7, lmax=args.serve_lmax)
    progress("serving: capacity run (%d requests at t = 0)" % len(base))
    sat = run_requests(ajd, args, precision, rank_share(ajd, [dict(r, t=0.0) for r in base], rank, world),
                       args.serve_slots, args.serve_setup_threads)
    capacity = sat["requests"] / sat["seconds"]
    out = {"capacity_requests_per_s": capacity, "saturated": sat, "rates": [], "skipped_rates": []}
    for i, mult in enumerate(args.serve_rates):
        elapsed = replicas_max(time.perf_counter() - t_start)
        if elapsed > args.serve_budget_s:
            out["skipped_rates"].append(mult)
            continue
        progress("serving: %g x capacity" % mult)
        # the same requests at every rate (same draws, arrival times scaled)
        reqs = workloads.serve_recipe(args.serve_requests, mult * capacity, seed=7, lmax=args.serve_lmax)
        res = run_requests(ajd, args, precision, rank_share(ajd, reqs, rank, world), args.serve_slots,
                           args.serve_setup_threads)
        res["rate_multiple"] = mult
        res["rate_per_s"] = mult * capacity
        out["rates"].append(res)
    out["sample"] = ("%d requests per point, L~U{16..%d}, W~U[8,24], sigma~U[-2,2], k in {1,5,10}, tol %g, at most "
                     "%d outer steps per request; capacity from all requests submitted at t=0, then Poisson arrivals "
                     "at %s x capacity, a rate skipped once the sweep has run %g s (a bounded sample of the "
                     "4096-request stream)"
                     % (args.serve_requests, args.serve_lmax, args.tol, args.serve_max_outer,
                        "/".join("%g" % m for m in args.serve_rates), args.serve_budget_s))
    return out


def replicas_max(x):
    from paper_math_0508111_gb300 import replicas
    return replicas.max_over_ranks(x)


def batch_sample(ajd, args, precision, rank=0, world=1):
    """A bounded sample of the batch workload (workloads.batch_recipe: L in
    {20,30,40,50}, W in {12,16.5,20}, sigma in {-1,0,1}, k = 5, seeds
    1000 + p), all problems submitted at t = 0 to one jd_server."""
    import workloads
    reqs = [dict(r, t=0.0) for r in workloads.batch_recipe(args.batch_sample, seed=42)]
    out = run_requests(ajd, args, precision, rank_share(ajd, reqs, rank, world), args.serve_slots,
                       args.serve_setup_threads)
    out["sample"] = ("first %d problems of the 256-problem batch (L in {20,30,40,50}, W in {12,16.5,20}, "
                     "sigma in {-1,0,1}, k=5), submitted at t=0" % len(reqs))
    return out


def run_batch_workload(args):
    """--workload batch: the 256-problem batch (workloads.batch_recipe: L in
    {20,30,40,50}, W in {12,16.5,20}, sigma in {-1,0,1}, k = 5, seeds 1000 + p)
    submitted at once to a jd_server; one JSON line."""
    import torch
    import paper_math_0508111_gb300 as ajd
    import workloads
    head = {"mixed": ajd.JD_MIXED, "fp32": ajd.JD_FP32, "fp64": ajd.JD_FP64}[args.precision]
    reqs = [dict(r, t=0.0) for r in workloads.batch_recipe(args.batch_problems, seed=42)]
    warm = [dict(r, t=0.0, seed=r["seed"] + 10 ** 5) for r in workloads.batch_recipe(max(args.warmup, 1), seed=43)]
    run_requests(ajd, args, head, warm, args.serve_slots, args.serve_setup_threads)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    out = run_requests(ajd, args, head, reqs, args.serve_slots, args.serve_setup_threads)
    clocks = sampler.stop()
    line = {"metric": "eigenpairs/s, batch of %d Anderson problems (L in {20,30,40,50}), resid<=%g" % (len(reqs), args.tol),
            "value": out["value"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": len(warm),
            "ms_per_step": 1e3 * out["seconds"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "f32+f64", "fp32": "f32+f64", "fp64": "f64"}[args.precision], "data": "synthetic",
            "config": {"workload": "batch-%d-L20..50-W12..20-sigma-1..1-k5" % len(reqs), "precision": args.precision,
                       "submission": "all requests at t = 0 to one jd_server"},
            "batch": out, "clocks": clocks}
    print(json.dumps(line), flush=True)


def cpu_baseline(W, sigma, k, tol, L_sample=30, threads=None):
    """The oracle (shift-and-invert Lanczos over SuperLU) on a bounded
    sample: one L_sample^3 lattice of the same disorder, shift and k, solved
    to the metric's residual tol * ||A||.  With ``threads`` the oracle runs
    in a child process whose BLAS/OpenMP pools have that many threads."""
    if threads is not None:
        env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
                   MKL_NUM_THREADS=str(threads))
        code = ("import json, sys; sys.path.insert(0, %r); import bench; "
                "print(json.dumps(bench.cpu_baseline(%r, %r, %r, %r, %r)))" % (ROOT, W, sigma, k, tol, L_sample))
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True)
        if r.returncode != 0:
            return {"error": r.stderr[-500:]}
        out = json.loads(r.stdout.strip().splitlines()[-1])
        out["threads"] = threads
        return out
    import numpy as np  # noqa: F401
    from oracle import lanczos, lattice, rng
    import resource
    eps = rng.potential(L_sample, W, 1)
    A = lattice.assemble(L_sample, eps)
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    w, X, info = lanczos.shift_invert_nearest(A, sigma, k, tol=tol, norm_a=lattice.norm_bound(eps))
    dt = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    # threads actually used: CPU time over wall time of the run (SuperLU's
    # factorization and solves are single-threaded; BLAS may add a little)
    busy = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    cores = round(busy / dt, 2) if dt > 0 else 1.0
    return {"value": k / dt, "unit": UNIT, "cores": cores, "cores_available": os.cpu_count(), "kind": "oracle",
            "sample": "oracle shift-invert Lanczos + SuperLU on one L=%d lattice (W=%g, sigma=%g, k=%d, residual "
                      "<= %g ||A||): %.1f s, %d Lanczos steps; a bounded sample of the L=100 workload, whose LU the "
                      "oracle does not reach in bounded time" % (L_sample, W, sigma, k, tol, dt, info["steps"]),
            "seconds": dt}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    for _ in range(args.warmup):
        pass  # the oracle has no state to warm; keep the contract's shape
    vals = []
    t0 = time.perf_counter()
    for s in range(args.steps):
        cb = cpu_baseline(args.W, args.sigma, args.k, args.tol, args.cpu_L)
        vals.append(cb["seconds"])
    total = time.perf_counter() - t0
    value = args.k * args.steps / sum(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "anderson-L%d-W%g-periodic-k%d-sigma%g (oracle sample of the L=100 workload)"
                       % (args.cpu_L, args.W, args.k, args.sigma)},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": cb["cores"],
                             "cores_available": cb["cores_available"], "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch":
        run_batch_workload(args)
        return
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_math_0508111_gb300 as ajd
    L, W, k, tol, sigma = args.L, args.W, args.k, args.tol, args.sigma
    nwarm, nsteps = args.warmup, args.steps
    from paper_math_0508111_gb300 import replicas
    seeds = replicas.realisation_seeds(nwarm + nsteps, rank)
    bc_code = ajd.JD_PERIODIC if args.bc == "periodic" else ajd.JD_HARDWALL

    def make_lattice(s):
        if args.model == "offdiag":
            return ajd.Anderson.offdiag(L, s, diag=1.28, width=1.0, bc=bc_code)
        return ajd.Anderson(L, W, s, bc_code)

    lattices = [make_lattice(s) for s in seeds]  # potentials (and bonds) resident before timing
    n = lattices[0].n
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda", dtype=torch.float32)
    stream = torch.cuda.current_stream()
    ev_out = np.zeros(k)
    X_dev = torch.empty((k, n), device="cuda", dtype=torch.float64)

    ildl_over = {"n_dense": args.n_dense} if args.n_dense > 0 else None

    def one(h, precision):
        p = ajd.jd_params(precision=precision, ildl=ildl_over)
        st = ajd._ffi.JdStats()
        rc = ajd._ffi.lib().jd_solve(h.handle, sigma, k, tol, ajd.ctypes.byref(p),
                                     ev_out.ctypes.data_as(ajd.ctypes.c_void_p),
                                     ajd.ctypes.c_void_p(X_dev.data_ptr()), ajd.ctypes.byref(st),
                                     ajd.ctypes.c_void_p(stream.cuda_stream))
        ajd._ffi.check(rc, "jd_solve")
        return ajd._stats_dict(st)

    def batch(handles, precision, ev_bufs, x_bufs):
        """jd_solve_batch over the given problems (or, with --method lanczos,
        jd_lanczos_solve one after another); ev_bufs/x_bufs are raw pointers
        (host or device)."""
        m = len(handles)
        vp = ajd.ctypes.c_void_p
        if args.method == "lanczos":
            out = []
            for i in range(m):
                p = ajd.jd_params(precision=precision, ildl=ildl_over)
                st = ajd._ffi.JdStats()
                hv = handles[i] if isinstance(handles[i], vp) else vp(handles[i])
                rc = ajd._ffi.lib().jd_lanczos_solve(hv, sigma, k, tol, ajd.ctypes.byref(p), vp(ev_bufs[i]),
                                                     vp(x_bufs[i]), ajd.ctypes.byref(st), vp(stream.cuda_stream))
                ajd._ffi.check(rc, "jd_lanczos_solve")
                out.append(ajd._stats_dict(st))
            return out
        hs = (vp * m)(*handles)
        sig = (ajd.ctypes.c_double * m)(*([sigma] * m))
        kk = (ajd.ctypes.c_int * m)(*([k] * m))
        ep = (vp * m)(*ev_bufs)
        xp = (vp * m)(*x_bufs)
        sts = (ajd._ffi.JdStats * m)()
        p = ajd.jd_params(precision=precision, ildl=ildl_over)
        rc = ajd._ffi.lib().jd_solve_batch(hs, m, sig, kk, tol, ajd.ctypes.byref(p), ep, xp, sts,
                                           args.setup_threads, vp(stream.cuda_stream))
        ajd._ffi.check(rc, "jd_solve_batch")
        return [ajd._stats_dict(sts[i]) for i in range(m)]

    head = {"mixed": ajd.JD_MIXED, "fp32": ajd.JD_FP32, "fp64": ajd.JD_FP64}[args.precision]
    ev_dev = torch.empty((nsteps, k), device="cuda", dtype=torch.float64)
    X_all = torch.empty((nsteps, k, n), device="cuda", dtype=torch.float64)
    ev_ptrs = [ev_dev[i].data_ptr() for i in range(nsteps)]
    x_ptrs = [X_all[i].data_ptr() for i in range(nsteps)]
    # warm-up: the same pipeline on the warm-up realisations
    progress("warm-up: %d realisations" % nwarm)
    batch([h.handle for h in lattices[:nwarm]], head, ev_ptrs[:1] * nwarm, x_ptrs[:1] * nwarm)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    progress("timed: %d realisations" % nsteps)
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    flush.zero_()  # L2 flushed before the step sequence (256 MiB write)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("bench_timed")  # ncu --nvtx --nvtx-include bench_timed/ captures this region only
    e0.record(stream)
    stats = batch([h.handle for h in lattices[nwarm:]], head, ev_ptrs, x_ptrs)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    elapsed = replicas.max_over_ranks(e0.elapsed_time(e1) / 1e3)  # the slowest rank's time
    value = world * nsteps * k / elapsed
    setup_s = sum(s["setup_ms"] for s in stats) / 1e3
    solve_s = sum(s["solve_ms"] for s in stats) / 1e3
    ev_batched = ev_dev.cpu().numpy()

    # binary64 comparison arms on the first fp64_steps timed realisations:
    # plain (one jd_solve after another) and pipelined (jd_solve_batch, the
    # same pipeline as the headline), so that the precision gain is
    # separated from the pipelining gain
    fp64 = None
    if not args.no_fp64:
        m64 = max(1, min(args.fp64_steps, nsteps))
        progress("binary64 arms: %d realisations" % m64)
        sub = lattices[nwarm:nwarm + m64]
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        st64, ev64 = [], []
        f0.record(stream)
        for i in range(m64):
            flush.zero_()
            st64.append(one(sub[i], ajd.JD_FP64))
            ev64.append(ev_out.copy())
        f1.record(stream)
        torch.cuda.synchronize()
        t64 = f0.elapsed_time(f1) / 1e3
        ev64 = np.array(ev64)
        flush.zero_()
        torch.cuda.synchronize()
        f0.record(stream)
        stp = batch([h.handle for h in sub], ajd.JD_FP64, ev_ptrs[:m64], x_ptrs[:m64])
        f1.record(stream)
        torch.cuda.synchronize()
        tp = f0.elapsed_time(f1) / 1e3
        fp64 = {"value": world * m64 * k / t64, "unit": UNIT, "realisations": m64, "ms_per_step": 1e3 * t64 / m64,
                "setup_s_per_step": sum(s["setup_ms"] for s in st64) / 1e3 / m64,
                "solve_only_value": world * m64 * k / (sum(s["solve_ms"] for s in st64) / 1e3),
                "outer_its": [s["outer_its"] for s in st64], "inner_its": [s["inner_its"] for s in st64],
                "headline_vs_fp64_max_abs_dlambda_over_normA":
                    float(np.max(np.abs(ev_batched[:m64] - ev64)) / max(h.norm() for h in sub)),
                "pipelined": {"value": world * m64 * k / tp, "unit": UNIT, "ms_per_step": 1e3 * tp / m64,
                              "setup_s_per_step": sum(s["setup_ms"] for s in stp) / 1e3 / m64,
                              "solve_s_per_step": sum(s["solve_ms"] for s in stp) / 1e3 / m64,
                              "inner_its": [s["inner_its"] for s in stp],
                              "note": "binary64 inner solve through the same jd_solve_batch pipeline "
                                      "(%d setup threads) as the headline" % args.setup_threads},
                "note": "plain: one binary64 jd_solve after another (setup + solve per realisation)"}

    # end to end through the public API from host memory: potentials copied
    # in from pinned buffers, the same pipelined batch writing eigenvalues
    # and eigenvectors into pinned host buffers
    e2e = None
    if not args.no_e2e and args.model == "diagonal":
        progress("end to end through the C ABI from host buffers")
        pots = [torch.from_numpy(h.potential()).pin_memory() for h in lattices[nwarm:]]
        Xh = torch.empty((nsteps, k, n), dtype=torch.float64).pin_memory()
        evh = torch.empty((nsteps, k), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs = []
        for i in range(nsteps):
            h = ajd.ctypes.c_void_p()
            ajd._ffi.call("anderson_create_from_potential", L, ajd.ctypes.c_void_p(pots[i].data_ptr()), bc_code,
                          ajd.ctypes.byref(h))
            hs.append(h.value)
        batch(hs, head, [evh[i].data_ptr() for i in range(nsteps)], [Xh[i].data_ptr() for i in range(nsteps)])
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        for h in hs:
            ajd._ffi.lib().anderson_destroy(ajd.ctypes.c_void_p(h))
        e2e = {"value": world * nsteps * k / te, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
               "d2h_bytes_per_step": 8 * n * k + 8 * k}

    # roofline of the dominant kernel: the preconditioner application
    peak, peak_kind = measured_peaks()
    calls = sum(s["precond_calls"] for s in stats)
    ms = sum(s["precond_ms"] for s in stats)
    info = stats[-1]["ildl"]
    val_b, vec_b = {"fp64": (8, 8), "fp32": (4, 4), "mixed": (4, 8)}[args.precision]
    bytes_per = apply_bytes(info, val_b, vec_b)
    achieved = bytes_per / (ms / calls / 1e3) / 1e9 if calls else 0.0
    forms = sorted({s["ildl"]["apply_form"] for s in stats})
    form = forms[0] if len(forms) == 1 else None
    traffic = measured_traffic(args.precision, info, form) if form is not None else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "kernel": APPLY_KERNELS[form] if form is not None else
                " / ".join(APPLY_KERNELS[f] for f in forms) + " (autotuned per factor)",
                "peak_kind": peak_kind + " (hbm_gbs, copy test)", "algorithmic_bytes_per_launch": bytes_per,
                "avg_launch_ms": ms / calls if calls else None, "launches_timed": calls,
                "timed_as": "CUDA events around each ildl apply call on the solver's stream (the dataflow form's "
                            "two sentinel fills of w and z included)"}
    # the inner solve's stencil runs in binary64 for the binary64 and mixed
    # solves (24 B/site: x, eps, y) and in binary32 for the binary32 one
    stencil_prec = "binary32" if args.precision == "fp32" else "binary64"
    stencil_bps = 12 if args.precision == "fp32" else 24
    stencil_calls = sum(s["stencil_calls"] for s in stats)
    stencil_ms = sum(s["stencil_ms"] for s in stats)

    # the batch sample and the serving stream split over the ranks by the
    # greedy work/HBM balance (independent problems, host-side gathers only)
    if args.batch_sample > 0:
        progress("batch sample: %d problems" % args.batch_sample)
    batch_c4 = batch_sample(ajd, args, head, rank, world) if args.batch_sample > 0 else None
    serving = serving_sweep(ajd, args, head, rank, world) if args.serve_requests > 0 else None

    cpu = None
    if rank == 0 and not args.no_cpu:
        progress("CPU oracle baseline (L = %d)" % args.cpu_L)
        cpu = cpu_baseline(W, sigma, k, tol, args.cpu_L)
        cpu.pop("seconds", None)
        one_thread = cpu_baseline(W, sigma, k, tol, args.cpu_L, threads=1)
        one_thread.pop("seconds", None)
        cpu["one_thread"] = one_thread

    if args.model == "diagonal":
        workload = "anderson-L%d-W%g-%s-k%d-sigma%g-tol%g" % (L, W, args.bc, k, sigma, tol)
    else:
        workload = "anderson-offdiag-L%d-diag1.28-hop0.5-%s-k%d-sigma%g-tol%g" % (L, args.bc, k, sigma, tol)
    vs_base, vs_note = None, None
    if L == 100 and k == 5 and sigma == 0.0 and (args.model, args.bc) == ("diagonal", "periodic") and W == 16.5:
        vs_base = value / PAPER_EIGENPAIRS_PER_S
        vs_note = ("paper Table 4: 978 s for 5 eigenpairs at M=100, w=16.5 on one Itanium2 core "
                   "(context; the paper does not state its residual tolerance)")
    elif L == 100 and k == 5 and sigma == 0.0 and (args.model, args.bc) in PAPER_TABLE6_S:
        vs_base = value / (5.0 / PAPER_TABLE6_S[(args.model, args.bc)])
        vs_note = "paper Table 6, M=100: %.0f s for 5 eigenpairs (context)" % PAPER_TABLE6_S[(args.model, args.bc)]
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": nsteps,
                "warmup": nwarm, "ms_per_step": 1e3 * elapsed / nsteps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": vs_base,
                "vs_baseline_note": vs_note,
                "dtype": {"mixed": "f32+f64", "fp32": "f32+f64", "fp64": "f64"}[args.precision], "data": "synthetic",
                "config": {"workload": workload, "model": args.model,
                           "L": L, "W": W if args.model == "diagonal" else None, "k": k, "sigma": sigma, "tol": tol,
                           "bc": args.bc,
                           "precision": {"mixed": "mixed: binary32 factor applied with float-float sums, binary64 "
                                                  "SQMR vectors/stencil/outer",
                                         "fp32": "binary32 inner solve (stencil, preconditioner, SQMR), binary64 outer",
                                         "fp64": "binary64 throughout"}[args.precision],
                           "step": "one realisation solved completely (preconditioner setup + Jacobi-Davidson); "
                                   "the K steps run as one pipelined jd_solve_batch (setups of later realisations "
                                   "on %d host threads overlap the GPU solves of earlier ones)" % args.setup_threads,
                           "l2": "flushed before the timed batch (256 MiB write); the working set of each solve "
                                 "(factor %.0f MB) exceeds L2" % (info["nnz_L"] * 16 / 1e6),
                           "seeds": seeds[nwarm:], "setup_threads": args.setup_threads,
                           "parallelism": "replicas (independent realisations per GPU)"},
                "setup_s_per_step": setup_s / nsteps, "solve_s_per_step": solve_s / nsteps,
                "solve_only_value": world * nsteps * k / solve_s,
                "iterations": {"outer": [s["outer_its"] for s in stats], "inner": [s["inner_its"] for s in stats],
                               "restarts": [s["restarts"] for s in stats]},
                "max_residual": max(s["max_residual"] for s in stats),
                "preconditioner": {"levels": info["levels"], "n_dense": info["n_dense"], "nnz_L": info["nnz_L"],
                                   "fill": info["fill"], "n_2x2": info["n_2x2"],
                                   "apply_threads_per_row_shift": [s["ildl"]["apply_shift"] for s in stats],
                                   "apply_form": [s["ildl"]["apply_form"] for s in stats]},
                "fp64": fp64, "e2e": e2e, "roofline": roofline, "batch": batch_c4, "serving": serving,
                "stencil": {"precision": stencil_prec, "bytes_per_site": stencil_bps, "sites": n,
                            "calls": stencil_calls, "avg_ms": stencil_ms / stencil_calls if stencil_calls else None,
                            "achieved_GBps": stencil_bps * n / (stencil_ms / stencil_calls / 1e3) / 1e9
                            if stencil_calls else None,
                            "note": "the stencil calls of the headline solves (SQMR and outer steps), timed with "
                                    "CUDA events around each call"},
                "cpu_baseline": cpu, "clocks": clocks,
                "gpu_launches": int(sum(s["kernel_launches"] for s in stats))}
        print(json.dumps(line), flush=True)
    for h in lattices:
        h.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
