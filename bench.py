#!/usr/bin/env python
"""Benchmark of the GB300 CGGM solver (alternating Newton coordinate descent).

One step is one Newton iteration of Algorithm 1 (every per-iteration step of the hot
path: products R, P, Psi, gradients, stopping quantity, active sets, the Lambda
coordinate pass, the Armijo search and the Theta coordinate pass) on the genotype chain
workload p = q = 5000, n = 1000, lambda = 0.05, in the mixed-precision path.  W warm-up
iterations start from Lambda = I, Theta = 0; the K timed iterations continue from there
(inputs resident on the device, warm start passed in device memory).

Printed (rank 0, one JSON line): Newton iterations per second over all ranks, the
roofline of the dominant kernel (the coordinate pass with the larger share of the timed
region) and of the other pass, the same iterations end to end through the C ABI from host
buffers, the double-precision path's rate on the same workload (fp64), a served
regularisation-path run at the served workload's full request sizes (trimmed in count and
iterations, and saying so), the time to a 1e-6 relative objective gap of the mixed and the
FP64 paths on the small chain workload (p=200, q=100, n=100), where a whole solve fits in
seconds, and the oracle's CPU rate on a bounded sample.  With --gpus N (torchrun) every rank
solves an independent replica (another seed): the solve does not shard.

Other modes: --gap-trace S records f against device time for both precisions on the
5000 x 5000 workload (S seconds each; --gap-fp64 S2 gives the FP64 path its own budget);
--large K runs K iterations of the 40000 x 20000 workload with a KKT check; --serve runs the
served paths alone; --profile-sweep, --profile-theta and --profile-contract are the bounded
cases of the ncu captures; --profile-chol times the FP64 factorisation against cuBLAS DGEMM.

--impl reference times the CPU oracle (the plain double-precision restatement of the
method) on a bounded sample of the same workload and prints the same kind of line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "chain-geno-p5000-q5000-n1000"
SMALL = "chain-gauss-p200-q100-n100"
METRIC = "time to 1e-6 rel obj gap, mixed vs FP64 GPU; λ-path solves/s, p50/p99"


SWEEP_SOURCES = ["paper_1509_04681_gb300/csrc/sweeps.cu", "paper_1509_04681_gb300/csrc/sweeps.cuh",
                 "paper_1509_04681_gb300/csrc/common.cuh", "paper_1509_04681_gb300/csrc/mbar.cuh"]


def profiled_traffic(kernel, units):
    """DRAM bytes (read + write) of one launch of `kernel` over `units` coordinates, scaled
    from the committed ncu summary of a bounded launch of the same kernel; None when there
    is none, or when the kernel sources no longer hash to the captured version."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel}-q5000-bounded.md")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if line.startswith("    ") and ":" in line:
            k, v = line.strip().split(":", 1)
            kv[k.strip()] = v.strip()
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if kv.get("kernel") != kernel or kv.get("source_sha256") != h.hexdigest():
        return None
    return float(kv["dram_bytes"]) / float(kv["units"]) * units


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                    "sw_power_cap"), f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    """Largest value over the ranks (the slowest rank's time decides the job's rate)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Each rank solves an independent replica of the workload: the seed is the rank."""
    return rank


def job_rate(iters_per_rank, sec_max, world):
    """Whole-job Newton iterations per second: every rank runs the same number of
    iterations on its replica; the job takes as long as its slowest rank."""
    return world * iters_per_rank / sec_max


def pass_cost(run, m, budget_s, k0=1024):
    """Seconds of one full oracle pass over m coordinates from a bounded sample.

    The oracle's pass wrappers do work that does not grow with the number of coordinates
    (array copies, zeroing the cache, the initial V = Theta Sigma of the Theta pass), so
    the pass is timed with no coordinates (that fixed part, t0) and over a prefix of k
    coordinates, k grown 4x at a time until the coordinate part t(k) - t0 is well above
    the fixed part's noise or the budget is spent; only the slope (t(k) - t0) / k is
    scaled to the full set: t_full = t0 + m (t(k) - t0) / k.
    Returns (t_full, t0, k, t(k))."""
    def timed(k):
        ts = time.perf_counter()
        run(k)
        return time.perf_counter() - ts
    t0 = timed(0)
    spent = t0
    k = min(m, k0)
    while True:
        tk = timed(k)
        spent += tk
        if k >= m:
            return tk, t0, k, tk
        resolved = tk - t0 >= max(0.5, 0.5 * t0)
        if resolved or spent + 4 * tk > budget_s:
            slope = max(0.0, tk - t0) / k
            return t0 + slope * m, t0, k, tk
        k = min(m, 4 * k)


def cpu_oracle_rate(pr, budget_s=25.0):
    """Oracle Newton iterations per second on a bounded sample of the workload: the dense
    steps of one iteration (covariances amortised out, Sigma, Psi, gradients, active sets,
    objective) once, counted twice (the Armijo trial evaluates the objective again), and
    each coordinate pass by pass_cost: its fixed part once plus its per-coordinate cost
    (timed on a prefix of the active set) times the full active set."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    q = Syy.shape[0]
    p = Sxy.shape[0]
    Lam, Th = np.eye(q), np.zeros((p, q))
    t1 = time.perf_counter()
    G_L, G_T, Sigma, Psi = oracle.gradients(Lam, Th, Sxx, Sxy, Syy)
    li, lj, ti, tj = oracle.active_sets(G_L, G_T, Lam, Th, pr.lam_L, pr.lam_T)
    oracle.objective(Lam, Th, Sxx, Sxy, Syy, pr.lam_L, pr.lam_T)
    t_dense = time.perf_counter() - t1
    left = max(2.0, budget_s - t_dense)
    tl = pass_cost(lambda k: oracle.lambda_sweep(Sigma, Psi, Syy, Lam, li[:k], lj[:k], pr.lam_L),
                   len(li), left / 2)
    tt = pass_cost(lambda k: oracle.theta_sweep(Sxx, Sxy, Sigma, Th, ti[:k], tj[:k], pr.lam_T),
                   len(ti), left / 2)
    t_iter = 2 * t_dense + tl[0] + tt[0]
    try:
        from threadpoolctl import threadpool_info
        cores = max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    return {"value": 1.0 / t_iter, "unit": "Newton iterations/s", "cores": cores,
            "kind": "oracle",
            "sample": (f"{WORKLOAD} iteration 0: dense steps (Sigma, Psi, gradients, "
                       f"objective, active sets) timed once ({t_dense:.2f} s) and counted twice "
                       f"(the Armijo objective); each coordinate pass timed with no coordinates "
                       f"(its fixed part: Lambda {tl[1]:.2f} s, Theta {tt[1]:.2f} s) and over a "
                       f"prefix (Lambda {tl[2]} of {len(li)} coordinates in {tl[3]:.2f} s, "
                       f"Theta {tt[2]} of {len(ti)} in {tt[3]:.2f} s), fixed part counted once "
                       f"and the per-coordinate slope scaled to the full active set; "
                       f"coordinate passes single-threaded C, dense steps numpy BLAS"),
            "seconds_per_iteration": t_iter,
            "seconds_measured": round(time.perf_counter() - t0, 2)}


def reference_config(pr):
    """The workload the reference arm ran: sizes from the generated problem, recipe from
    the workload table."""
    import synth
    w = synth.WORKLOADS[WORKLOAD]
    x = ("genotype Binomial(2, MAF~U(0.05,0.5)) standardised" if w["x_kind"] == "genotype"
         else "iid N(0,1) standardised")
    net = "chain (1.0 / 0.4)" if w["lam_kind"] == "chain" else w["lam_kind"]
    return {"workload": WORKLOAD, "p": int(pr.X.shape[1]), "q": int(pr.Y.shape[1]),
            "n": int(pr.X.shape[0]), "lambda": pr.lam_L, "x": x, "network": net,
            "theta_nnz_per_col": w["theta_nnz"], "seed": w["seed"]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    pr = synth.workload(WORKLOAD)
    rates = []
    budget = max(8.0, 180.0 / max(1, args.steps + args.warmup))
    t_run = time.perf_counter()
    for k in range(args.warmup + args.steps):
        r = cpu_oracle_rate(pr, budget_s=budget)
        if k >= args.warmup:
            rates.append(r)
    v = statistics.median([r["value"] for r in rates])
    wall = time.perf_counter() - t_run
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Newton iterations/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": reference_config(pr),
            "cpu_baseline": {"kind": "oracle", "cores": rates[0]["cores"],
                             "sample": rates[0]["sample"], "value": v,
                             "unit": "Newton iterations/s"},
            "timing": {"extrapolated": True,
                       "note": "each step times a bounded sample of one oracle Newton "
                               "iteration (dense steps, each pass's fixed part, a prefix of "
                               "each pass); ms_per_step is the whole iteration it implies",
                       "sample_wall_s_per_step": wall / max(1, args.warmup + args.steps),
                       "wall_s": wall},
            "e2e": {"value": v, "unit": "Newton iterations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_to_gap(ctx, cg, pr, torch):
    """Seconds (device time of the solve) to reach (f - f*)/|f*| <= 1e-6, f* from the
    double-precision path run until progress stops."""
    ref = ctx.cggm_solve_dense(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-12,
                         opts=cg.make_opts(precision=cg.CGGM_FP64, max_iter=4000))
    fstar = ctx.cggm_objective(pr.X, pr.Y, ref.Lambda, ref.Theta, pr.lam_L, pr.lam_T)
    target = fstar + 1e-6 * abs(fstar)
    out = {"workload": SMALL, "f_star": fstar}
    for name, prec in (("mixed", cg.CGGM_MIXED), ("fp64", cg.CGGM_FP64)):
        r = ctx.cggm_solve_dense(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-12,
                           opts=cg.make_opts(precision=prec, max_iter=4000, target_f=target))
        f = ctx.cggm_objective(pr.X, pr.Y, r.Lambda, r.Theta, pr.lam_L, pr.lam_T)
        out[name] = {"seconds": r.info["seconds"], "iterations": r.info["iterations"],
                     "reached": bool((f - fstar) / abs(fstar) <= 1e-6),
                     "rel_gap": (f - fstar) / abs(fstar)}
    return out


def run_profile_sweep(args):
    """A bounded Lambda coordinate pass at q = 5000 (Sigma, Psi and the cache, 100 MB each,
    exceed L2): rows 0..39 of a dense active set, ~2e5 coordinates, run twice through
    cggm_lambda_sweep.  Used for ncu captures of the sweep kernel."""
    import numpy as np
    import paper_1509_04681_gb300 as cg
    from paper_1509_04681_gb300 import build as pkg_build
    pkg_build.build()
    q = 5000
    rng = np.random.default_rng(0)
    A = rng.standard_normal((q, q + 8)) / np.sqrt(q)
    Sig = A @ A.T + np.eye(q)
    Bm = rng.standard_normal((q, 64)) / 8
    Psi = Bm @ Bm.T
    Syy = Sig + 0.1 * np.eye(q)
    Lam = np.linalg.inv(Sig)
    iu, ju = np.triu_indices(q)
    keep = iu < 40
    li, lj = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
    prec = cg.CGGM_MIXED if args.precision == "mixed" else cg.CGGM_FP64
    with cg.Context(0) as ctx:
        for _ in range(2):
            D = ctx.cggm_lambda_sweep(Sig, Psi, Syy, Lam, li, lj, 0.01, precision=prec)
    print(json.dumps({"profile_sweep": {"q": q, "coordinates": int(len(li)),
                                        "precision": args.precision,
                                        "d_abs_sum": float(np.abs(D).sum())}}))


def run_profile_theta(args):
    """A bounded Theta coordinate pass at p = q = 5000, n = 1000 (S_xx, Delta V^T and Sigma,
    100 MB each, exceed L2): every column of 40 rows spread evenly over the inputs (so that
    the dot products' lengths average those of a whole pass), ~2e5 coordinates, run twice
    through cggm_theta_sweep.  Used for ncu captures of the Theta sweep kernel."""
    import numpy as np
    import paper_1509_04681_gb300 as cg
    from paper_1509_04681_gb300 import build as pkg_build
    pkg_build.build()
    p = q = 5000
    n = 1000
    rng = np.random.default_rng(0)
    X = rng.standard_normal((n, p))
    A = rng.standard_normal((q, q + 8)) / np.sqrt(q)
    Sig = A @ A.T + np.eye(q)
    Sxy = rng.standard_normal((p, q)) * 0.05
    Th = np.zeros((p, q))
    rows = np.arange(0, p, p // 40)[:40]
    ti = np.repeat(rows, q).astype(np.int32)
    tj = np.tile(np.arange(q), rows.size).astype(np.int32)
    prec = cg.CGGM_MIXED if args.precision == "mixed" else cg.CGGM_FP64
    with cg.Context(0) as ctx:
        for _ in range(2):
            T = ctx.cggm_theta_sweep(X, Sxy, Sig, Th, ti, tj, 0.01, precision=prec)
    print(json.dumps({"profile_theta": {"p": p, "q": q, "n": n, "coordinates": int(ti.size),
                                        "precision": args.precision,
                                        "theta_abs_sum": float(np.abs(T).sum())}}))


def run_profile_chol(args):
    """FP64 factorisation throughput: cggm_cholesky (Cholesky of Lambda, log det and Sigma =
    Lambda^-1, the step every Newton iteration and every Armijo trial runs) on device buffers
    at q = 5000 and 20000, timed with CUDA events; flops q^3/3 for the factor and 2 q^3/3 for
    Sigma (W = L^-1 with a triangular right-hand side, then W^T W).  Beside it, cuBLAS's
    double-precision GEMM rate (torch.matmul at 8192^3) as the reference FP64 rate."""
    import ctypes
    import torch
    import paper_1509_04681_gb300 as cg
    from paper_1509_04681_gb300 import build as pkg_build
    pkg_build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = cg.Context(0, stream=stream.cuda_stream)
    lib = cg.cggm._lib()
    g = torch.Generator(device=dev).manual_seed(0)
    out = {}
    for q in (5000, 20000):
        M = torch.randn(q, q, device=dev, dtype=torch.float64, generator=g) / q ** 0.5
        Lam = M @ M.T + torch.eye(q, device=dev, dtype=torch.float64)
        del M
        L = torch.empty_like(Lam)
        S = torch.empty_like(Lam)
        ld = ctypes.c_double()
        times = []
        for rep in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = lib.cggm_cholesky(ctx._h, q, Lam.data_ptr(), L.data_ptr(), ctypes.byref(ld),
                                   S.data_ptr(), cg.CGGM_FP64)
            e1.record(stream)
            torch.cuda.synchronize()
            assert st == 0, st
            if rep:
                times.append(e0.elapsed_time(e1) / 1e3)
        sec = min(times)
        flops = q ** 3 / 3 + 2 * q ** 3 / 3
        out[f"q{q}"] = {"seconds": sec, "tflops": flops / sec / 1e12,
                        "flops": "q^3/3 (factor) + 2 q^3/3 (Sigma)"}
        del Lam, L, S
        torch.cuda.empty_cache()
    a = torch.randn(8192, 8192, device=dev, dtype=torch.float64, generator=g)
    b = torch.randn(8192, 8192, device=dev, dtype=torch.float64, generator=g)
    best = None
    for _ in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.matmul(a, b)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    ref = 2 * 8192 ** 3 / best / 1e12
    for k in out:
        out[k]["frac_of_cublas_dgemm"] = out[k]["tflops"] / ref
    ctx.close()
    print(json.dumps({"profile_chol": out, "cublas_dgemm_tflops": ref}), flush=True)


def run_profile_contract(args):
    """The tensor-core contraction alone at 8192 x 8192 x 4096 (3xTF32 split mode, the mode
    the mixed path uses), twice through cggm_contract: for ncu captures of gemm_tc_kernel."""
    import torch
    import paper_1509_04681_gb300 as cg
    from paper_1509_04681_gb300 import build as pkg_build
    pkg_build.build()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(0)
    M, N, K = 8192, 8192, 4096
    A = torch.randn(M, K, device=dev, generator=g)
    B = torch.randn(N, K, device=dev, generator=g)
    with cg.Context(0) as ctx:
        for _ in range(2):
            C = ctx.cggm_contract(A, B, mode=1)
        torch.cuda.synchronize()
    print(json.dumps({"profile_contract": {"M": M, "N": N, "K": K, "mode": "split",
                                           "c_abs_sum": float(C.abs().sum())}}))


def serve_measure(n_requests, scale, slots, max_iter, rate=20.0):
    """Served regularisation paths: n_requests requests of uneven size (p, q, n log-uniform in
    [500, 8000], [200, 4000], [200, 1000], each divided by `scale`) arriving as a Poisson
    process (`rate` per second), each an 8-point lambda grid from 0.5 down to 0.02 solved with
    warm starts (tol 0.01, at most max_iter Newton iterations per point), admitted by
    device-memory footprint into `slots` concurrent workers whose coordinate passes share
    cooperative launches.  Returns lambda-point solves per second over the makespan and p50 /
    p99 latency (arrival to the last lambda point)."""
    import numpy as np
    import paper_1509_04681_gb300 as cg
    import synth
    lo = lambda v: max(1, int(v / scale))  # noqa: E731
    reqs = synth.serving_requests(n_req=n_requests, rate_per_s=rate, seed=0,
                                  p_range=(lo(500), lo(8000)), q_range=(lo(200), lo(4000)),
                                  n_range=(lo(200), lo(1000)))
    probs = [(r, r.problem()) for r in reqs]
    with cg.Server(0, slots=slots) as srv:
        t0 = time.perf_counter()
        ids = []
        for r, pr in probs:
            wait = r.arrival_s - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            ids.append(srv.submit(pr.X.astype(np.float32), pr.Y.astype(np.float32), r.lambdas,
                                  tol=0.01, max_iter=max_iter, precision=cg.CGGM_MIXED,
                                  want_outputs=False))
        res = [srv.poll(i, wait=True) for i in ids]
        makespan = time.perf_counter() - t0
        stats = srv.stats()
    lat = sorted(r["finish_s"] - r["arrival_s"] for r in res)
    pts = sum(len(r.lambdas) for r, _ in probs)
    return {"value": pts / makespan, "unit": "lambda-point solves/s", "requests": len(res),
            "lambda_points": pts, "makespan_s": makespan,
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "slots": slots,
            "statuses": sorted(set(r["status"] for r in res)),
            "iterations": sum(r["iterations"] for r in res), "pass_batching": stats,
            "workload": (f"{len(res)} requests, sizes log-uniform p in [{lo(500)}, {lo(8000)}], "
                         f"q in [{lo(200)}, {lo(4000)}], n in [{lo(200)}, {lo(1000)}]; 8-point "
                         f"grid 0.5 -> 0.02 with warm starts; Poisson arrivals {rate:g}/s; tol "
                         f"0.01, at most {max_iter} Newton iterations per point; mixed precision")}


def run_serve(args):
    """Served regularisation paths alone (one JSON line with the "serving" object)."""
    from paper_1509_04681_gb300 import build as pkg_build
    pkg_build.build()
    line = {"metric": METRIC, "serving": serve_measure(args.serve_requests, args.serve_scale,
                                                       args.serve_slots, args.serve_max_iter)}
    print(json.dumps(line), flush=True)


def pass_rooflines(info, p, q, mixed, step_sec):
    """Roofline objects of the two coordinate passes over a timed solve: algorithmic bytes
    (10 q words per Lambda coordinate: the dots Sigma_i.U_j, Psi_i.U_j, Psi_j.U_i and the
    updates of U_i, U_j; (2 p + 3 q) words per Theta coordinate: (S_xx)_i . Delta V_j and
    the update of Delta V_i with Sigma_j) over each pass's event-timed seconds."""
    esz = 4 if mixed else 8
    iters = max(1, info["iterations"])
    hbm, src = peaks()
    out = []
    for kname, units, per, ksec in (
            ("lambda_sweep_kernel", info["coords_lambda"], 10 * q,
             info["sec_sweep_lambda"]),
            ("theta_sweep_kernel", info["coords_theta"], 2 * p + 3 * q,
             info["sec_sweep_theta"])):
        kbytes = units * per * esz
        achieved = kbytes / ksec / 1e9 if ksec > 0 else 0.0
        per_unit = (f"10 q x {esz} B per Lambda coordinate" if kname.startswith("lambda")
                    else f"(2 p + 3 q) x {esz} B per Theta coordinate")
        out.append({"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm,
                    "unit": "GB/s", "frac": achieved / hbm,
                    "traffic": profiled_traffic(kname, units / iters),  # per launch
                    "peak_source": src, "algorithmic_bytes": per_unit,
                    "launch_seconds": ksec / iters, "share_of_step": ksec / step_sec})
    return out[0], out[1]


def fp64_leg(ctx, cg, Xd, Yd, pr, p, q, dev, steps, warmup):
    """Newton iterations/s of the double-precision path on the same workload: W iterations
    from Lambda = I, Theta = 0, then K timed ones (CUDA events on the context's stream)."""
    import torch
    L0 = torch.empty((q, q), device=dev, dtype=torch.float64)
    T0 = torch.empty((p, q), device=dev, dtype=torch.float64)
    ctx.cggm_solve_dense(Xd, Yd, pr.lam_L, pr.lam_T, tol=1e-12,
                   opts=cg.make_opts(precision=cg.CGGM_FP64, max_iter=warmup),
                   Lambda_out=L0, Theta_out=T0)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    res = ctx.cggm_solve_dense(Xd, Yd, pr.lam_L, pr.lam_T, tol=1e-12, warm_Lambda=L0, warm_Theta=T0,
                         opts=cg.make_opts(precision=cg.CGGM_FP64, max_iter=steps),
                         Lambda_out=L0, Theta_out=T0)
    ev1.record(stream)
    torch.cuda.synchronize()
    sec = ev0.elapsed_time(ev1) / 1e3
    info = res.info
    it = max(1, info["iterations"])
    rl, rt = pass_rooflines(info, p, q, False, sec)
    return {"value": info["iterations"] / sec, "unit": "Newton iterations/s",
            "steps": info["iterations"], "warmup": warmup, "ms_per_step": 1e3 * sec / it,
            "dtype": "f64",
            "per_iteration": {k: info[k] / it for k in ("sec_products", "sec_sweep_lambda",
                                                          "sec_linesearch", "sec_factor",
                                                          "sec_sweep_theta")},
            "roofline_lambda_pass": rl, "roofline_theta_pass": rt,
            "gpu_launches": info["launches"]}


def run_gap_trace(args):
    """Objective against device time for both precisions on the 5000 x 5000 workload: each
    path runs from Lambda = I, Theta = 0 in chunks of Newton iterations (warm-started from
    the previous chunk in device memory) until its time budget is spent; after each chunk
    f(Lambda, Theta) is evaluated in double precision (cggm_objective, not timed).  f_best
    is the lowest f seen by either path; the gap of an iterate is (f - f_best) / |f_best|
    (f* <= f_best, so true gaps are at least these).  Also the paper's stopping quantity
    (the min-norm subgradient ratio of Section 5.1) at each chunk's last iteration.  Gaps are
    taken against f* extrapolated from the best path's last chunks (Aitken), which lies below
    f_best; both are reported."""
    import numpy as np
    import torch
    import paper_1509_04681_gb300 as cg
    from paper_1509_04681_gb300 import build as pkg_build
    pkg_build.build()
    import synth
    pr = synth.workload(WORKLOAD)
    n, p = pr.X.shape
    q = pr.Y.shape[1]
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    Xd = torch.from_numpy(pr.X_raw).to(dev)
    Yd = torch.from_numpy(pr.Y.astype(np.float32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = cg.Context(0, stream=stream.cuda_stream)
    traces = {}
    budgets = {"fp64": args.gap_fp64 if args.gap_fp64 > 0 else args.gap_trace,
               "mixed": args.gap_trace}
    for name, prec in (("fp64", cg.CGGM_FP64), ("mixed", cg.CGGM_MIXED)):
        L = torch.empty((q, q), device=dev, dtype=torch.float64)
        T = torch.empty((p, q), device=dev, dtype=torch.float64)
        t_dev, its, first = 0.0, 0, True
        rows = []
        with Clocks(0) as clk:
            while t_dev < budgets[name]:
                kw = {} if first else {"warm_Lambda": L, "warm_Theta": T}
                r = ctx.cggm_solve_dense(Xd, Yd, pr.lam_L, pr.lam_T, tol=1e-12,
                                   opts=cg.make_opts(precision=prec, max_iter=args.gap_chunk),
                                   Lambda_out=L, Theta_out=T, **kw)
                first = False
                t_dev += r.info["seconds"]
                its += r.info["iterations"]
                f = ctx.cggm_objective(Xd, Yd, L, T, pr.lam_L, pr.lam_T)
                rows.append({"seconds": t_dev, "iterations": its, "f": f,
                             "subgrad_ratio": r.info["subgrad"] / max(1e-300, r.info["l1norm"]),
                             "m_lambda": r.info["m_lambda"], "m_theta": r.info["m_theta"]})
                print(json.dumps({"trace": name, **rows[-1]}), flush=True)
                if r.status == cg.CGGM_OK:
                    break
        traces[name] = {"rows": rows, "clocks": clk.summary()}
    ctx.close()
    f_best = min(r["f"] for t in traces.values() for r in t["rows"])
    # the method converges linearly near the optimum: Aitken's extrapolation of the best
    # path's last three chunk values estimates f* below f_best
    best_rows = min(traces.values(), key=lambda t: t["rows"][-1]["f"])["rows"]
    f_star = f_best
    if len(best_rows) >= 3:
        f1, f2, f3 = (r["f"] for r in best_rows[-3:])
        d1, d2 = f2 - f1, f3 - f2
        if d1 < 0 and d2 < 0 and abs(d2) < abs(d1):
            f_star = f3 - d2 * d2 / (d2 - d1)
    out = {"gap_trace": {"workload": WORKLOAD, "p": p, "q": q, "n": n, "lambda": pr.lam_L,
                         "budget_s": budgets, "chunk": args.gap_chunk,
                         "f_best": f_best, "f_star_extrapolated": f_star}}
    for name, t in traces.items():
        rows = t["rows"]
        reach = {}
        for g in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
            hit = [r for r in rows if (r["f"] - f_star) / abs(f_star) <= g]
            reach[f"{g:g}"] = ({"seconds": hit[0]["seconds"], "iterations": hit[0]["iterations"]}
                               if hit else None)
        stop = [r for r in rows if r["subgrad_ratio"] < 0.01]
        out["gap_trace"][name] = {
            "seconds": rows[-1]["seconds"], "iterations": rows[-1]["iterations"],
            "f_last": rows[-1]["f"], "gap_last": (rows[-1]["f"] - f_star) / abs(f_star),
            "subgrad_ratio_last": rows[-1]["subgrad_ratio"], "time_to_gap": reach,
            "time_to_paper_stop_0.01": ({"seconds": stop[0]["seconds"],
                                          "iterations": stop[0]["iterations"]} if stop else None),
            "clocks": t["clocks"], "trace": rows}
    print(json.dumps(out), flush=True)


def run_large(args):
    """The 40000-input, 20000-output workload (n = 500, random degree-4 Lambda, Theta with 20
    nonzeros per column, X standardised genotypes stored in bf16, lambda 0.1) end to end in the
    mixed path: K Newton iterations from Lambda = I, Theta = 0 through cggm_solve_dense with
    inputs and outputs in device memory, then a KKT check of the returned point from
    cggm_grad (double precision): the min-norm subgradient of every Lambda entry and of a
    random sample of 10^6 Theta entries (Section 5.1's stopping quantity, entry by entry)."""
    import numpy as np
    import torch
    import paper_1509_04681_gb300 as cg
    from paper_1509_04681_gb300 import build as pkg_build
    pkg_build.build()
    import synth
    t0 = time.perf_counter()
    pr = synth.workload("rand4-geno-p40000-q20000-n500")
    t_gen = time.perf_counter() - t0
    n, p = pr.X.shape
    q = pr.Y.shape[1]
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    Xd = torch.from_numpy(pr.X).to(dev).to(torch.bfloat16)
    Yd = torch.from_numpy(pr.Y.astype(np.float32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = cg.Context(0, stream=stream.cuda_stream)
    L = torch.empty((q, q), device=dev, dtype=torch.float64)
    T = torch.empty((p, q), device=dev, dtype=torch.float64)
    with Clocks(0) as clk:
        r = ctx.cggm_solve_dense(Xd, Yd, pr.lam_L, pr.lam_T, tol=0.01,
                                 opts=cg.make_opts(precision=cg.CGGM_MIXED, max_iter=args.large),
                                 Lambda_out=L, Theta_out=T)
    info = r.info
    it = max(1, info["iterations"])
    f = ctx.cggm_objective(Xd, Yd, L, T, pr.lam_L, pr.lam_T)
    # KKT residual of the returned point (the checks use torch on the device; the gradients
    # come from the library)
    GL = torch.empty((q, q), device=dev, dtype=torch.float64)
    GT = torch.empty((p, q), device=dev, dtype=torch.float64)
    lib = cg.cggm._lib()
    Xa = cg.cggm._Arr(Xd, "bf16")
    st = lib.cggm_grad(ctx._h, Xa.ptr, cg.CGGM_BF16, Yd.data_ptr(), cg.CGGM_F32, n, p, q,
                       L.data_ptr(), T.data_ptr(), GL.data_ptr(), GT.data_ptr())
    assert st == 0, st
    torch.cuda.synchronize()

    def subgrad(G, P, lam):
        nz = P != 0
        s_nz = (G + lam * torch.sign(P)).abs()
        s_z = torch.clamp(G.abs() - lam, min=0.0)
        return torch.where(nz, s_nz, s_z)

    sl = subgrad(GL, L, pr.lam_L)
    g = torch.Generator(device=dev).manual_seed(0)
    idx = torch.randint(0, p * q, (1_000_000,), device=dev, generator=g)
    st_ = subgrad(GT.reshape(-1)[idx], T.reshape(-1)[idx], pr.lam_T)
    ratio = (sl.sum() + st_.sum() * (p * q / idx.numel())) / (L.abs().sum() + T.abs().sum())
    out = {"large": {
        "workload": "rand4-geno-p40000-q20000-n500", "p": p, "q": q, "n": n,
        "lambda": pr.lam_L, "x": "standardised genotypes in bf16", "y": "fp32",
        "precision": "mixed", "iterations": info["iterations"], "status": r.status,
        "seconds": info["seconds"], "seconds_per_iteration": info["seconds"] / it,
        "per_iteration": {k: info[k] / it for k in ("sec_products", "sec_active",
                                                      "sec_sweep_lambda", "sec_linesearch",
                                                      "sec_factor", "sec_sweep_theta")},
        "ls_trials": info["ls_trials"], "m_lambda_last": info["m_lambda"],
        "m_theta_last": info["m_theta"], "f": f,
        "subgrad_ratio_at_last_check": info["subgrad"] / max(1e-300, info["l1norm"]),
        "kkt": {"lambda_max_subgrad": float(sl.max()), "lambda_subgrad_l1": float(sl.sum()),
                "theta_sample": int(idx.numel()),
                "theta_sample_max_subgrad": float(st_.max()),
                "ratio_estimate": float(ratio)},
        "nnz_lambda": int((L != 0).sum()), "nnz_theta": int((T != 0).sum()),
        "generate_s": t_gen, "clocks": clk.summary(), "gpu_launches": info["launches"]}}
    ctx.close()
    print(json.dumps(out), flush=True)


def run_cuda(args):
    import numpy as np
    import torch
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1509_04681_gb300 as cg
    from paper_1509_04681_gb300 import build as pkg_build
    pkg_build.build()
    import synth

    pr = synth.workload(WORKLOAD, seed=replica_seed(rank))  # independent replica per rank
    n, p = pr.X.shape
    q = pr.Y.shape[1]
    # X as stored: int8 genotype counts, standardised by the library on the device; Y fp32
    Y32 = pr.Y.astype(np.float32)
    Xd = torch.from_numpy(pr.X_raw).to(dev)
    Yd = torch.from_numpy(Y32).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = cg.Context(local, stream=stream.cuda_stream)
    prec = cg.CGGM_MIXED if args.precision == "mixed" else cg.CGGM_FP64
    L0 = torch.empty((q, q), device=dev, dtype=torch.float64)
    T0 = torch.empty((p, q), device=dev, dtype=torch.float64)
    L1 = torch.empty_like(L0)
    T1 = torch.empty_like(T0)

    # warm-up: W Newton iterations from Lambda = I, Theta = 0
    ctx.cggm_solve_dense(Xd, Yd, pr.lam_L, pr.lam_T, tol=1e-12,
                   opts=cg.make_opts(precision=prec, max_iter=args.warmup,
                                     sweep_batch=args.sweep_batch),
                   Lambda_out=L0, Theta_out=T0)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        res = ctx.cggm_solve_dense(Xd, Yd, pr.lam_L, pr.lam_T, tol=1e-12, warm_Lambda=L0,
                             warm_Theta=T0,
                             opts=cg.make_opts(precision=prec, max_iter=args.steps,
                                               sweep_batch=args.sweep_batch),
                             Lambda_out=L1, Theta_out=T1)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    sec = ev0.elapsed_time(ev1) / 1e3
    sec_max = max_over_ranks(sec, world)
    info = res.info
    iters = info["iterations"]
    value = job_rate(iters, sec_max, world)
    clocks = clk.summary()

    # roofline of the dominant kernel (the coordinate pass with the larger time) and of the
    # other pass beside it
    rl, rt = pass_rooflines(info, p, q, prec == cg.CGGM_MIXED, sec)
    roof, roof_other = (rl, rt) if info["sec_sweep_lambda"] >= info["sec_sweep_theta"] else (rt, rl)

    line = {"metric": METRIC, "value": value, "unit": "Newton iterations/s",
            "n_gpus": world, "steps": iters, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec_max / max(1, iters), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 caches + f64 scalars" if prec == cg.CGGM_MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "p": p, "q": q, "n": n, "lambda": pr.lam_L,
                       "precision": args.precision, "parallelism": "replicas",
                       "x": "genotype Binomial(2, MAF~U(0.05,0.5)) as int8 counts, standardised on the device", "y": "fp32",
                       "network": "chain (1.0 / 0.4)", "theta_nnz_per_col": 10,
                       "seed": 0, "l2": "working set (Sigma, Psi, U, S_xx, Delta V: "
                       "~100 MB each) larger than L2; no flush"},
            "roofline": roof, "roofline_other_pass": roof_other, "clocks": clocks,
            "gpu_launches": info["launches"],
            "per_iteration": {"active_lambda_last": info["m_lambda"],
                              "active_theta_last": info["m_theta"],
                              "sec_products": info["sec_products"] / max(1, iters),
                              "sec_sweep_lambda": info["sec_sweep_lambda"] / max(1, iters),
                              "sec_linesearch": info["sec_linesearch"] / max(1, iters),
                              "sec_factor": info["sec_factor"] / max(1, iters),
                              "sec_sweep_theta": info["sec_sweep_theta"] / max(1, iters),
                              "coords_per_s": (info["coords_lambda"] + info["coords_theta"]) /
                              max(1e-9, info["sec_sweep_lambda"] + info["sec_sweep_theta"])},
            "reported_as": "Newton iterations/s on the 5000 x 5000 workload (mixed; fp64 beside "
                           "it); time-to-gap on the 200 x 100 workload (time_to_gap); the "
                           "5000 x 5000 time-to-gap trace is bench.py --gap-trace; served "
                           "lambda-point solves/s with p50/p99 (serving)"}

    # end to end through the C ABI from host buffers (copies inside the timed region)
    if not args.no_e2e:
        # pinned host buffers: inputs, warm start and the returned Lambda, Theta
        Xh = torch.from_numpy(pr.X_raw).pin_memory()
        Yh = torch.from_numpy(Y32).pin_memory()
        Lh, Th_ = L0.cpu().pin_memory(), T0.cpu().pin_memory()
        Lo = torch.empty((q, q), dtype=torch.float64).pin_memory()
        To = torch.empty((p, q), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        r2 = ctx.cggm_solve_dense(Xh, Yh, pr.lam_L, pr.lam_T, tol=1e-12, warm_Lambda=Lh,
                            warm_Theta=Th_, Lambda_out=Lo, Theta_out=To,
                            opts=cg.make_opts(precision=prec, max_iter=args.steps))
        torch.cuda.synchronize()
        e2e_sec = max_over_ranks(time.perf_counter() - t0, world)
        it2 = r2.info["iterations"]
        h2d = Xh.numel() * Xh.element_size() + Yh.numel() * Yh.element_size() + \
            (Lh.numel() + Th_.numel()) * 8
        line["e2e"] = {"value": world * it2 / e2e_sec, "unit": "Newton iterations/s",
                       "h2d_bytes_per_step": int(h2d / max(1, it2)),
                       "d2h_bytes_per_step": int((Lo.numel() + To.numel()) * 8 / max(1, it2))}

    if rank == 0 and world == 1 and not args.no_fp64:
        line["fp64"] = fp64_leg(ctx, cg, Xd, Yd, pr, p, q, dev, min(args.steps, 5), 3)
        line["mixed_over_fp64_iterations_per_s"] = value / line["fp64"]["value"]
    if rank == 0 and world == 1 and not args.no_serve:
        sv = serve_measure(args.line_serve_requests, 1.0, args.serve_slots,
                           args.line_serve_max_iter)
        sv["trimmed"] = (f"{args.line_serve_requests} of the 64 requests of the served "
                         f"workload, at most {args.line_serve_max_iter} iterations per lambda "
                         f"point, to keep the benchmark within minutes; request sizes in full")
        line["serving"] = sv
    if rank == 0 and world == 1 and not args.no_ttg:
        small = synth.workload(SMALL)
        line["time_to_gap"] = time_to_gap(ctx, cg, small, torch)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_rate(pr)
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ttg", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--sweep-batch", type=int, default=0,
                    help="coordinates per blocked Gauss-Seidel batch (0: the library default)")
    ap.add_argument("--gap-fp64", type=float, default=0.0,
                    help="device-time budget of the FP64 path in --gap-trace (default: the same)")
    ap.add_argument("--gap-trace", type=float, default=0.0,
                    help="seconds of device time per precision: record f against time on the "
                         "5000 x 5000 workload instead of the default line")
    ap.add_argument("--gap-chunk", type=int, default=10)
    ap.add_argument("--large", type=int, default=0,
                    help="Newton iterations on the 40000 x 20000 workload instead of the "
                         "default line")
    ap.add_argument("--serve", action="store_true",
                    help="served lambda paths (Poisson arrivals) instead of the default line")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-scale", type=float, default=1.0,
                    help="divide the request size ranges by this factor")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-max-iter", type=int, default=100)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--line-serve-requests", type=int, default=8,
                    help="served requests measured within the default line")
    ap.add_argument("--line-serve-max-iter", type=int, default=8)
    ap.add_argument("--profile-sweep", action="store_true",
                    help="run only a bounded Lambda pass at q=5000 (for ncu captures)")
    ap.add_argument("--profile-theta", action="store_true",
                    help="run only a bounded Theta pass at p = q = 5000 (for ncu captures)")
    ap.add_argument("--profile-chol", action="store_true",
                    help="time the FP64 Cholesky and inverse against cuBLAS double GEMM")
    ap.add_argument("--profile-contract", action="store_true",
                    help="run only the tensor-core contraction at 8192^2 x 4096 (for ncu captures)")
    args = ap.parse_args()
    if args.profile_sweep:
        run_profile_sweep(args)
    elif args.profile_theta:
        run_profile_theta(args)
    elif args.profile_chol:
        run_profile_chol(args)
    elif args.profile_contract:
        run_profile_contract(args)
    elif args.gap_trace > 0:
        run_gap_trace(args)
    elif args.large > 0:
        run_large(args)
    elif args.serve:
        run_serve(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
