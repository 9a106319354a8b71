#!/usr/bin/env python
"""QP solves per second of the GPU interior point method on the RT-shaped workload.

Workload (the configuration the headline metric is quoted on): an RT-shaped convex QP with a
dose-like matrix D of V = 200000 voxels x n = 50000 beam spots (0.5 % density, lognormal
values, contiguous spot bands per voxel row), H = D^T W D + 1e-4 I applied matrix-free,
c = -D^T W d_presc, A = the 20000 D rows of organ voxels with b = 0.6, 0 <= x <= 5; FP64.
Synthetic data from paper_2405_03584_gb300.workloads.rt_qp (seed 1).

A step is one complete solve (start point, every IPM iteration with its PCG solve, to a
relative KKT residual <= 1e-6) with the QP already resident in HBM; the operator's working
set (about 1.2 GB) is larger than L2, so no explicit flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With torchrun (N > 1) every rank solves its own replica (the path does not shard a single
QP); the value is the whole-job solves/s over the max-over-ranks time.  --impl reference
times the CPU FP64 oracle (dense Cholesky IPM) on the host cores instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QP solves/sec & p50/p99 latency at rel. KKT <=1e-6; PCG SpMV HBM GB/s"
N_FULL, SEED, TOL = 50_000, 1, 1e-6
WORKLOAD = ("RT-shaped QP: D 200000 voxels x 50000 spots, 0.5% banded lognormal, H = D^T W D + 1e-4 I "
            "matrix-free, A = 20000 organ rows (b = 0.6), 0 <= x <= 5, FP64, seed 1")
SAMPLE_SIZES = (2000, 4000, 6000)   # oracle samples: the same generator at these n (V = 4n)
FALLBACK_HBM_GBS = 6800.0
FP64_NOMINAL_TFLOPS = 1.25      # GB300 FP64 (non-tensor) nominal rate


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(value, device="cuda"):
    """The largest of one float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, world, max_ms):
    """Whole-job rate of independent replicas: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1000.0)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d["hbm_gbs"]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def _cores_used():
    try:
        from threadpoolctl import threadpool_info
        th = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if th:
            return int(max(th))
    except Exception:
        pass
    return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def operator_source_hash():
    """Hash of the library's device sources (every csrc file): an ncu figure recorded under
    another hash was taken on other kernels and is not reported."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2405_03584_gb300", "csrc", "*"))):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(os.path.basename(f).encode())
            h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel, lanes):
    """DRAM bytes per launch of `kernel` (with `lanes` lanes per row) from the committed ncu
    summary, if it was taken on the current operator source (recorded hash matches); else None."""
    summ = os.path.join(ROOT, "profiles", "pcg_operator_rt_c1.md")
    if not os.path.exists(summ):
        return None
    txt = open(summ).read()
    if ("source_hash: " + operator_source_hash()) not in txt:
        return None
    key = "traffic_per_launch_bytes[%s<%d>]:" % (kernel, lanes)
    for line in txt.splitlines():
        if line.strip().startswith(key):
            return float(line.split(":")[1])
    return None


def _oracle_time(n):
    """The CPU oracle as it stands: one full solve of the same generator at n variables
    (V = 4n voxels, m = n/2.5 organ rows), wall-clock seconds of the oracle alone."""
    from oracle import ipm as O
    from paper_2405_03584_gb300 import workloads as W
    p = W.rt_qp(n=n, seed=SEED)
    t0 = time.perf_counter()
    qp = O.from_rt(p)
    it, info = O.solve(qp, tol=TOL)
    t = time.perf_counter() - t0
    return dict(n=n, seconds=t, ipm_iters=info.iterations, status=info.status)


def power_law(points):
    """Least-squares fit of log t = log a + b log n over measured (n, seconds) points; with
    one size only the exponent of the oracle's dense Cholesky steps (3) is assumed."""
    ns = np.array([float(q[0]) for q in points])
    ts = np.array([float(q[1]) for q in points])
    if len(set(ns.tolist())) < 2:
        b = 3.0
        a = float(np.exp(np.mean(np.log(ts) - b * np.log(ns))))
        return a, b, False
    b, la = np.polyfit(np.log(ns), np.log(ts), 1)
    return float(np.exp(la)), float(b), True


def _cpu_law(points):
    """Full-size oracle rate from the measured points and its description."""
    a, b, fitted = power_law([(q["n"], q["seconds"]) for q in points])
    t_full = a * N_FULL ** b
    by_n = {}
    for q in points:
        by_n.setdefault(q["n"], []).append(q["seconds"])
    pts = ", ".join("n=%d: %.2f s" % (n, statistics.mean(v)) for n, v in sorted(by_n.items()))
    law = ("t(n) = %.3g * n^%.2f s, %s over the measured sizes (%s)" %
           (a, b, "least-squares fit" if fitted else "exponent 3 assumed (one size)", pts))
    return 1.0 / t_full, law, {"coef": a, "exponent": b, "fitted": fitted, "t_full_s": t_full,
                                "points": [[q["n"], q["seconds"], q["ipm_iters"]] for q in points]}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    cores = _cores_used()
    sizes = args.sample_sizes
    pts, step_s = [], []
    for k in range(args.warmup + args.steps):
        n = sizes[k % len(sizes)]
        r = _oracle_time(n)
        if k >= args.warmup:
            pts.append(r)
            step_s.append(r["seconds"])
    value, law, fit = _cpu_law(pts)
    sample = ("oracle (dense-Cholesky FP64 IPM) full solves of the same RT generator at n in %s (V = 4n, "
              "m = n/2.5), one size per step; full-size rate from %s" % (list(sizes), law))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(step_s),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "l2": "host run",
                      "step": "one oracle solve at a sample size (ms_per_step is the measured mean); value is "
                              "the full-size rate from the fitted law"},
           "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample,
                            "fit": fit},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def _operator_opts(args):
    """Operator arithmetic and rows format given on the command line (else the preset's)."""
    o = {}
    if args.op_arith:
        o["op_arith"] = args.op_arith
    if args.rows_format:
        o["rows_format"] = args.rows_format
    if args.rows_stage is not None:
        o["rows_stage"] = args.rows_stage
    if args.cols_format is not None:
        o["cols_format"] = args.cols_format
    if args.refine_eta is not None:
        o["refine_eta"] = args.refine_eta
    if args.refine_mode is not None:
        o["refine_mode"] = args.refine_mode
    return o


def run_operator_only(args):
    """Small capture target for profilers: the RT workload (or --bfgs), three IPM iterations,
    then the two operator passes three times each (ipm_profile_operator), in the storage of
    --storage."""
    import torch
    from paper_2405_03584_gb300 import build, ipm, workloads as W
    torch.cuda.set_device(0)
    build.build()
    lr, lc = (int(v) for v in args.lanes.split(","))
    s = ipm.Solver(tol_kkt=TOL, precond="jacobi_lr", max_ipm=3, lanes_rows=lr, lanes_cols=lc,
                   storage=args.storage, **_operator_opts(args))
    if args.bfgs:
        s.set_qp_bfgs(_bfgs_problem(args.bfgs))
    else:
        s.set_qp_rt(W.rt_qp(n=N_FULL, seed=SEED))
    s.solve()
    out = s.profile_operator(reps=3)
    out["lanes"] = [s.get()["info"]["lanes_rows"], s.get()["info"]["lanes_cols"]]
    out["operator_source_hash"] = operator_source_hash()
    print(json.dumps(out), flush=True)
    s.close()
    return 0


def run_batch(args):
    """The uneven batch: 64 RT-shaped QPs (n ~ U[2000, 40000], V = 4n, density U[0.2%, 1%],
    n/2 constraint rows), FP32 operator storage with FP64 refinement and reductions, schedules
    autotuned per instance, all solved by one graph launch; against the plain FP64 solver
    running the same QPs one after another.  Prints one JSON line."""
    import torch
    from paper_2405_03584_gb300 import build, ipm, workloads as W
    torch.cuda.set_device(0)
    build.build()
    count = args.batch_count
    scale = args.batch_scale
    t0 = time.perf_counter()
    probs = W.rt_batch(count, seed=3, scale=scale)
    t_gen = time.perf_counter() - t0
    nnz = [int(p["D_indptr"][-1]) for p in probs]
    t0 = time.perf_counter()
    solvers = []
    for p in probs:
        sv = ipm.Solver(tol_kkt=TOL, precond="jacobi_lr", storage="f32", autotune=1)
        sv.set_qp_rt(p)
        solvers.append(sv)
    t_load = time.perf_counter() - t0
    b = ipm.Batch(solvers)
    for _ in range(args.warmup):
        st = b.solve()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(args.steps):
        st = b.solve()
    ev[1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    infos = [sv.get()["info"] for sv in solvers]
    b.close()
    for sv in solvers:
        sv.close()
    # baseline: the plain FP64 solver, one QP at a time
    seq_ms, seq_status = 0.0, []
    for p in probs:
        sv = ipm.Solver(tol_kkt=TOL, precond="jacobi_lr")
        sv.set_qp_rt(p)
        sv.solve()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        seq_status.append(sv.solve())
        e1.record(stream)
        torch.cuda.synchronize()
        seq_ms += e0.elapsed_time(e1)
        sv.close()
    out = {"mode": "batch", "metric": "QP solves/sec (64-QP uneven batch, rel. KKT <= 1e-6)",
           "value": count / (ms / 1000.0), "unit": "solves/s", "ms_per_batch": ms, "steps": args.steps,
           "warmup": args.warmup, "dtype": "f32 storage, f64 refinement and reductions",
           "config": {"count": count, "scale": scale, "n": [p["n"] for p in probs], "nnz_total": int(sum(nnz)),
                      "generator": "workloads.rt_batch(64, seed=3)"},
           "status": [int(x) for x in st], "max_rel_kkt_device": max(i["rel_kkt"] for i in infos),
           "ipm_iters": [i["ipm_iters"] for i in infos], "lanes": [[i["lanes_rows"], i["lanes_cols"]] for i in infos],
           "baseline_sequential_f64": {"value": count / (seq_ms / 1000.0), "unit": "solves/s", "ms_total": seq_ms,
                                       "status": [int(x) for x in seq_status]},
           "speedup_vs_sequential_f64": seq_ms / ms, "setup_s": {"generate": t_gen, "load": t_load},
           "clocks": clk}
    print(json.dumps(out), flush=True)
    return 0


def _serve_once(plans, reqs, horizon, **kw):
    from paper_2405_03584_gb300 import serve
    srv = serve.Server(plans, **kw)
    # one solve per plan handle before the clock starts (graph capture and instantiation)
    for sl in srv.plan_slot:
        sl.solver.solve(stream=sl.sid)
    t0 = time.perf_counter()
    qrec, rrec = srv.run(reqs)
    wall = time.perf_counter() - t0
    stats = dict(srv.stats)
    srv.close()
    summ = serve.latency_summary(qrec, rrec, horizon, stats["busy_s"])
    summ.update(stats)
    summ["wall_s"] = wall
    return summ, qrec


def run_serve(args):
    """The serving workload: Poisson arrivals (lambda req/s) over a fixed horizon; 30 % of the
    requests are chains of 20 related QPs (weights and cost perturbed by 1 % per step, each
    warm-started from the previous solution), the rest single QPs; plans from the uneven
    64-QP size mix; BF16 operator storage with FP64 refinement; admission against a 120 GB
    HBM ledger with up to --serve-inflight solves in flight.  The baseline serves the same
    stream with the plain FP64 solver, one solve at a time, cold starts.  One JSON line."""
    import torch
    from paper_2405_03584_gb300 import build, workloads as W
    torch.cuda.set_device(0)
    build.build()
    t0 = time.perf_counter()
    plans = W.rt_batch(64, seed=3, scale=args.batch_scale)
    t_gen = time.perf_counter() - t0
    reqs = W.serving_stream(horizon=args.serve_horizon, lam=args.serve_lambda, chain_frac=0.3, chain_len=20,
                            n_plans=len(plans), seed=4)
    common = dict(budget_bytes=120e9, tol_kkt=TOL, precond="jacobi_lr")
    t0 = time.perf_counter()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ours, qrec = _serve_once(plans, reqs, args.serve_horizon, max_inflight=args.serve_inflight, warm=True,
                             keep_x=False, storage="bf16", **common)
    clk = clocks.stop()
    t_ours = time.perf_counter() - t0
    base = None
    if not args.serve_no_baseline:
        t0 = time.perf_counter()
        base, _ = _serve_once(plans, reqs, args.serve_horizon, max_inflight=1, warm=False, keep_x=False,
                              storage="f64", **common)
        base["run_s"] = time.perf_counter() - t0
    out = {"mode": "serve", "metric": "QP solves/sec & p50/p99 latency at rel. KKT <=1e-6 (serving stream)",
           "value": ours["solves_per_s"], "unit": "solves/s", "p50_ms": ours["p50_ms"], "p99_ms": ours["p99_ms"],
           "dtype": "bf16 storage, f32 accumulate, f64 refinement and reductions",
           "config": {"lambda": args.serve_lambda, "horizon_s": args.serve_horizon, "requests": len(reqs),
                      "qps": sum(r["steps"] for r in reqs), "chain_frac": 0.3, "chain_len": 20,
                      "plans": "workloads.rt_batch(64, seed=3, scale=%g)" % args.batch_scale,
                      "stream": "workloads.serving_stream(seed=4)", "max_inflight": args.serve_inflight,
                      "budget_bytes": 120e9},
           "ours": ours,
           "baseline_f64_one_at_a_time": base,
           "setup_s": {"generate": t_gen, "serve_run": t_ours}, "clocks": clk}
    if base:
        out["speedup_solves_per_s"] = ours["solves_per_s"] / base["solves_per_s"]
        out["p99_ratio_baseline_over_ours"] = base["p99_ms"] / ours["p99_ms"]
    print(json.dumps(out), flush=True)
    return 0


def _bfgs_problem(case):
    from paper_2405_03584_gb300 import workloads as W
    if case == "proton":
        return W.bfgs_qp(n=77373, k=100, seed=5)
    return W.bfgs_qp(n=13425, k=33, m_ub=52867, m_lb=15751, density=0.01, seed=6, c_mode="target",
                     ub_fac=1.1, lb_fac=0.9)


def run_bfgs(args):
    """The paper's quasi-Newton Hessian regime (Section 3.3, eq:bfgs_hessian; Table 1 sizes):
    proton n = 77373, bounds only, 2k = 200 update columns; VMAT n = 13425 with 52867 upper
    and 15751 lower sparse constraint rows, 2k = 66.  Synthetic (workloads.bfgs_qp).  Steps =
    complete FP64 solves to rel. KKT <= 1e-6; roofline of the slower operator half."""
    import torch
    from paper_2405_03584_gb300 import build, ipm, workloads as W
    torch.cuda.set_device(0)
    build.build()
    p = _bfgs_problem(args.bfgs)
    s = ipm.Solver(tol_kkt=TOL, precond=args.precond or "jacobi_lr", storage=args.storage,
                   stiff_max=1024 if args.bfgs == "vmat" else 256)
    s.set_qp_bfgs(p)
    for _ in range(args.warmup):
        s.solve()
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    torch.cuda.synchronize()
    sts, infos = [], []
    for k in range(args.steps):
        evs[k][0].record(stream)
        sts.append(s.solve())
        evs[k][1].record(stream)
        infos.append(s.get()["info"])
    torch.cuda.synchronize()
    clk = clocks.stop()
    lat = [a.elapsed_time(b) for a, b in evs]
    total = evs[0][0].elapsed_time(evs[-1][1])
    prof = s.profile_operator(reps=20)
    key = "rows" if prof["ms_rows"] >= prof["ms_cols"] else "cols"
    peak, peak_kind = _peaks()
    ach = prof["bytes_" + key] / (prof["ms_" + key] / 1000.0) / 1e9
    other = "cols" if key == "rows" else "rows"
    roof = {"bound": "hbm", "kernel": ("U^T p pass (k_lr_part + k_op_rows)" if key == "rows"
                                       else "column pass (k_op_cols with U (W t))"),
            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
            "peak_kind": peak_kind + " hbm_gbs", "algorithmic_bytes": prof["bytes_" + key],
            "ms_per_launch": prof["ms_" + key],
            "fp64_tflops": prof["flops_" + key] / (prof["ms_" + key] / 1000.0) / 1e12,
            "other_half": {"ms": prof["ms_" + other],
                           "gbs": prof["bytes_" + other] / (prof["ms_" + other] / 1000.0) / 1e9}}
    s.close()
    res = {"mode": "bfgs", "metric": "QP solves/sec at rel. KKT <= 1e-6 (quasi-Newton Hessian, %s shape)" % args.bfgs,
           "value": args.steps / (total / 1000.0), "unit": "solves/s", "ms_per_step": total / args.steps,
           "steps": args.steps, "warmup": args.warmup, "dtype": "f64" if args.storage == "f64" else args.storage,
           "config": {"workload": args.bfgs, "n": p["n"], "m": p["m"], "u_cols": int(p["U"].shape[1]),
                      "nnz_A": int(p["A_indptr"][-1]) if p["m"] else 0,
                      "generator": "workloads.bfgs_qp (synthetic; the paper's RayStation exports are not available)"},
           "latency_ms": {"p50": statistics.median(lat), "max": max(lat)},
           "solve": {"status": [int(x) for x in sts], "ipm_iters": [i["ipm_iters"] for i in infos],
                     "cg_iters": [i["cg_iters"] for i in infos], "rel_kkt_device": infos[-1]["rel_kkt"]},
           "gpu_launches": int(sum(i["kernel_launches"] for i in infos)), "roofline": roof, "clocks": clk}
    print(json.dumps(res), flush=True)
    return 0


def run_sqp(args):
    """SQP outer loop (Sections 3.2-3.3) on a synthetic dose objective (workloads.sqp_problem:
    the RT generator's D, one-sided quadratic under/overdose penalties, hard organ limits):
    QP sub-problems with the quasi-Newton Hessian on the GPU, warm-started, against the same
    loop with cold starts.  One JSON line."""
    import torch
    import scipy.sparse as sp
    from paper_2405_03584_gb300 import build, ipm, sqp, workloads as W
    torch.cuda.set_device(0)
    build.build()
    p = W.sqp_problem(n=args.sqp_n, density=0.005, seed=7)
    D = sp.csr_matrix((p["D_data"], p["D_indices"], p["D_indptr"]), shape=(p["V"], p["n"]))
    A = D[p["a_rows"]]
    runs = {}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for warm in (True, False):
        obj = sqp.DoseObjective(D, p["target"], p["presc"], p["organ"], p["soft_max"], p["w_target"], p["w_organ"])
        with ipm.Solver(tol_kkt=TOL, precond="jacobi_lr", u_cap=200, stiff_max=1024) as s:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = sqp.sqp_solve(obj, A, p["b"], p["l"], p["u"], np.zeros(p["n"]), s, max_iter=args.sqp_iters,
                                tol=1e-4, u_cap=200, warm=warm)
            wall = time.perf_counter() - t0
        h = res.history
        runs["warm" if warm else "cold"] = {
            "converged": res.converged, "sqp_iterations": res.iterations, "f": res.f, "wall_s": wall,
            "qp_s_total": sum(r["qp_s"] for r in h), "qp_ms_mean": 1000 * float(np.mean([r["qp_s"] for r in h])),
            "qp_ipm_iters_first": h[0]["qp_ipm_iters"],
            "qp_ipm_iters_mean_after_first": float(np.mean([r["qp_ipm_iters"] for r in h[1:]])) if len(h) > 1 else None,
            "qp_cg_iters_mean": float(np.mean([r["qp_cg_iters"] for r in h])),
            "max_u_cols": max(r["u_cols"] for r in h), "qp_not_ok": int(sum(r["qp_status"] != 0 for r in h)), "qp_cold_retries": int(sum(r.get("qp_cold_retry", False) for r in h)),
            "objective_evals": obj.evals}
    clk = clocks.stop()
    w, c = runs["warm"], runs["cold"]
    out = {"mode": "sqp", "clocks": clk, "metric": "QP sub-problems solved per second inside the SQP loop (rel. KKT <= 1e-6)",
           "value": w["sqp_iterations"] / w["qp_s_total"], "unit": "QP/s", "dtype": "f64",
           "config": {"n": p["n"], "V": p["V"], "m": int(p["a_rows"].size), "nnz_D": int(p["D_indptr"][-1]),
                      "u_cap": 200, "sqp_tol": 1e-4,
                      "generator": "workloads.sqp_problem(seed=7) (synthetic dose objective)"},
           "warm": w, "cold": c,
           "qp_time_ratio_cold_over_warm": c["qp_s_total"] / w["qp_s_total"] if w["qp_s_total"] else None}
    print(json.dumps(out), flush=True)
    return 0


def run_dense(args):
    """The dense QP (n = 500, m = 1000, seed 0, tol 1e-8; H = Q Lambda Q^T): FP64 solves with
    the DENSE preconditioner (the condensed matrix formed and factored on the device once per
    IPM iteration).  At about 10 MB per operator apply this case is L2- and launch-latency
    bound, so it reports us per IPM and per PCG iteration rather than HBM bandwidth; beside it
    the oracle's own solve of the same QP on the host cores."""
    import torch
    from paper_2405_03584_gb300 import build, ipm, workloads as W
    from oracle import ipm as O          # the cpu_baseline leg only
    torch.cuda.set_device(0)
    build.build()
    p = W.dense_qp(n=500, m=1000, seed=0)
    s = ipm.Solver(tol_kkt=1e-8, use_graphs=0 if args.no_graphs else 1, autotune=args.dense_autotune)
    s.set_qp_dense(p["H"], p["c"], p["A"], p["b"], p["l"], p["u"])
    for _ in range(args.warmup):
        s.solve()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    torch.cuda.synchronize()
    e0.record(stream)
    sts = [s.solve() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    out = s.get()
    info = out["info"]
    s.close()
    cpu = None
    if not args.no_cpu_baseline:
        qp = O.from_dense(p)
        O.solve(qp, tol=1e-8)                     # warm-up (BLAS threads, page faults)
        t_or = []
        for _ in range(3):
            t0 = time.perf_counter()
            ref, rinfo = O.solve(qp, tol=1e-8)
            t_or.append(time.perf_counter() - t0)
        cpu = {"value": 1.0 / min(t_or), "unit": "solves/s", "cores": _cores_used(), "kind": "oracle",
               "sample": "the whole oracle solve of the same QP (%d IPM iterations), best of 3 after a warm-up "
                         "solve" % rinfo.iterations}
    res = {"mode": "dense", "metric": "QP solves/sec at rel. KKT <= 1e-8 (dense QP)", "value": 1000.0 / ms,
           "unit": "solves/s", "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup, "dtype": "f64",
           "config": {"workload": "dense QP n=500, m=1000, seed 0 (workloads.dense_qp)", "precond": "dense",
                      "autotune": args.dense_autotune},
           "status": [int(x) for x in sts], "ipm_iters": info["ipm_iters"], "cg_iters": info["cg_iters"],
           "us_per_ipm_iter": 1000.0 * ms / max(info["ipm_iters"], 1),
           "us_per_pcg_iter_upper_bound": 1000.0 * ms / max(info["cg_iters"], 1),
           "rel_kkt_device": info["rel_kkt"],
           "gpu_launches": int(info["kernel_launches"]), "clocks": clk, "cpu_baseline": cpu}
    print(json.dumps(res), flush=True)
    return 0


def run_two_sided(args):
    """The RT workload with the paper's two-sided rows (Section 4: l_A <= A x <= u_A, stacked
    as B = [A; -A]): the 20000 organ rows keep their upper limit and dose windows
    (1 -/+ 0.2) D x_f around a strictly feasible x_f are added on --window-rows targets and as
    many other voxels, 1/8 of them lower-only (workloads.rt_two_sided).  Nearly every window
    binds (the cost pulls target doses far above the window and the others to zero), so the
    stiff-row correction is widened to 1024 rows; with thousands of binding rows it cannot
    cover them and PCG runs to its limits.  Solves/s at rel. KKT <= 1e-6 beside the one-sided
    workload solved with the same options (the cost of the stacked rows)."""
    import torch
    from paper_2405_03584_gb300 import build, ipm, workloads as W
    torch.cuda.set_device(0)
    build.build()
    base = W.rt_qp(n=N_FULL, seed=SEED)
    two = W.rt_two_sided(base, n_window=args.window_rows)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    res = {}
    for name, q in (("two_sided", two), ("one_sided", base)):
        s = ipm.Solver(tol_kkt=TOL, precond="jacobi_lr", autotune=1, storage=args.storage, stiff_max=1024)
        s.set_qp(q["n"], q["m"], q["c"], q["b"], q["l"], q["u"], h0=q["h0"],
                 F=(q["D_indptr"], q["D_indices"], q["D_data"]), f_w=q["w"], a_rows=q["a_rows"], bl=q.get("bl"))
        for _ in range(args.warmup):
            s.solve()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sts = [s.solve() for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out = s.get()
        info = out["info"]
        y = out["y"][base["m"]:]
        res[name] = {"solves_per_s": 1000.0 / ms, "ms_per_solve": ms, "status": [int(x) for x in sts],
                     "ipm_iters": info["ipm_iters"], "cg_iters": info["cg_iters"], "rel_kkt_device": info["rel_kkt"],
                     "m": q["m"], "m_rows": s.sizes()["m_rows"],
                     "gpu_launches": int(info["kernel_launches"])}
        if name == "two_sided":
            res[name]["window_rows_binding"] = {"upper": int((y > 0).sum()), "lower": int((y < 0).sum()),
                                                "of": int(y.size)}
        s.close()
    clk = clocks.stop()
    out = {"mode": "two_sided", "metric": "QP solves/sec at rel. KKT <= 1e-6 (two-sided rows)",
           "value": res["two_sided"]["solves_per_s"], "unit": "solves/s", "steps": args.steps, "warmup": args.warmup,
           "dtype": "f64" if args.storage == "f64" else "%s storage, f64 refinement" % args.storage,
           "config": {"workload": WORKLOAD + "; plus two-sided dose windows on %d target and %d other voxels "
                                             "(workloads.rt_two_sided)" % (args.window_rows, args.window_rows),
                      "storage": args.storage, "precond": "jacobi_lr", "stiff_max": 1024},
           "two_sided": res["two_sided"], "one_sided": res["one_sided"], "clocks": clk}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2405_03584_gb300 import build, ipm, presets, workloads as W

    rank, world, local = _env_rank()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    build.build()
    dev = torch.cuda.current_device()
    p = W.rt_qp(n=N_FULL, seed=SEED)
    opts = presets.rt(args.storage, **_operator_opts(args))
    if args.precond:
        opts["precond"] = args.precond
    if args.system != "condensed":
        opts.update(system=args.system, precond="jacobi")
    s = ipm.Solver(use_graphs=0 if args.no_graphs else 1, **opts)
    s.set_qp_rt(p)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        st = s.solve()
    clocks = ClockSampler(dev)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    statuses, infos = [], []
    for k in range(args.steps):
        evs[k][0].record(stream)
        st = s.solve()
        evs[k][1].record(stream)
        out_info = s.get()["info"]
        statuses.append(st)
        infos.append(out_info)
        launches += out_info["kernel_launches"]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    lat = [a.elapsed_time(b) for a, b in evs]
    total_ms = max_over_ranks(evs[0][0].elapsed_time(evs[-1][1]))
    value = replica_rate(args.steps, world, total_ms)
    # roofline of the dominant kernel (PCG operator pass), timed live with CUDA events
    prof = s.profile_operator(reps=20)
    kern = "k_op_rows" if prof["ms_rows"] >= prof["ms_cols"] else "k_op_cols"
    key = "rows" if kern == "k_op_rows" else "cols"
    ms, byts, flops = prof["ms_" + key], prof["bytes_" + key], prof["flops_" + key]
    peak, peak_kind = _peaks()
    achieved = byts / (ms / 1000.0) / 1e9
    lanes = infos[-1]["lanes_rows"] if kern == "k_op_rows" else infos[-1]["lanes_cols"]
    lp = args.storage != "f64"
    df = infos[-1]["op_arith"] == 1
    mx = infos[-1]["op_arith"] == 2
    runs = infos[-1]["rows_runs"] == 1 and kern == "k_op_rows"
    base = kern + ("_lp" if lp else "") + ("_df" if df and not lp else "") + ("_mx" if mx and not lp else "") + \
        ("_runs" if runs else "")
    kname = "%s<%s%d lanes/row>" % (base, (args.storage + ", ") if lp else "", lanes)
    roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": _ncu_traffic(base, lanes),
            "peak_kind": peak_kind + " hbm_gbs",
            "algorithmic_bytes": byts, "ms_per_launch": ms,
            ("fp32_tflops" if lp or df else "fp64_tflops"): flops / (ms / 1000.0) / 1e12,
            "arith": "f32" if lp else ("double-float" if df else ("split f64 / double-float" if mx else "f64")),
            "fp64_nominal_tflops": FP64_NOMINAL_TFLOPS,
            "other_kernel": {"ms_per_launch": prof["ms_" + ("cols" if key == "rows" else "rows")],
                             "gbs": prof["bytes_" + ("cols" if key == "rows" else "rows")] /
                             (prof["ms_" + ("cols" if key == "rows" else "rows")] / 1000.0) / 1e9}}
    s.close()
    # end to end through the public API with host buffers (copies inside the timed region)
    e2e = None
    if args.e2e_steps > 0:
        pin = {}
        for k in ("D_indptr", "D_indices", "D_data", "w", "c", "b", "l", "u", "h0", "a_rows"):
            t = torch.from_numpy(np.ascontiguousarray(p[k])).pin_memory()
            pin[k] = t.numpy()
        q = dict(p)
        q.update(pin)
        h2d = sum(v.nbytes for v in pin.values())
        d2h = 8 * (3 * p["n"] + 2 * p["m"])
        def e2e_once():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            se = ipm.Solver(**opts)
            se.set_qp_rt(q)
            se.solve()
            se.get()
            se.close()
            torch.cuda.synchronize()
            return time.perf_counter() - t0

        e2e_once()                                   # untimed: first-call costs of the process
        e2e_t = [e2e_once() for _ in range(args.e2e_steps)]
        ipm.autotune_reset()                         # one more with the autotuner's cache emptied
        t_cold = e2e_once()
        e2e_val = len(e2e_t) / sum(e2e_t)
        if world > 1:
            e2e_val = replica_rate(len(e2e_t), world, 1000.0 * max_over_ranks(sum(e2e_t)))
        e2e = {"value": e2e_val, "unit": "solves/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": len(e2e_t), "includes": "ipm_create + ipm_set_qp (host arrays, pinned) + ipm_solve + ipm_get_xyz",
               "options": "as the device-timed solve; lanes from the autotuner's per-process cache (filled by the "
                          "untimed first pass)",
               "cold_autotune": {"value": 1.0 / t_cold, "unit": "solves/s", "seconds": t_cold,
                                 "note": "one more step after ipm_autotune_reset: ipm_set_qp times the lane widths again"}}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pts = [_oracle_time(n) for n in args.sample_sizes]
        v, law, fit = _cpu_law(pts)
        cpu = {"value": v, "unit": "solves/s", "cores": _cores_used(), "kind": "oracle",
               "sample": "oracle (dense-Cholesky FP64 IPM) full solves of the same RT generator at n in %s "
                         "(V = 4n, m = n/2.5); full-size rate from %s" % (list(args.sample_sizes), law),
               "fit": fit}
    if rank == 0:
        lat_sorted = sorted(lat)
        p99 = lat_sorted[min(len(lat_sorted) - 1, int(np.ceil(0.99 * len(lat_sorted))) - 1)]
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if args.storage == "f64" else
                        "%s operator storage, f32 accumulate, f64 refinement and reductions" % args.storage,
               "data": "synthetic",
               "config": {"workload": WORKLOAD, "storage": args.storage, "system": args.system, "n": p["n"], "V": p["V"], "m": p["m"], "nnz_D": int(p["D_indptr"][-1]),
                          "tol_kkt": TOL, "precond": opts["precond"], "parallelism": "replicas" if world > 1 else "single",
                          "l2": "no flush: operator working set (~1.2 GB) > 129 MB L2"},
               "latency_ms": {"p50": statistics.median(lat), "p99": p99, "mean": statistics.mean(lat)},
               "solve": {"status": [int(x) for x in statuses], "ipm_iters": [i["ipm_iters"] for i in infos],
                         "cg_iters": [i["cg_iters"] for i in infos], "rel_kkt_device": infos[-1]["rel_kkt"],
                         "max_stiff_rows": infos[-1]["max_stiff_rows"],
                         "lanes_per_row": [infos[-1]["lanes_rows"], infos[-1]["lanes_cols"]],
                         "op_arith": ["f64", "df32", "mixed"][infos[-1]["op_arith"]], "rows_runs": infos[-1]["rows_runs"],
                         "cols_gap": infos[-1]["cols_gap"], "refine_passes": infos[-1]["refine_passes"]},
               "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sample-n", default=",".join(str(v) for v in SAMPLE_SIZES),
                    help="comma-separated n of the oracle samples behind cpu_baseline and --impl reference")
    ap.add_argument("--operator-only", action="store_true",
                    help="profiler capture target: a few IPM iterations, then the operator kernels")
    ap.add_argument("--lanes", default="8,16", help="--operator-only: lanes per row over R and R^T")
    ap.add_argument("--batch", action="store_true", help="the 64-QP uneven batch instead of the single RT QP")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-scale", type=float, default=1.0, help="scale every n of the batch (testing)")
    ap.add_argument("--bfgs", choices=["proton", "vmat"], help="the quasi-Newton Hessian shapes of the paper")
    ap.add_argument("--sqp", action="store_true", help="the SQP outer loop with GPU QP sub-problems")
    ap.add_argument("--dense", action="store_true", help="the dense QP (n = 500, m = 1000)")
    ap.add_argument("--dense-autotune", type=int, default=1, help="--dense: time the lane widths per matrix (0: fixed)")
    ap.add_argument("--two-sided", action="store_true", help="the RT workload with two-sided dose-window rows")
    ap.add_argument("--window-rows", type=int, default=200, help="--two-sided: window rows per voxel class")
    ap.add_argument("--sqp-n", type=int, default=10000)
    ap.add_argument("--sqp-iters", type=int, default=150)
    ap.add_argument("--serve", action="store_true", help="the serving stream (Poisson arrivals, chains, warm start)")
    ap.add_argument("--serve-lambda", type=float, default=20.0)
    ap.add_argument("--serve-horizon", type=float, default=60.0)
    ap.add_argument("--serve-inflight", type=int, default=16)
    ap.add_argument("--serve-no-baseline", action="store_true")
    ap.add_argument("--system", choices=["condensed", "augmented"], default="condensed",
                    help="the linear system of the Newton step (augmented: the paper's eq:2x2_augmented, Jacobi PCG)")
    ap.add_argument("--storage", choices=["f64", "f32", "bf16", "fp8"], default="f64",
                    help="operator storage of the single RT QP (reduced ones add FP64 refinement)")
    ap.add_argument("--precond", choices=["jacobi", "jacobi_lr", "block32"], default=None,
                    help="preconditioner of the RT and quasi-Newton modes (default: jacobi_lr)")
    ap.add_argument("--op-arith", choices=["f64", "df32", "mixed"], default=None,
                    help="PCG operator arithmetic with f64 storage (default: the preset's)")
    ap.add_argument("--rows-format", choices=["auto", "csr", "runs"], default=None,
                    help="format of the PCG rows pass (default: the preset's)")
    ap.add_argument("--rows-stage", type=int, choices=[0, 1], default=None,
                    help="1: rows pass staged through shared memory by bulk copies where available; 0: not")
    ap.add_argument("--cols-format", type=int, choices=[0, 1], default=None,
                    help="reduced storages: 0 column pass on int32 indices (default), 1 on 16-bit row gaps")
    ap.add_argument("--refine-eta", type=float, default=None,
                    help="reduced storages: factor between FP64 residual evaluations (default: automatic)")
    ap.add_argument("--refine-mode", type=int, choices=[0, 1, 2], default=None,
                    help="reduced storages: 0 restarted refinement passes, 1 one PCG with residual replacement, "
                         "2 automatic (the default)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel directly (for per-kernel profilers; same kernels, slower)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    args.sample_sizes = tuple(int(v) for v in str(args.sample_n).split(",") if v.strip())
    if args.impl == "reference":
        return run_reference(args)
    if args.operator_only:
        return run_operator_only(args)
    if args.batch:
        return run_batch(args)
    if args.bfgs:
        return run_bfgs(args)
    if args.sqp:
        return run_sqp(args)
    if args.dense:
        return run_dense(args)
    if args.two_sided:
        return run_two_sided(args)
    if args.serve:
        # more hardware work queues than the default 8, so many slots' streams run side by side
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
