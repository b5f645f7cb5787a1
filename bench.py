#!/usr/bin/env python3
"""Benchmark: time to a 1e-6 relative duality gap on the large single problem
(n = 1e7 jobs, m = 32 resources; FP32 row-major A of 1.28 GB), plus the HBM
roofline of one dual evaluation.

One step = one complete price-discovery solve (Algorithm 2 of arXiv
2104.00282 on the device: Eq. e-initialization, then dual evaluations and
L-BFGS price updates until the certified relative gap is <= 1e-6), inputs
already resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (same algorithm, scipy L-BFGS-B
price updates) on the host cores on a bounded sample of the same workload.
With N > 1 ranks the one problem is split by job range across the ranks
(ra_solve_sharded: an all-gather of 4 + 2m sums per evaluation, the same
price update on every rank), so the total work is fixed: strong scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-6 rel. duality gap at n=1e7,m=32; dual-eval HBM GB/s vs peak"
N_JOBS, M_RES, TOL = 10_000_000, 32, 1e-6
BATCH_MAX_EVALS = 500
WORKLOAD = ("large single problem: n=1e7 jobs, m=32 resources, A_ij = s_j exp(0.75 z), "
            "s_j~U[0.25,8], FP32 row-major (1.28 GB); utilities 40% log, 40% power p~U[0.2,0.8], "
            "20% linear with cap T~U[1,10]; w~U[0.5,2]; R_j~U[0.05,0.3] n; maximize sum_i u_i(a_i^T x_i) "
            "over X >= 0 with X^T 1 <= R; cold start (Eq. e-initialization) to 1e-6 relative duality gap")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl"
        dist.init_process_group(backend=backend)
        return dist, dist.get_rank(), ws
    return None, 0, 1


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            # the timed region is tens of ms: start it once samples flow
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_hash():
    h = hashlib.sha256()
    for f in ("ra_dual.cu", "ra_kernels.cuh", "ra_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2104_00282_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """dram bytes per launch of the dual kernel from the committed ncu summary,
    or None when the kernel source changed since it was captured."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "dual_eval_large_traffic.json")))
    except Exception:
        return None
    if d.get("kernel_hash") != kernel_hash():
        return None
    return d.get("dram_bytes_per_launch")


ORACLE_MAX_EVALS = 2000
REF_BUDGET_S = 120.0        # host seconds the whole --impl reference run may take
ORACLE_US_PER_JOB = 4.0     # oracle solve time per job of the workload (16 host cores)


def oracle_sample_size(steps, warmup):
    """Jobs in the oracle's sample: the reference arm solves it once per step
    (warm-up included) within about REF_BUDGET_S; the GPU arm's cpu_baseline
    leg uses the same size for the same --steps/--warmup, so the two oracle
    figures of one run describe the same computation."""
    per_step = REF_BUDGET_S / max(steps + warmup, 1)
    n = int(per_step / (ORACLE_US_PER_JOB * 1e-6))
    return int(min(max(n, 500_000), 2_000_000) // 100_000 * 100_000)


def cpu_baseline(sample_n, seed=0, cap=False):
    """Oracle solve (FP64, OpenMP, scipy L-BFGS-B) of the first sample_n jobs
    of the workload with R scaled to the sample, to the same 1e-6 relative
    gap; returns a dict with the time for the sample, the time scaled
    linearly to n = 1e7, the thread count, the evaluations, the gap reached
    and whether it converged (an unconverged time is flagged, not hidden)."""
    from oracle import oracle as O
    from paper_2104_00282_gb300 import workloads as W
    prob = W.config_large(n=sample_n, m=M_RES, seed=seed)
    t0 = time.perf_counter()
    sol = O.solve(prob, cap=cap, tol=TOL, max_evals=ORACLE_MAX_EVALS)
    dt = (time.perf_counter() - t0) * 1e3
    return dict(ms=dt, scaled=dt * (N_JOBS / sample_n), threads=O.max_threads(), evals=sol.evals,
                gap=sol.gap, converged=bool(sol.converged), sample_n=sample_n)


def _sample_text(r):
    return (f"oracle solve of the first {r['sample_n']} jobs of the workload (seed 0, R scaled to the "
            f"sample) to a {TOL:g} relative gap: {r['evals']} evaluations, gap {r['gap']:.2e}, "
            f"{'converged' if r['converged'] else 'NOT converged'}, {r['ms']:.0f} ms; "
            f"time scaled x{N_JOBS / r['sample_n']:g} to n=1e7 (linear in n)")


def run_reference(args):
    dist, rank, ws = _dist()
    if rank != 0:
        return
    sample_n = args.cpu_sample or oracle_sample_size(args.steps, args.warmup)
    vals, runs = [], []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(sample_n, seed=0, cap=args.job_cap)
        if k >= args.warmup:
            vals.append(r["scaled"])
            runs.append(r)
    v = statistics.median(vals)
    last = runs[-1]
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_JOBS, "m": M_RES, "tol_rel": TOL,
                   "job_cap": args.job_cap},
        "cpu_baseline": {"value": v, "unit": "ms", "cores": last["threads"], "kind": "oracle",
                         "converged": all(r["converged"] for r in runs), "gap": last["gap"],
                         "sample": _sample_text(last)},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def certify_headline(prob, P, cap):
    """FP64 oracle check of a GPU solve of the full workload: g at the GPU's
    best prices, the utility of the GPU's lower-bound allocation rebuilt by
    the oracle, the relative gap between them, the worst usage / R of that
    allocation, and the GPU's own g and U_lb against the oracle's."""
    from oracle import oracle as O
    import numpy as np
    lam = P.prices.cpu().numpy()
    theta, lams, scaled = P.certificate()
    repaired = None
    if 2 in list(scaled):   # the bound is the repaired allocation at lams[0]
        out = P.recover_feasible(lams[0])
        repaired = (out["jk"].cpu().numpy(), out["xk"].cpu().numpy())
    c = O.certify(prob, lam, theta, lams, scaled, cap, repaired=repaired)
    return {"rel_gap_oracle": c["rel_gap"], "g_oracle": c["g"], "U_lb_oracle": c["U_lb"],
            "max_usage_over_R": c["max_usage_over_R"], "oracle_seconds": c["seconds"],
            "certificate_entries": int(np.sum(np.asarray(theta) > 0))}


def run_gpu(args):
    import numpy as np
    import torch

    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__ as G
    if rank == 0:
        G.build()
    if dist:
        dist.barrier()
    from paper_2104_00282_gb300 import ra
    from paper_2104_00282_gb300 import workloads as W

    n, m = args.n, M_RES
    prob = W.config_large(n=n, m=m, seed=rank)
    stream = torch.cuda.Stream()
    dev = torch.device("cuda", local)
    cap = args.job_cap
    use_graph = not args.no_graph
    with torch.cuda.stream(stream):
        P = ra.AllocationProblem.from_numpy(prob, dev, stream=stream, job_cap=cap)

    def step():
        return P.solve(tol=TOL, max_evals=args.max_evals, use_graph=use_graph)

    times, infos = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            info = step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            info = step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = statistics.median(times)
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = t.item()

    # FP64 oracle certificate of the last timed solve (error against the oracle
    # stated for the headline result)
    cert = certify_headline(prob, P, cap) if (rank == 0 and not args.no_certify) else None

    # roofline of one dual evaluation (the dominant kernel), CUDA events on its stream
    lam0 = P.init_prices()
    with torch.cuda.stream(stream):
        for _ in range(3):
            ra.ra_eval_dual(P.handle, lam0)
        reps = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ra.ra_eval_dual(P.handle, lam0)
        e1.record(stream)
    e1.synchronize()
    eval_ms = e0.elapsed_time(e1) / reps
    alg_bytes = n * (4 * m + 4 + 4 + 1)
    achieved = alg_bytes / (eval_ms * 1e-3) / 1e9
    peaks = _peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0

    # end to end through the public API: pinned host inputs -> device, solve, prices back
    hA = torch.from_numpy(prob.A).pin_memory()
    hk = torch.from_numpy(prob.kind).pin_memory()
    hw = torch.from_numpy(prob.w).pin_memory()
    hp = torch.from_numpy(prob.param).pin_memory()
    hR = torch.from_numpy(prob.R).pin_memory()
    e2e_times = []
    for k in range(max(2, min(args.steps, 3)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            Q = ra.AllocationProblem(hA.to(dev, non_blocking=True), hk.to(dev, non_blocking=True),
                                     hw.to(dev, non_blocking=True), hp.to(dev, non_blocking=True),
                                     hR.to(dev, non_blocking=True), stream=stream, job_cap=cap)
            Q.solve(tol=TOL, max_evals=args.max_evals, use_graph=use_graph)
            out = Q.prices.to("cpu", non_blocking=False)
        Q.close()
        del Q
        if k > 0:
            e2e_times.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = statistics.median(e2e_times)
    h2d = prob.A.nbytes + prob.kind.nbytes + prob.w.nbytes + prob.param.nbytes + prob.R.nbytes
    d2h = out.numel() * 8

    # the same workload in the other mode: with / without the paper's per-job
    # time cap 1^T x_i <= 1 (problem (e-res-alloc))
    P.close()
    with torch.cuda.stream(stream):
        Po = ra.AllocationProblem.from_numpy(prob, dev, stream=stream, job_cap=not cap)
    o_times, o_info = [], None
    for k in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        o_info = Po.solve(tol=TOL, max_evals=args.max_evals, use_graph=use_graph)
        e1.record(stream)
        e1.synchronize()
        if k > 0:
            o_times.append(e0.elapsed_time(e1))
    # the other mode's standalone evaluation (CUDA events, as the headline's)
    lam_o = Po.init_prices()
    with torch.cuda.stream(stream):
        for _ in range(3):
            ra.ra_eval_dual(Po.handle, lam_o)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ra.ra_eval_dual(Po.handle, lam_o)
        e1.record(stream)
    e1.synchronize()
    o_eval_ms = e0.elapsed_time(e1) / reps
    Po.close()
    other = {"ms": statistics.median(o_times), "evals": o_info["evals"],
             "rel_gap": o_info["rel_gap"], "status": o_info["status"]}

    # precision study: the same workload with FP64 per-job arithmetic
    # (RA_FP64_JOBMATH), timed and certified by the oracle like the headline
    prec = None
    if args.fp64_study:
        with torch.cuda.stream(stream):
            P64 = ra.AllocationProblem.from_numpy(prob, dev, stream=stream, job_cap=cap,
                                                  fp64_jobmath=True)
        p_times, p_info = [], None
        for k in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            p_info = P64.solve(tol=TOL, max_evals=args.max_evals, use_graph=use_graph)
            e1.record(stream)
            e1.synchronize()
            if k > 0:
                p_times.append(e0.elapsed_time(e1))
        c64 = certify_headline(prob, P64, cap) if (rank == 0 and not args.no_certify) else None
        P64.close()
        prec = {"fp32_jobmath": {"ms": ms, "evals": infos[-1]["evals"],
                                 "rel_gap_gpu": infos[-1]["rel_gap"], "oracle": cert},
                "fp64_jobmath": {"ms": statistics.median(p_times), "evals": p_info["evals"],
                                 "rel_gap_gpu": p_info["rel_gap"], "status": p_info["status"],
                                 "oracle": c64},
                "note": "per-job arithmetic in FP32 (headline) or FP64; reductions, dual value "
                        "and price update FP64 in both; each result re-checked by the FP64 oracle"}

    batch = run_batch(args, dev, stream) if args.batch > 0 else None
    medium = run_paper_medium(args, dev, stream) if args.paper_medium > 0 else None
    warm = run_warm(args) if args.warm > 0 else None

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        sample_n = args.cpu_sample or oracle_sample_size(args.steps, args.warmup)
        r = cpu_baseline(sample_n, cap=cap)
        cpu = {"value": r["scaled"], "unit": "ms", "cores": r["threads"], "kind": "oracle",
               "converged": r["converged"], "gap": r["gap"], "sample": _sample_text(r)}
    evals = [i["evals"] for i in infos]
    # per solve: initialisation (+ the ray scaling without the cap) and setup,
    # then per evaluation: dual pass, lower-bound pass (it returns at once
    # when the evaluation wrote no records), solver step; per repair of the
    # lower bound: scan, collect, gather, apply, FP64 evaluation, accept
    launches = sum((2 if cap else 3) + 3 * i["evals"] + 6 * i["repairs"] for i in infos)
    # the in-solve evaluation kernel: device time between price updates (the
    # solver's own global-timer accounting), against the bytes of A, w,
    # param and kind alone (the lower-bound records, 10 B/job written and 10
    # read once the records are on, are left out: a lower bound on the rate)
    ev_ms = statistics.median(i["eval_ms"] / max(i["evals"], 1) for i in infos)
    st_ms = statistics.median(i["step_ms"] / max(i["evals"], 1) for i in infos)
    in_solve = {"achieved": alg_bytes / (ev_ms * 1e-3) / 1e9, "frac": alg_bytes / (ev_ms * 1e-3) / 1e9 / peak,
                "launch_ms": ev_ms, "step_ms": st_ms,
                "kernel": (f"dual_tma_kernel in the solve ({'with cap; records for the lagged bound' if cap else 'no cap; own bound from its sums, no records'})"
                           if n >= 4_000_000 or cap else
                           "dual_tma_kernel in the solve (no cap; own bound and records for the lagged one)"),
                "timing": "device global timer between solver steps (graph launch gaps included)"}
    other_mode = {"achieved": alg_bytes / (o_eval_ms * 1e-3) / 1e9,
                  "frac": alg_bytes / (o_eval_ms * 1e-3) / 1e9 / peak, "launch_ms": o_eval_ms,
                  "kernel": f"dual_tma_kernel, {'no' if cap else 'with'} per-job cap (ra_eval_dual)",
                  "timing": "CUDA events, 20 launches"}
    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "m": m, "tol_rel": TOL,
                   "job_cap": cap, "cuda_graph": use_graph,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs 1.37 GB per evaluation > 126 MB L2; no flush needed",
                   "precision": "per-job math f32; reductions, dual value, price update f64"},
        "solve": {"evals_median": statistics.median(evals), "rel_gap": infos[-1]["rel_gap"],
                  "status": infos[-1]["status"], "ms_per_eval_in_solve": ms / statistics.median(evals),
                  "g": infos[-1]["g"], "U_lb": infos[-1]["U_lb"],
                  "oracle_certificate": cert, "step_ms_all": times},
        "precision_study": prec,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": ncu_traffic(),
                     "kernel": f"dual_tma_kernel, {'with' if cap else 'no'} per-job cap "
                               "(ra_eval_dual, no lower-bound record)",
                     "alg_bytes_per_launch": alg_bytes, "launch_ms": eval_ms,
                     "peak_source": f"{peak_src} hbm_gbs (burst copy)",
                     "in_solve": in_solve,
                     ("capped" if not cap else "uncapped"): other_mode},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        ("no_job_cap" if cap else "with_job_cap"): other,
        "batched": batch,
        "warm_start": warm,
        "paper_medium": medium,
    }
    print(json.dumps(line), flush=True)


def run_sharded(args):
    """One n = 1e7 problem split by job range across the ranks (one GPU each):
    every rank evaluates its shard, the ranks all-gather m-sized sums once
    per evaluation (NCCL) and run the same price update (ra_solve_sharded).
    The total work is fixed as ranks are added: strong scaling."""
    import numpy as np
    import torch

    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__ as G
    if rank == 0:
        G.build()
    if dist:
        dist.barrier()
    from paper_2104_00282_gb300 import ra, sharded
    from paper_2104_00282_gb300 import workloads as W

    n, m = args.n, M_RES
    cap = args.job_cap
    prob = W.config_large(n=n, m=m, seed=0)          # the same problem on every rank
    lo, hi = sharded.shard_bounds(n, ws)[rank]
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    host = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
            for x in (prob.A[lo:hi], prob.kind[lo:hi], prob.w[lo:hi], prob.param[lo:hi], prob.R)]
    gather = sharded.torch_gather() if dist else (lambda send, recv: recv.copy_(send))

    def make_shard():
        with torch.cuda.stream(stream):
            A, kind, w, par, R = (t.to(dev, non_blocking=True) for t in host)
            return ra.AllocationProblem(A, kind, w, par, R, job_cap=cap, stream=stream), R

    P, R_dev = make_shard()

    def step():
        with torch.cuda.stream(stream):
            return sharded.solve(P, n, rank, ws, gather, tol=TOL, max_evals=args.max_evals)

    times, infos = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            lam, info = step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
        torch.cuda.synchronize()
    ms = statistics.median(times)
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = t.item()
    cert = None
    if rank == 0 and not args.no_certify:
        from oracle import oracle as O
        theta, lams, scaled = P.certificate()
        c = O.certify(prob, lam.cpu().numpy(), theta, lams, scaled, cap)
        cert = {"rel_gap_oracle": c["rel_gap"], "max_usage_over_R": c["max_usage_over_R"],
                "g_oracle": c["g"], "U_lb_oracle": c["U_lb"], "oracle_seconds": c["seconds"]}
    # roofline: this rank's partial evaluation (its shard's jobs)
    lam0 = P.init_prices()
    part = torch.empty(ra.RA_SHARD_WIDTH(m), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(3):
            ra.ra_eval_partial(P.handle, lam0, part)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            ra.ra_eval_partial(P.handle, lam0, part)
        e1.record(stream)
    e1.synchronize()
    eval_ms = e0.elapsed_time(e1) / 20
    alg_bytes = (hi - lo) * (4 * m + 9)
    peak = _peaks().get("hbm_gbs") or 6800.0
    # end to end: pinned host shard -> device, solve, prices back
    e2e = []
    for k in range(3):
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        Q, _ = make_shard()
        with torch.cuda.stream(stream):
            lq, _ = sharded.solve(Q, n, rank, ws, gather, tol=TOL, max_evals=args.max_evals)
            lq.to("cpu")
        Q.close()
        if k > 0:
            e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = statistics.median(e2e)
    if dist:
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = t.item()
    P.close()
    if rank != 0:
        return
    evals = [i["evals"] for i in infos]
    h2d = prob.A.nbytes + prob.kind.nbytes + prob.w.nbytes + prob.param.nbytes + prob.R.nbytes
    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "m": m, "tol_rel": TOL, "job_cap": cap,
                   "parallelism": f"one problem in {ws} job-range shards (ra_solve_sharded, "
                                  "all-gather of 4+2m sums per evaluation)",
                   "l2": "inputs 1.37 GB per evaluation > 126 MB L2; no flush needed"},
        "solve": {"evals_median": statistics.median(evals), "rel_gap": infos[-1]["rel_gap"],
                  "status": infos[-1]["status"], "oracle_certificate": cert, "step_ms_all": times},
        "roofline": {"bound": "hbm", "achieved": alg_bytes / (eval_ms * 1e-3) / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": alg_bytes / (eval_ms * 1e-3) / 1e9 / peak, "traffic": None,
                     "kernel": "dual_tma_kernel over rank 0's shard (ra_eval_partial)",
                     "alg_bytes_per_launch": alg_bytes, "launch_ms": eval_ms},
        "cpu_baseline": None,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": m * 8},
        "gpu_launches": sum(5 + 4 * e for e in evals),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_paper_medium(args, dev, stream):
    """The paper's medium problem (Section 6.2: n = 1e6, m = 4, the per-job
    cap, log utility and target-priority utility with t_des = 0.2, w in
    {1, 2}) solved to 1e-6, with the statistics of the allocation the
    library returns (ra_recover_feasible at the final prices) beside the
    paper's: jobs on two resources, jobs with slack, jobs reaching the
    target.  The paper's own times (GTX 1070, FP32 PyTorch, absolute gap
    1e-3 n) are context only."""
    import numpy as np
    import torch
    from paper_2104_00282_gb300 import ra
    from paper_2104_00282_gb300 import workloads as W
    out = {}
    paper = {"log": {"gpu_s": 0.30, "two_resources": 0.17, "positive_slack": 0.18},
             "target": {"gpu_s": 0.89, "two_resources": 0.67, "positive_slack": 0.50,
                        "reach_target": ">0.95", "low_priority_miss": 0.10}}
    for util in ("log", "target"):
        prob = W.paper_medium(n=args.paper_medium, utility=util, seed=0)
        with torch.cuda.stream(stream):
            P = ra.AllocationProblem.from_numpy(prob, dev, stream=stream, job_cap=True)
        times, info = [], None
        for k in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            info = P.solve(tol=TOL, max_evals=args.max_evals)
            e1.record(stream)
            e1.synchronize()
            if k > 0:
                times.append(e0.elapsed_time(e1))
        rec = P.recover_feasible()
        jk = rec["jk"].cpu().numpy().reshape(-1, 4)
        xk = rec["xk"].cpu().numpy().reshape(-1, 4).astype(np.float64)
        P.close()
        used = (jk >= 0) & (xk > 1e-9)
        a = np.where(jk >= 0, prob.A[np.arange(prob.n)[:, None], np.maximum(jk, 0)], 0.0)
        t = (a * np.where(jk >= 0, xk, 0.0)).sum(1)
        st = {"ms": statistics.median(times), "evals": info["evals"], "rel_gap": info["rel_gap"],
              "status": info["status"], "repairs": info["repairs"],
              "two_resources": float(np.mean(used.sum(1) == 2)),
              "positive_slack": float(np.mean(1.0 - np.where(jk >= 0, xk, 0.0).sum(1) > 1e-6)),
              "max_usage_over_R": rec["info"]["max_usage_over_R"]}
        if util == "target":
            reach = t >= 0.2 - 1e-6
            st["reach_target"] = float(reach.mean())
            st["low_priority_miss"] = float((~reach[prob.w == 1]).mean())
            st["high_priority_miss"] = float((~reach[prob.w == 2]).mean())
        out[util] = {"gb300": st, "paper": paper[util]}
    out["note"] = ("n = %d, m = 4, per-job cap; target-priority optima are not unique (a linear "
                   "program): the two-resource fraction depends on which optimum a solver returns" % args.paper_medium)
    return out


def run_sweep(args):
    """The scaling experiments of Section 6.4 (Fig. 10) and the large problem of
    Section 6.3, on this GPU.  Dual evaluation time (CUDA events, the mean of
    20 back-to-back ra_eval_dual launches at the Eq. e-initialization prices,
    the per-job cap of the paper's experiments) against m at n = 1e5 and
    against n at m = 4, reported as algorithmic GB/s (n (4m + 9) bytes per
    evaluation) and as a fraction of the measured copy bandwidth; and the
    n = 5e7, m = 4 log-utility problem solved to 1e-6.  Workloads: the
    Section 6.1 code example generator (A ~ U[0, 1], R = U[0, 1] n + 1e3,
    log utility).  Prints one JSON object."""
    import torch
    import __graft_entry__ as G
    G.build()
    from paper_2104_00282_gb300 import ra
    from paper_2104_00282_gb300 import workloads as W
    peak = _peaks().get("hbm_gbs") or 6800.0
    l2 = torch.cuda.get_device_properties(0).L2_cache_size

    def eval_point(n, m):
        prob = W.paper_code_example(n=n, m=m, seed=0)
        P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=True)
        lam = P.init_prices()
        for _ in range(3):
            ra.ra_eval_dual(P.handle, lam)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            ra.ra_eval_dual(P.handle, lam)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 20
        P.close()
        b = n * (4 * m + 9)
        return {"n": n, "m": m, "ms": ms, "GB_s": b / (ms * 1e-3) / 1e9,
                "hbm_frac": b / (ms * 1e-3) / 1e9 / peak, "bytes": b,
                "l2_resident": b < l2}

    out = {"peak_gbs": peak, "peak_source": "measured hbm_gbs", "l2_bytes": l2,
           "vs_m": [eval_point(100_000, m) for m in (2, 4, 8, 16, 32)],
           "vs_n": [eval_point(n, 4) for n in (100, 1_000, 10_000, 100_000, 1_000_000,
                                               10_000_000, 100_000_000)]}
    # Section 6.3: n = 5e7, m = 4, log utility, solved with the per-job cap
    prob = W.paper_code_example(n=50_000_000, m=4, seed=1)
    P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=True)
    ts, info = [], None
    for k in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        info = P.solve(tol=TOL, max_evals=args.max_evals)
        e1.record()
        e1.synchronize()
        if k > 0:
            ts.append(e0.elapsed_time(e1))
    P.close()
    out["large_5e7_m4"] = {"ms": statistics.median(ts), "evals": info["evals"],
                           "rel_gap": info["rel_gap"], "status": info["status"],
                           "paper": "228 s CPU (i7-6700K), about 7.9 s GPU (V100), FP32, absolute gap 1e-3 n"}
    print(json.dumps(out), flush=True)


def run_warm(args):
    """Learned warm start (the committed network, trained by
    paper_2104_00282_gb300.warmstart on 20000 solved problems): cold and warm
    ra_solve of held-out problems of the same recipe (n log-uniform in
    [1e4, 1e6], m = 16, no per-job cap), median device time and evaluations
    to a 1e-6 relative gap; the warm time includes the statistics, the
    network and both start-point evaluations."""
    import os
    from paper_2104_00282_gb300 import warmstart as WS
    if not os.path.exists(WS.WEIGHTS):
        return {"unavailable": "no trained network in the package"}
    net = WS.load()
    max_evals = 3000
    rec = WS.evaluate(net, P=args.warm, log=None, max_evals=max_evals)
    net.close()
    out = WS.summarize(rec)
    out["held_out_seed"] = WS.EVAL_SEED
    out["max_evals"] = max_evals
    out["note"] = ("medians over all held-out problems; a solve that stops at the evaluation "
                   "limit counts with its time")
    return out


def run_batch(args, dev, stream):
    """Batched price discovery: P independent problems (n log-uniform in
    [100, 2e5], m in {4, 8, 16, 32}) solved together to the same tolerance,
    cold start.  The launch shape of the batched evaluation is chosen by the
    package's autotuner on this workload (cached per GPU and workload).
    Reports problems/s over the whole batch, the percentiles of the
    per-problem device time to tolerance, and the bytes the batched passes
    streamed (sum over problems of evaluations x n (4m + 29): the A rows,
    w, param, kind and the 20-byte lower-bound records) per second."""
    import numpy as np
    import torch
    from paper_2104_00282_gb300 import autotune
    from paper_2104_00282_gb300 import ra
    from paper_2104_00282_gb300 import workloads as W

    P = args.batch
    n, m = W.batched_shapes(P)
    probs = W.batched_workload(P)
    tensors = [tuple(torch.from_numpy(np.ascontiguousarray(x)).to(dev)
                     for x in (p.A, p.kind, p.w, p.param, p.R)) for p in probs]
    del probs
    torch.cuda.synchronize()
    shape, tuned = autotune.tune(tensors, job_cap=True, tol=TOL, max_evals=BATCH_MAX_EVALS)

    def timed(shape):
        with torch.cuda.stream(stream):
            B = ra.AllocationBatch.from_tensors(tensors, job_cap=True, stream=stream, shape=shape)
        times, secs, infos = [], None, None
        for k in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            infos, secs = B.solve(tol=TOL, max_evals=BATCH_MAX_EVALS)
            e1.record(stream)
            e1.synchronize()
            if k > 0:
                times.append(e0.elapsed_time(e1))
        B.close()
        return statistics.median(times), times, infos, np.asarray(secs)

    ms, times, infos, secs = timed(shape)
    ms_default, _, _, secs_default = timed(None)
    evals = np.array([i["evals"] for i in infos])
    status = np.array([i["status"] for i in infos])
    bytes_streamed = float(np.sum(evals * n * (4 * m + 29)))
    peak = _peaks().get("hbm_gbs") or 6800.0
    return {"problems": P, "jobs": int(n.sum()), "A_bytes": int((n * m).sum() * 4),
            "ms": ms, "problems_per_s": P / (ms * 1e-3),
            "jobs_per_s": float(n.sum()) / (ms * 1e-3),
            "time_to_tol_ms": {"p50": float(np.percentile(secs, 50) * 1e3),
                               "p99": float(np.percentile(secs, 99) * 1e3),
                               "max": float(secs.max() * 1e3)},
            "evals": {"p50": float(np.median(evals)), "p99": float(np.percentile(evals, 99)),
                      "max": int(evals.max())},
            "converged": int((status == 0).sum()), "step_ms_all": times,
            "streamed_GB_s": bytes_streamed / (ms * 1e-3) / 1e9,
            "streamed_hbm_frac": bytes_streamed / (ms * 1e-3) / 1e9 / peak,
            "shape": {"chunk_tiles": shape[0], "whole_tiles": shape[1], "ctas_per_sm": shape[2],
                      "chosen_by": "autotune over " + str(len(tuned.get("trials", []))) +
                                   " shapes (0 = cached)"},
            "default_shape": {"shape": [16, 0, 0], "ms": ms_default,
                              "p50": float(np.percentile(secs_default, 50) * 1e3),
                              "p99": float(np.percentile(secs_default, 99) * 1e3)},
            "workload": "n log-uniform in [100, 2e5], m uniform in {4, 8, 16, 32}, "
                        "heterogeneous-hardware recipe, per-job cap 1^T x_i <= 1 (problem "
                        "e-res-alloc), cold start to 1e-6 relative gap, at most 500 evaluations"}


def run_profile(args):
    """Small, self-contained workloads for a profiler (ncu), one per kind of
    launch: ``eval`` runs --reps standalone dual evaluations (ra_eval_dual) at
    the Eq. e-initialization prices of the large recipe (n = --n, m = --m);
    ``solve`` one solve with the host-driven loop, so that every launch is a
    separate kernel the profiler can see (inside a CUDA graph's conditional
    node it cannot); ``batch`` one batched solve of the batched workload's
    first --problems problems with the host loop; ``warm`` one warm-started
    solve (statistics, network, start prices, solve) of a held-out problem of
    the warm-start recipe (n = --n, m = 16)."""
    import torch
    import __graft_entry__ as G
    G.build()
    from paper_2104_00282_gb300 import ra
    from paper_2104_00282_gb300 import workloads as W
    what = args.profile
    if what in ("eval", "solve"):
        prob = W.config_large(n=args.n, m=args.m, seed=0)
        P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=args.job_cap)
        if what == "eval":
            lam = P.init_prices()
            for _ in range(args.reps):
                ra.ra_eval_dual(P.handle, lam)
            out = f"{args.reps} evaluations"
        else:
            out = P.solve(tol=TOL, max_evals=args.max_evals, use_graph=False)
        P.close()
    elif what == "batch":
        probs = W.batched_workload(args.problems)
        B = ra.AllocationBatch(probs, job_cap=True)
        infos, _ = B.solve(tol=TOL, max_evals=BATCH_MAX_EVALS, use_graph=False)
        out = f"{sum(i['status'] == 0 for i in infos)} of {len(infos)} converged"
        B.close()
    else:
        from paper_2104_00282_gb300 import warmstart as WS
        net = WS.load()
        A, kind, w, param, R = W.hetero_device(args.n, 16, WS.EVAL_SEED, 5, "cuda")
        P = ra.AllocationProblem(A, kind, w, param, R, job_cap=False)
        lam0, used = P.warm_prices(net)
        out = P.solve(tol=TOL, max_evals=BATCH_MAX_EVALS, lam0=lam0, use_graph=False)
        P.close()
        net.close()
    torch.cuda.synchronize()
    print("profile", what, out, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_JOBS)
    ap.add_argument("--m", type=int, default=M_RES, help="resources (--profile eval/solve only)")
    ap.add_argument("--profile", choices=["eval", "solve", "batch", "warm"], default=None,
                    help="run one small workload for a profiler instead of the benchmark")
    ap.add_argument("--reps", type=int, default=6, help="evaluations of --profile eval")
    ap.add_argument("--problems", type=int, default=512, help="problems of --profile batch")
    ap.add_argument("--max-evals", type=int, default=400)
    ap.add_argument("--cpu-sample", type=int, default=0, help="jobs in the oracle sample (0 = auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--job-cap", action="store_true",
                    help="headline with the paper's per-job cap 1^T x_i <= 1 (default: X >= 0 only)")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven solver loop (same kernels; lets ncu see every launch)")
    ap.add_argument("--warm", type=int, default=1000,
                    help="held-out problems in the warm-start comparison (0 = skip)")
    ap.add_argument("--sweep", action="store_true",
                    help="the Section 6.3-6.4 scaling experiments instead of the benchmark")
    ap.add_argument("--shard", action="store_true",
                    help="use the job-range sharded solve even on one rank (it is the default "
                         "with more than one rank)")
    ap.add_argument("--no-certify", action="store_true",
                    help="skip the FP64 oracle re-check of the headline solve")
    ap.add_argument("--fp64-study", type=int, default=1,
                    help="1 = also solve the workload with FP64 per-job arithmetic (precision study)")
    ap.add_argument("--paper-medium", type=int, default=1_000_000,
                    help="jobs of the paper's medium problem solved beside the headline (0 = skip)")
    ap.add_argument("--batch", type=int, default=4096,
                    help="problems in the batched solve reported beside the headline (0 = skip)")
    args = ap.parse_args()
    if args.sweep:
        run_sweep(args)
    elif args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    elif int(os.environ.get("WORLD_SIZE", "1")) > 1 or args.shard:
        run_sharded(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
