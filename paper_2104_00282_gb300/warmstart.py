"""Learned warm start: corpus labelling, training and evaluation.

A corpus of problems of the heterogeneous-hardware recipe (n log-uniform in
[1e4, 1e6], m = 16) is drawn on the GPU, every problem is solved to a 1e-6
relative duality gap by the batched solver (ra_batch_solve), and the network
input of each resource (ra_batch_features) is paired with the target
log(lambda*_j + RA_MLP_PRICE_OFFSET).  The network is trained with
ra_mlp_train_step (the library's forward, back-propagation and Adam
kernels) and evaluated on held-out problems by solving each one twice with
ra_solve: from the paper's Eq. e-initialization prices (cold) and from
ra_warmstart_prices (warm, which falls back to the cold prices when the
network's prices give a larger dual value g).

The problems are solved without the per-job cap by default: with the cap
this recipe leaves about three quarters of the capacity idle and a cold
solve ends in 3 to 9 evaluations, leaving nothing for a start point to save.

    python -m paper_2104_00282_gb300.warmstart train [--problems 20000] [--out FILE]
    python -m paper_2104_00282_gb300.warmstart evaluate [--problems 1000] [--weights FILE]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "warmstart_mlp.npy")
M = 16
TRAIN_SEED, EVAL_SEED = 0, 1
# first price step from the network's prices, as a fraction of |lambda| (the
# cold start's 0.05 overshoots from a start a few percent from the optimum)
WARM_INIT_STEP = 0.01


def _torch():
    import torch
    return torch


def label_corpus(P, seed=TRAIN_SEED, device="cuda", group_jobs=150_000_000, tol=1e-6,
                 max_evals=300, job_cap=False, log=print):
    """Features (rows x 26) and targets (rows) of P generated problems, labelled
    by batched GPU solves; a problem the batch leaves above the tolerance is
    solved once more on its own from the batch's prices (ra_solve, whose
    repair of the lower bound closes the gaps that few jobs per resource
    leave), so that every problem is labelled.  Returns (X, Y, info) with X,
    Y FP32 device tensors; info counts the problems the second solve needed
    and any that still missed the tolerance (labelled with their best
    prices)."""
    torch = _torch()
    from . import ra
    from . import workloads as W
    sizes = W.warmstart_sizes(P, seed)
    Xs, Ys = [], []
    converged, solve_s, t0, k = 0, 0.0, time.time(), 0
    resolved = missed = 0
    while k < P:
        grp, jobs = [], 0
        while k < P and (not grp or jobs + sizes[k] <= group_jobs):
            grp.append(k)
            jobs += int(sizes[k])
            k += 1
        tensors = [W.hetero_device(int(sizes[i]), M, seed, i, device) for i in grp]
        B = ra.AllocationBatch.from_tensors(tensors, job_cap=job_cap)
        feats = B.features()
        t1 = time.time()
        infos, _ = B.solve(tol=tol, max_evals=max_evals)
        prices = B.prices.clone()
        for j, info in enumerate(infos):
            if info["status"] == ra.RA_OK:
                continue
            resolved += 1
            Pj = ra.AllocationProblem(*tensors[j], job_cap=job_cap)
            o = M * j
            sj = Pj.solve(tol=tol, max_evals=1000, lam0=prices[o:o + M], init_step=WARM_INIT_STEP)
            prices[o:o + M] = Pj.prices
            Pj.close()
            missed += sj["status"] != ra.RA_OK
        solve_s += time.time() - t1
        Xs.append(feats.clone())
        Ys.append(torch.log(prices + ra.RA_MLP_PRICE_OFFSET).float())
        converged += len(infos)
        B.close()
        del tensors, B, feats
        if log:
            log(f"labelled {k}/{P} problems ({resolved} solved again, {missed} above the "
                f"tolerance), {time.time() - t0:.0f} s")
    X = torch.cat(Xs)
    Y = torch.cat(Ys)
    return X, Y, {"problems": P, "labelled": converged, "solved_again": resolved,
                  "missed_tolerance": missed, "rows": int(X.shape[0]),
                  "solve_s": solve_s, "total_s": time.time() - t0}


def train(X, Y, epochs=60, rows_per_step=4096, lr=2e-3, seed=0, holdout=0.05, log=print):
    """Adam on the mean squared error of log prices, cosine-decayed learning
    rate; returns (net, history).  A fixed fraction of the problems (whole
    problems, M rows each) is held out to report the validation loss."""
    torch = _torch()
    from . import ra
    from . import workloads as W
    P = X.shape[0] // M
    rng = np.random.default_rng(seed)
    perm = rng.permutation(P)
    n_val = max(1, int(round(holdout * P)))
    val_p, tr_p = perm[:n_val], perm[n_val:]

    def to_rows(ps):
        idx = (ps[:, None] * M + np.arange(M)[None, :]).ravel()
        return torch.from_numpy(idx).to(X.device)

    Xv, Yv = X[to_rows(val_p)], Y[to_rows(val_p)]
    net = ra.WarmStartMLP(W.mlp_init(seed))
    hist = []
    steps_per_epoch = max(1, (len(tr_p) * M) // rows_per_step)
    total = epochs * steps_per_epoch
    step = 0
    for ep in range(epochs):
        rows = to_rows(rng.permutation(tr_p))
        losses = []
        for s in range(steps_per_epoch):
            idx = rows[s * rows_per_step:(s + 1) * rows_per_step]
            a = lr * 0.5 * (1.0 + math.cos(math.pi * step / total))
            losses.append(net.train_step(X[idx], Y[idx], max(a, 1e-6)))
            step += 1
        yv = net.forward(Xv)
        val = float(torch.mean((yv - Yv) ** 2).item())
        tr = float(torch.stack(losses).mean().item())
        hist.append({"epoch": ep + 1, "train_mse": tr, "val_mse": val})
        if log and (ep % 10 == 9 or ep == epochs - 1):
            log(f"epoch {ep + 1}: train mse {tr:.5f}  held-out mse {val:.5f}")
    return net, hist


def evaluate(net, P=1000, seed=EVAL_SEED, device="cuda", tol=1e-6, max_evals=3000, job_cap=False,
             log=print):
    """Cold and warm ra_solve of P held-out problems; per problem the device
    time (CUDA events on the solve's stream, the warm one including the
    statistics, the network and both start-point evaluations) and the
    evaluation count.  The cold start is the paper's Eq. e-initialization;
    the library's default (those prices scaled by the minimiser of g along
    their ray) is solved too, for comparison.  The order of the cold and warm
    solves alternates, so neither always finds the problem's data in L2."""
    torch = _torch()
    from . import ra
    from . import workloads as W
    sizes = W.warmstart_sizes(P, seed)
    rec = []
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return out, e0.elapsed_time(e1)

    for i in range(P):
        A, kind, w, param, R = W.hetero_device(int(sizes[i]), M, seed, i, device)
        prob = ra.AllocationProblem(A, kind, w, param, R, job_cap=job_cap)

        def cold():   # the paper's Eq. e-initialization, unscaled
            return prob.solve(tol=tol, max_evals=max_evals, init_scale=False)

        def cold_scaled():   # the library's default cold start: Eq. e-initialization
            return prob.solve(tol=tol, max_evals=max_evals)   # scaled along its ray

        def warm():   # nothing waits for the start-price choice
            lam0, _ = prob.warm_prices(net, sync=False)
            return prob.solve(tol=tol, max_evals=max_evals, lam0=lam0, init_step=WARM_INIT_STEP)

        if i % 2 == 0:
            ci, ct = timed(cold)
            wi, wt = timed(warm)
        else:
            wi, wt = timed(warm)
            ci, ct = timed(cold)
        used = prob.warm_used()
        si, sct = timed(cold_scaled)
        rec.append({"n": int(sizes[i]), "cold_ms": ct, "warm_ms": wt, "cold_evals": ci["evals"],
                    "warm_evals": wi["evals"], "cold_status": ci["status"],
                    "warm_status": wi["status"], "cold_gap": ci["rel_gap"], "warm_gap": wi["rel_gap"],
                    "used_warm": bool(used), "cold_scaled_ms": sct, "cold_scaled_evals": si["evals"],
                    "cold_scaled_status": si["status"]})
        prob.close()
        if log and (i + 1) % 100 == 0:
            log(f"evaluated {i + 1}/{P}")
    return rec


def summarize(rec):
    med = lambda key, rs: statistics.median(r[key] for r in rs)
    both = [r for r in rec if r["cold_status"] == 0 and r["warm_status"] == 0]
    out = {
        "problems": len(rec),
        "cold": {"median_ms": med("cold_ms", rec), "median_evals": med("cold_evals", rec),
                 "converged": sum(r["cold_status"] == 0 for r in rec)},
        "warm": {"median_ms": med("warm_ms", rec), "median_evals": med("warm_evals", rec),
                 "converged": sum(r["warm_status"] == 0 for r in rec),
                 "used_network_prices": sum(r["used_warm"] for r in rec)},
    }
    out["speedup_median_time"] = out["cold"]["median_ms"] / out["warm"]["median_ms"]
    out["speedup_median_evals"] = out["cold"]["median_evals"] / out["warm"]["median_evals"]
    if rec and "cold_scaled_ms" in rec[0]:
        # the library's default cold start (Eq. e-initialization scaled by the
        # minimiser of g along its ray, one more pass) for comparison
        out["cold_scaled"] = {"median_ms": med("cold_scaled_ms", rec),
                              "median_evals": med("cold_scaled_evals", rec),
                              "converged": sum(r["cold_scaled_status"] == 0 for r in rec)}
        out["speedup_vs_scaled_cold_time"] = out["cold_scaled"]["median_ms"] / out["warm"]["median_ms"]
    if both:
        out["both_converged"] = {
            "problems": len(both),
            "speedup_median_time": med("cold_ms", both) / med("warm_ms", both),
            "median_ratio_time": statistics.median(r["cold_ms"] / r["warm_ms"] for r in both),
            "speedup_median_evals": med("cold_evals", both) / med("warm_evals", both)}
    return out


def load(path=WEIGHTS, stream=None):
    from . import ra
    return ra.WarmStartMLP(np.load(path).astype(np.float32), stream)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "evaluate"])
    ap.add_argument("--problems", type=int, default=None)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--report", default=None, help="write a JSON summary here")
    ap.add_argument("--job-cap", action="store_true", help="problems with 1^T x_i <= 1")
    ap.add_argument("--max-evals", type=int, default=None,
                    help="evaluation limit (default: 300 for the batched labelling, 500 per "
                         "held-out solve)")
    args = ap.parse_args(argv)
    torch = _torch()
    from . import build
    build.build()
    if args.cmd == "train":
        X, Y, info = label_corpus(args.problems or 20000, job_cap=args.job_cap,
                                  max_evals=args.max_evals or 300)
        print(json.dumps(info), flush=True)
        t0 = time.time()
        net, hist = train(X, Y, epochs=args.epochs)
        torch.cuda.synchronize()
        info["train_s"] = time.time() - t0
        np.save(args.out, net.params())
        report = {"corpus": info, "history": hist}
    else:
        net = load(args.weights)
        rec = evaluate(net, P=args.problems or 1000, job_cap=args.job_cap,
                       max_evals=args.max_evals or 3000)
        report = summarize(rec)
        report["per_problem"] = rec
    print(json.dumps({k: v for k, v in report.items() if k not in ("per_problem", "history")}),
          flush=True)
    if args.report:
        with open(args.report, "w") as f:
            json.dump(report, f)
    return 0


if __name__ == "__main__":
    sys.exit(main())
