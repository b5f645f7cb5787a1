"""Small, self-contained workloads to run under a profiler (ncu).

    python -m paper_2104_00282_gb300.profile_targets eval  [--n N] [--m M] [--cap] [--reps K]
    python -m paper_2104_00282_gb300.profile_targets solve [--n N] [--m M] [--cap]
    python -m paper_2104_00282_gb300.profile_targets batch [--problems P]
    python -m paper_2104_00282_gb300.profile_targets warm  [--n N]

``eval`` runs K standalone dual evaluations (ra_eval_dual) at the Eq.
e-initialization prices of the large recipe; ``solve`` runs one solve with
the host-driven loop, so that every launch is a separate kernel the
profiler can see (inside a CUDA graph's conditional node it cannot);
``batch`` one batched solve of the batched workload's first P problems with
the host loop; ``warm`` one warm-started solve (statistics, network, start
prices, solve) of a held-out warm-start problem.
"""
from __future__ import annotations

import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["eval", "solve", "batch", "warm"])
    ap.add_argument("--n", type=int, default=2_000_000)
    ap.add_argument("--m", type=int, default=32)
    ap.add_argument("--cap", action="store_true")
    ap.add_argument("--reps", type=int, default=6)
    ap.add_argument("--problems", type=int, default=512)
    args = ap.parse_args(argv)
    import torch
    from . import build
    build.build()
    from . import ra
    from . import workloads as W
    if args.what in ("eval", "solve"):
        prob = W.config_large(n=args.n, m=args.m, seed=0)
        P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=args.cap)
        if args.what == "eval":
            lam = P.init_prices()
            for _ in range(args.reps):
                ra.ra_eval_dual(P.handle, lam)
            out = "evaluations"
        else:
            out = P.solve(tol=1e-6, max_evals=400, use_graph=False)
        P.close()
    elif args.what == "batch":
        n, m = W.batched_shapes(args.problems)
        probs = W.batched_workload(args.problems)
        B = ra.AllocationBatch(probs, job_cap=True)
        infos, _ = B.solve(tol=1e-6, max_evals=500, use_graph=False)
        out = f"{sum(i['status'] == 0 for i in infos)} of {len(infos)} converged"
        B.close()
    else:
        from . import warmstart as WS
        net = WS.load()
        A, kind, w, param, R = W.hetero_device(args.n, 16, WS.EVAL_SEED, 5, "cuda")
        P = ra.AllocationProblem(A, kind, w, param, R, job_cap=False)
        lam0, used = P.warm_prices(net)
        out = P.solve(tol=1e-6, max_evals=500, lam0=lam0, use_graph=False)
        P.close()
        net.close()
    torch.cuda.synchronize()
    print(args.what, out, flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
