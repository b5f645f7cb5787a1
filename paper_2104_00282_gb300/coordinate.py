"""Price-coordinated shards (Section 7 of arXiv 2104.00282).

A problem too large, or too spread out, to solve as one can be split into M
shards of jobs, each solved independently with a share R_k of the resources
(initially R / M).  The shards' optimal prices tell where resources are
worth more: moving budget from shards with low prices to shards with high
prices (ra_batch_rebalance) is a primal decomposition of the whole problem,
and it converges to the whole problem's solution; when the shards' prices
agree the split costs nothing.  The shards are one batch (ra_batch_solve),
re-solved warm from their previous prices after every rebalancing.
"""
from __future__ import annotations

import math

import torch

from . import ra
from . import sharded


def solve(A, kind, w, param, R, M, rounds=40, tol=1e-6, job_cap=True, step=1.0,
          spread_tol=1e-3, max_evals=500, log=None):
    """Split the problem given as device tensors into M job-range shards and
    coordinate their budgets.  Returns a dict: per round the total utility
    of the shards' feasible allocations (a lower bound on the whole
    problem's optimum), the price spread max_kj |lambda_kj / pbar_j - 1|
    over resources with positive mean price, and the budgets; the final
    prices (M x m) and budgets."""
    n, m = A.shape
    dev = A.device
    bounds = sharded.shard_bounds(n, M)
    budgets = [(R / M).clone() for _ in range(M)]
    tensors = [(A[s:e], kind[s:e], w[s:e], param[s:e], budgets[k])
               for k, (s, e) in enumerate(bounds)]
    B = ra.AllocationBatch.from_tensors(tensors, job_cap=job_cap)
    R_tot = R.to(torch.float64).contiguous()
    hist = []
    lam0 = None
    # With log utilities a shard's price is inversely proportional to its
    # budget, so moving (lambda_k - pbar) / pbar of a share is a Newton step;
    # the step is halved whenever the price spread fails to shrink.
    prev_spread = math.inf
    try:
        for t in range(rounds):
            infos, _ = B.solve(tol=tol, max_evals=max_evals, lam0=lam0)
            lam = B.prices.clone()
            P = lam.view(M, m)
            pbar = P.mean(0)
            pos = pbar > 1e-12 * float(pbar.max())
            spread = float(((P[:, pos] / pbar[pos]) - 1).abs().max()) if bool(pos.any()) else 0.0
            U = sum(i["U_lb"] for i in infos)
            g_sum = sum(i["g"] for i in infos)
            hist.append({"round": t, "U_total": U, "g_shards": g_sum, "spread": spread,
                         "evals": sum(i["evals"] for i in infos),
                         "converged": sum(i["status"] == ra.RA_OK for i in infos)})
            if log:
                log(f"round {t}: U {U:.10e} spread {spread:.3e}")
            if spread <= spread_tol:
                break
            if spread >= prev_spread:
                step *= 0.5
            prev_spread = spread
            ra.ra_batch_rebalance(B.handle, lam, R_tot, step)
            lam0 = lam
        torch.cuda.synchronize()
        return {"history": hist, "prices": B.prices.view(M, m).clone(),
                "budgets": torch.stack([b.clone() for b in budgets]),
                "bounds": bounds}
    finally:
        B.close()
