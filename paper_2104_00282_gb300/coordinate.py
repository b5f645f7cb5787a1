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
    over resources with positive mean price, the step and whether the round's
    budgets were kept; the final prices (M x m) and budgets (the best
    found)."""
    n, m = A.shape
    bounds = sharded.shard_bounds(n, M)
    budgets = [(R / M).clone() for _ in range(M)]
    tensors = [(A[s:e], kind[s:e], w[s:e], param[s:e], budgets[k])
               for k, (s, e) in enumerate(bounds)]
    B = ra.AllocationBatch.from_tensors(tensors, job_cap=job_cap)
    R_tot = R.to(torch.float64).contiguous()
    hist = []
    lam0 = None
    # Moving budget towards the shards that price a resource higher is a
    # supergradient step on sum_k U_k(R_k) (primal decomposition).  With log
    # utilities a shard's price is inversely proportional to its budget, so
    # the step (lambda_k - pbar) / pbar of a share is Newton-like; a round
    # whose budgets lower the total utility is undone and the step halved,
    # and each kept round lengthens it again a little.
    best_U, best_budgets, best_lam = -math.inf, None, None
    try:
        for t in range(rounds):
            infos, _ = B.solve(tol=tol, max_evals=max_evals, lam0=lam0)
            lam = B.prices.clone()
            U = sum(i["U_lb"] for i in infos)
            P = lam.view(M, m)
            pbar = P.mean(0)
            pos = pbar > 1e-12 * float(pbar.max())
            spread = float(((P[:, pos] / pbar[pos]) - 1).abs().max()) if bool(pos.any()) else 0.0
            kept = U >= best_U
            hist.append({"round": t, "U_total": U, "g_shards": sum(i["g"] for i in infos),
                         "spread": spread, "step": step, "kept": kept,
                         "evals": sum(i["evals"] for i in infos),
                         "converged": sum(i["status"] == ra.RA_OK for i in infos)})
            if log:
                log(f"round {t}: U {U:.10e} spread {spread:.3e} step {step:.3g} "
                    f"{'kept' if kept else 'undone'}")
            if kept:
                best_U, best_lam = U, lam
                best_budgets = [b.clone() for b in budgets]
                step = min(1.0, 1.25 * step)
                if spread <= spread_tol:
                    break
            else:
                for b, bb in zip(budgets, best_budgets):
                    b.copy_(bb)
                step *= 0.5
            ra.ra_batch_rebalance(B.handle, best_lam, R_tot, step)
            lam0 = best_lam
        for b, bb in zip(budgets, best_budgets):
            b.copy_(bb)
        torch.cuda.synchronize()
        return {"history": hist, "prices": best_lam.view(M, m).clone(),
                "budgets": torch.stack([b.clone() for b in budgets]),
                "U_total": best_U, "bounds": bounds}
    finally:
        B.close()
