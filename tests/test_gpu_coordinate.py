"""Price-coordinated shards (Section 7): M shards of one problem solved as a
batch, their budgets moved towards the shards with higher prices
(ra_batch_rebalance) until the prices agree -- compared with the FP64
oracle's solution of the whole problem."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2104_00282_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ra():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_00282_gb300 import build as B
    B.build()
    from paper_2104_00282_gb300 import ra as R
    R.lib()
    return R


def _sorted_problem(seed):
    """Heterogeneous-hardware jobs ordered by their efficiency on resource 1
    (priced in both cap modes), so that job-range shards differ and an even
    split of R is far from optimal (2-3 % of the optimum)."""
    p = W.config_hetero(n=120_000, m=8, seed=seed)
    order = np.argsort(p.A[:, 1], kind="stable")
    return W.Problem(np.ascontiguousarray(p.A[order]), p.kind[order].copy(), p.w[order].copy(),
                     p.param[order].copy(), p.R.copy())


@pytest.mark.parametrize("cap", [True, False])
def test_price_coordination_reaches_the_whole_problem(ra, oracle, cap):
    from paper_2104_00282_gb300 import coordinate
    prob = _sorted_problem(41)
    A, kind, w, par, R = (torch.from_numpy(x).to("cuda") for x in
                          (prob.A, prob.kind, prob.w, prob.param, prob.R))
    ref = oracle.solve(prob, cap=cap, tol=1e-9, max_evals=3000)
    out = coordinate.solve(A, kind, w, par, R, M=4, rounds=40, job_cap=cap, spread_tol=1e-4)
    h = out["history"]
    U0, U1 = h[0]["U_total"], out["U_total"]
    assert U1 == max(x["U_total"] for x in h)
    scale = abs(ref.g)
    # the shards' budgets always add up to R, so their allocations together
    # are feasible: a lower bound on the whole problem's optimum
    assert torch.allclose(out["budgets"].sum(0), R, rtol=1e-12, atol=0)
    assert bool((out["budgets"] >= 1e-3 * R / 4 * (1 - 1e-12)).all())
    assert all(np.isfinite(x["U_total"]) for x in h)
    assert U1 <= ref.g + 1e-9 * scale
    # the even split is measurably suboptimal; coordination closes most of it
    assert (ref.g - U0) / scale > 1e-5
    assert (ref.g - U1) / scale <= 5e-4, [(x["round"], x["U_total"], x["spread"]) for x in h]
    assert (ref.g - U1) <= 0.05 * (ref.g - U0)
    kept = [x for x in h if x["kept"]]
    assert kept[-1]["spread"] < h[0]["spread"]
    # the shards' prices approach the whole problem's (the utility is flat in
    # the split of the most heterogeneous resource, whose price converges last)
    pbar = out["prices"].mean(0).cpu().numpy()
    big = ref.lam > 1e-3 * ref.lam.max()
    err = np.abs(pbar[big] / ref.lam[big] - 1)
    assert np.median(err) <= 2e-2 and err.max() <= 0.15, err


def _project_floor(y, total, fl):
    """Euclidean projection of y onto {x >= fl, sum x = total} (bisection on
    the shift tau in x = max(y - tau, fl), FP64)."""
    lo, hi = y.min() - total / len(y), y.max()
    for _ in range(200):
        tau = 0.5 * (lo + hi)
        if np.maximum(y - tau, fl).sum() > total:
            lo = tau
        else:
            hi = tau
    return np.maximum(y - 0.5 * (lo + hi), fl)


def test_rebalance_step_is_the_projected_price_step(ra):
    M, m = 5, 4
    rng = np.random.default_rng(3)
    R_tot = rng.uniform(100.0, 400.0, m)
    shares = rng.dirichlet(np.ones(M), size=m).T          # M x m, columns sum to 1
    shares[0, 2] = 0.0005                                   # a shard near the floor
    shares[:, 2] /= shares[:, 2].sum()
    budgets = shares * R_tot
    probs = [W.random_small(1000, m, seed=10 + k) for k in range(M)]
    tensors = []
    for k, p in enumerate(probs):
        t = [torch.from_numpy(x).to("cuda") for x in (p.A, p.kind, p.w, p.param)]
        tensors.append((*t, torch.from_numpy(budgets[k].copy()).to("cuda")))
    B = ra.AllocationBatch.from_tensors(tensors, job_cap=False)
    lam = rng.uniform(0.2, 2.0, (M, m))
    lam[:, 3] = 0.0                                         # an unpriced resource stays put
    step = 0.7
    ra.ra_batch_rebalance(B.handle, torch.from_numpy(lam.ravel()).to("cuda"),
                          torch.from_numpy(R_tot).to("cuda"), step)
    torch.cuda.synchronize()
    got = np.stack([t[4].cpu().numpy() for t in tensors])
    B.close()
    pbar = lam.mean(0)
    for j in range(m):
        d = (lam[:, j] - pbar[j]) / pbar[j] if pbar[j] > 0 else np.zeros(M)
        want = _project_floor(budgets[:, j] + step * d * R_tot[j] / M, R_tot[j], 1e-3 * R_tot[j] / M)
        assert np.allclose(got[:, j], want, rtol=0, atol=1e-9 * R_tot[j]), (j, got[:, j], want)
        assert abs(got[:, j].sum() - R_tot[j]) <= 1e-12 * R_tot[j]
