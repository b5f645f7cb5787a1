"""The feasible allocation with tie-aware repair (ra_recover_feasible) and its
use inside ra_solve, against the FP64 oracle, through the C ABI.

Checked from the returned allocation itself (FP32 outputs summed in FP64):
usage <= R_j (1 + 1e-6), the reported utility equals the oracle's utility of
that allocation, weak duality against the oracle's optimum, and -- at the
solver's best prices -- a primal objective within 1e-6 of the optimum.
"""
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


def check_allocation(O, prob, out, dense=False):
    """Feasibility and utility of a returned allocation, in FP64."""
    jk = out["jk"].cpu().numpy()
    xk = out["xk"].cpu().numpy()
    info = out["info"]
    U, usage, t = O.sparse_allocation_check(prob, jk, xk)
    assert np.all(xk.reshape(-1, 4)[jk.reshape(-1, 4) >= 0] >= 0)
    assert np.all(usage <= prob.R * (1 + 1e-6) + 1e-12), usage / prob.R
    assert info["max_usage_over_R"] <= 1 + 1e-6
    assert info["U"] == pytest.approx(U, rel=1e-6, abs=1e-6)
    if dense:
        X = out["X"].cpu().numpy().reshape(prob.n, prob.m).astype(np.float64)
        Xs = np.zeros_like(X)
        rows = np.broadcast_to(np.arange(prob.n)[:, None], jk.reshape(-1, 4).shape)
        j4 = jk.reshape(-1, 4)
        sel = j4 >= 0
        np.add.at(Xs, (rows[sel], j4[sel]), xk.reshape(-1, 4)[sel])
        assert np.array_equal(X, Xs.astype(np.float32).astype(np.float64))
    return U, usage


@pytest.mark.parametrize("cap", [False, True])
def test_repair_at_optimal_prices_closes_the_gap(ra, oracle, cap):
    """Few jobs per resource: at the oracle's optimal prices the plain
    subproblem solutions overuse some resources; the re-mixed allocation is
    feasible and its utility is within 1e-6 of the optimum."""
    prob = W.config_hetero(n=20_000, m=16, seed=8) if not cap else \
        W.paper_medium(n=20_000, utility="log", seed=2)
    ref = oracle.solve(prob, cap=cap, tol=1e-9, max_evals=3000)
    assert ref.converged
    P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=cap)
    # with the cap the jobs at ties of the medium problem sit at hull kinks a
    # little further from a tie (margins up to about 5e-3)
    out = P.recover_feasible(ref.lam, dense=True, tie_rel=1e-2 if cap else 1e-3)
    P.close()
    U, _ = check_allocation(oracle, prob, out, dense=True)
    assert U <= ref.g + 1e-9 * abs(ref.g)                      # weak duality
    assert (ref.g - U) / max(abs(ref.g), 1.0) <= 1e-6, (ref.g, U, out["info"])
    assert out["info"]["n_flex"] >= 1


def test_solve_repairs_a_stalled_lower_bound(ra, oracle):
    """Without the cap and with about 1250 jobs per resource the column-scaled
    bound stalls near 1e-5; the solve leaves the device loop, repairs the
    bound at its best prices and stops at the tolerance, certified by the
    oracle on the returned allocation."""
    prob = W.config_hetero(n=20_000, m=16, seed=8)
    P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=False)
    info = P.solve(tol=1e-6, max_evals=500)
    assert info["status"] == ra.RA_OK and info["rel_gap"] <= 1e-6, info
    assert info["repairs"] >= 1
    theta, lams, scaled = P.certificate()
    repaired = None
    if 2 in list(scaled):
        out = P.recover_feasible(lams[0])
        check_allocation(oracle, prob, out)
        repaired = (out["jk"].cpu().numpy(), out["xk"].cpu().numpy())
    c = oracle.certify(prob, P.prices.cpu().numpy(), theta, lams, scaled, False, repaired=repaired)
    assert c["rel_gap"] <= 1e-6 and c["max_usage_over_R"] <= 1 + 1e-6, c
    # with repairs switched off the same solve stalls
    off = P.solve(tol=1e-6, max_evals=300, repair_window=0)
    P.close()
    assert off["status"] == ra.RA_ENOTCONV and off["repairs"] == 0


def test_repair_at_any_prices_is_feasible(ra, oracle):
    """Away from the optimum the LP cannot remove all overuse; the column
    scaling takes out the rest, so the allocation is still feasible and its
    utility is a valid lower bound."""
    prob = W.random_small(50_000, 8, seed=4, r_scale=0.3)
    lam = W.random_prices(8, seed=5, lo=0.3, hi=3.0)
    for cap in (True, False):
        P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=cap)
        out = P.recover_feasible(lam, tie_rel=1e-2, max_flex=256)
        P.close()
        U, _ = check_allocation(oracle, prob, out)
        ref = oracle.solve(prob, cap=cap, tol=1e-8, max_evals=2000)
        assert U <= ref.g + 1e-9 * abs(ref.g)
        assert out["info"]["n_flex"] <= 256


def test_repair_rejects_bad_options(ra):
    prob = W.random_small(1000, 4, seed=1)
    P = ra.AllocationProblem.from_numpy(prob, "cuda")
    lam = torch.ones(4, dtype=torch.float64, device="cuda")
    for kw in (dict(tie_rel=0.0), dict(tie_rel=2.0), dict(max_flex=0), dict(max_flex=5000)):
        with pytest.raises(ra.RaError) as e:
            P.recover_feasible(lam, **kw)
        assert e.value.status == ra.RA_EINVAL
    P.close()
