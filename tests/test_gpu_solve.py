"""GPU price discovery (ra_solve, Algorithm 2 on the device) against the
FP64 CPU oracle.

At sizes the oracle solves in seconds: the GPU's certified relative duality
gap meets the tolerance, its bounds bracket the oracle's optimum, and the
prices agree.  The GPU's certificate is re-checked by the oracle: g at the
GPU's best prices and the column-scaled utility at the GPU's lower-bound
prices, both evaluated in FP64 on the CPU.
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


@pytest.fixture(scope="module")
def oracle():
    from oracle import oracle as O
    O.lib()
    return O


def certify(O, prob, P, cap=True):
    """Oracle-side certificate of the GPU's result (FP64): g at the GPU's best
    prices, and the utility of the GPU's lower-bound allocation -- the mixture
    sum_k theta_k X(lam_k) (column-scaled where flagged) rebuilt by the oracle
    and scaled once more by min(1, R/usage) to exact feasibility in FP64."""
    theta, lams, scaled = P.certificate()
    assert len(theta) >= 1 and abs(theta.sum() - 1.0) < 1e-9 and np.all(theta >= 0)
    repaired = None
    if 2 in list(scaled):   # the bound is a repaired allocation at lams[0]
        assert len(theta) == 1
        out = P.recover_feasible(lams[0])
        repaired = (out["jk"].cpu().numpy(), out["xk"].cpu().numpy())
    c = O.certify(prob, P.prices.cpu().numpy(), theta, lams, scaled, cap, repaired=repaired)
    # constraint violation of the GPU's allocation: <= 1e-6 R_j
    assert c["max_usage_over_R"] <= 1 + 1e-6, c["usage_over_R"]
    return c["g"], c["U_lb"], c["rel_gap"]


def price_err(lam, ref):
    return float(np.max(np.abs(lam - ref)) / max(np.max(np.abs(ref)), 1e-300))


# prices: "unique" -- the dual optimum is unique and sharp at this gap, prices
# within 1e-5; "sqrt" -- unique but smooth, error of order sqrt(gap); None --
# not unique (jobs at kinks or idle resources leave g flat in some direction)
@pytest.mark.parametrize("make,tol,fp64,prices,cap", [
    (lambda: W.config_hetero(n=200_000, m=8, seed=3), 1e-6, False, "unique", True),
    (lambda: W.config_large(n=200_000, m=32, seed=3), 1e-6, False, "unique", True),
    (lambda: W.random_small(100_000, 5, seed=8, r_scale=0.1), 1e-6, False, "sqrt", True),
    (lambda: W.config_plain_small(), 1e-9, True, None, True),
    (lambda: W.paper_medium(n=200_000, utility="target", seed=1), 1e-6, False, "sqrt", True),
    (lambda: W.random_small(100_000, 5, seed=8, r_scale=0.25), 1e-6, False, None, True),
    # without the cap: log, power and linear-with-cap jobs (the split column
    # scaling of the lower bound), FP32 and FP64 job math
    (lambda: W.config_large(n=150_000, m=32, seed=4), 1e-6, False, "sqrt", False),
    (lambda: W.config_large(n=200_000, m=8, seed=5), 1e-6, True, "sqrt", False),
    (lambda: W.config_hetero(n=150_000, m=16, seed=6), 1e-6, False, "sqrt", False),
    # few jobs per resource without the cap: the optimum needs jobs split
    # between tied resources, which only the repair of the lower bound finds
    (lambda: W.config_hetero(n=20_000, m=16, seed=8), 1e-6, False, "sqrt", False),
    (lambda: W.random_small(3_000, 8, seed=9, kinds=(0, 1, 2)), 1e-6, False, None, False),
    # alpha-fair utilities (power with p < 0), with and without the cap
    (lambda: W.alpha_fair(n=150_000, m=8, seed=5), 1e-6, False, "sqrt", False),
    (lambda: W.alpha_fair(n=150_000, m=8, seed=6), 1e-6, False, "sqrt", True),
], ids=["hetero-200k-m8", "large-200k-m32", "mixed-100k-m5", "plain-small-fp64",
        "paper-medium-target", "degenerate-100k-m5", "large-150k-m32-nocap",
        "large-200k-m8-nocap-fp64", "hetero-150k-m16-nocap", "hetero-20k-m16-nocap",
        "mixed-3k-m8-nocap", "alpha-fair-150k-m8-nocap", "alpha-fair-150k-m8-cap"])
def test_solve_matches_oracle(ra, oracle, make, tol, fp64, prices, cap):
    prob = make()
    P = ra.AllocationProblem.from_numpy(prob, "cuda", fp64_jobmath=fp64, job_cap=cap)
    info = P.solve(tol=tol, max_evals=800)
    assert info["status"] == ra.RA_OK, info
    assert info["rel_gap"] <= tol
    ref = oracle.solve(prob, cap=cap, tol=min(tol, 1e-8) * 0.1, max_evals=2000)
    # the GPU's own bounds bracket the oracle's optimum, up to the FP32
    # rounding of its per-job arithmetic (1e-6) or FP64 rounding
    slack = 1e-6 if not fp64 else 1e-11
    scale = max(abs(ref.g), 1.0)
    assert info["g"] >= ref.U_lb - slack * scale
    assert info["U_lb"] <= ref.g + slack * scale
    # the oracle certifies the GPU's result in FP64: the gap meets the tolerance
    # and the allocation's utility (the primal objective) is within the
    # tolerance of the optimum
    g, lb, gap = certify(oracle, prob, P, cap)
    assert gap <= tol, (g, lb, gap)
    assert ref.U_lb <= g + tol * scale            # the oracle's feasible point vs the GPU's g
    if ref.converged:
        assert (ref.g - lb) / scale <= tol, (ref.g, lb)
        assert g <= ref.g + tol * scale
    # prices: within 1e-5 where the dual optimum is unique and g has curvature
    # at this gap (with the cap, prices pinned by capped jobs); elsewhere the
    # price error of a point with dual gap eps is of order sqrt(eps) (g is
    # quadratic about a smooth minimiser) -- see the FP64 test below
    err = price_err(P.prices.cpu().numpy(), ref.lam)
    if prices is not None:
        assert err <= (1e-5 if prices == "unique" else 5e-3), err
    P.close()


def test_own_bound_matches_oracle(ra, oracle):
    """From 4e6 jobs without the cap the solver's lower bound is each
    evaluation's own bound, formed from its sums (r, r_lin, U(X)).  At the
    prices the certificate names, the oracle's FP64 form of that bound
    (own_lower_bound) and the exact utility of the same column-scaled
    allocation (lower_bound) bracket the GPU's U_lb, which sits on the
    former to FP32 rounding."""
    prob = W.config_large(n=4_200_000, m=32, seed=11)
    P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=False)
    info = P.solve(tol=1e-6, master_lb=False)
    assert info["status"] == ra.RA_OK, info
    theta, lams, scaled = P.certificate()
    P.close()
    assert len(theta) == 1 and scaled[0] == 1, (theta, scaled)
    own, _ = oracle.own_lower_bound(prob, lams[0])
    exact, _ = oracle.lower_bound(prob, lams[0], cap=False)
    scale = max(abs(info["g"]), 1.0)
    assert own - 1e-6 * scale <= info["U_lb"] <= exact + 1e-6 * scale, (own, info["U_lb"], exact)
    assert abs(info["U_lb"] - own) <= 1e-6 * scale, (own, info["U_lb"])


def test_large_solve_with_sampled_start(ra, oracle):
    """From about 2.5e6 jobs a cold start without the cap reads a strided
    sample of the tiles for Eq. e-initialization's direction and for the
    scale along its ray; the solve still meets the tolerance, certified by
    the oracle in FP64, in fewer evaluations than from the paper's unscaled
    start (full pass)."""
    prob = W.config_large(n=2_600_000, m=32, seed=7)
    P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=False)
    info = P.solve(tol=1e-6)
    assert info["status"] == ra.RA_OK, info
    g, lb, gap = certify(oracle, prob, P, cap=False)
    assert gap <= 1e-6, (g, lb, gap)
    paper = P.solve(tol=1e-6, init_scale=False)
    assert info["evals"] < paper["evals"], (info["evals"], paper["evals"])
    P.close()


def test_graph_and_host_loop_agree_bitwise(ra):
    prob = W.config_hetero(n=150_000, m=8, seed=4)
    P = ra.AllocationProblem.from_numpy(prob, "cuda")
    a = P.solve(tol=1e-7, use_graph=True)
    la = P.prices.cpu().numpy().copy()
    b = P.solve(tol=1e-7, use_graph=False)
    lb = P.prices.cpu().numpy().copy()
    c = P.solve(tol=1e-7, use_graph=True)
    lc = P.prices.cpu().numpy().copy()
    P.close()
    timing = ("eval_ms", "step_ms")
    a, b, c = ({k: v for k, v in i.items() if k not in timing} for i in (a, b, c))
    assert a == b == c
    assert np.array_equal(la, lb) and np.array_equal(la, lc)


def test_single_resource_closed_form(ra):
    n = 50_000
    rng = np.random.default_rng(1)
    A = rng.uniform(0.5, 1.0, (n, 1)).astype(np.float32)
    w = rng.uniform(0.5, 2.0, n).astype(np.float32)
    R = np.array([0.3 * w.astype(np.float64).sum() / 2.0])
    prob = W.Problem(A, np.zeros(n, np.uint8), w, np.zeros(n, np.float32), R)
    P = ra.AllocationProblem.from_numpy(prob, "cuda")
    info = P.solve(tol=1e-8)
    lam = P.prices.item()
    P.close()
    assert info["rel_gap"] <= 1e-8
    assert lam == pytest.approx(w.astype(np.float64).sum() / R[0], rel=1e-6)


def test_uncapped_fisher_market_spending(ra):
    prob = W.random_small(100_000, 6, seed=13, kinds=(0,))
    P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=False)
    info = P.solve(tol=1e-6, max_evals=800)
    lam = P.prices.cpu().numpy()
    P.close()
    assert info["status"] == ra.RA_OK, info
    assert float(lam @ prob.R) == pytest.approx(float(prob.w.astype(np.float64).sum()), rel=1e-5)


def test_subgradient_update_converges(ra, oracle):
    prob = W.config_hetero(n=50_000, m=4, seed=6)
    P = ra.AllocationProblem.from_numpy(prob, "cuda")
    info = P.solve(tol=1e-2, update="subgradient", max_evals=3000)
    P.close()
    assert info["status"] == ra.RA_OK and info["rel_gap"] <= 1e-2
    ref = oracle.solve(prob, tol=1e-8)
    assert info["U_lb"] <= ref.g * (1 + 1e-9) + 1e-9 and info["g"] >= ref.U_lb - 1e-6 * abs(ref.U_lb)


def test_warm_start_from_optimum_is_fast(ra):
    prob = W.config_hetero(n=100_000, m=8, seed=7)
    P = ra.AllocationProblem.from_numpy(prob, "cuda")
    cold = P.solve(tol=1e-6)
    warm = P.solve(tol=1e-6, lam0=P.prices)
    P.close()
    # from the optimum: the first evaluation's column-scaled bound is read by
    # the step after the next evaluation, so two evaluations is the floor
    assert warm["evals"] <= max(5, cold["evals"] // 2), (warm, cold)


def test_history_and_verbose_log(ra):
    prob = W.paper_code_example(n=100_000, m=4, seed=0)
    P = ra.AllocationProblem.from_numpy(prob, "cuda")
    info = P.solve(tol=1e-6)
    h = P.history()
    lines = P.verbose_log()
    P.close()
    assert len(h) == info["evals"]
    gaps = h[:, 3][np.isfinite(h[:, 3])]
    assert np.all(np.diff(gaps) <= 1e-15)            # best-so-far gap never increases
    assert lines[0].startswith("iteration 01 | utility=")
    assert "Converged" in lines[-1]


def test_not_converged_is_reported(ra):
    prob = W.config_large(n=50_000, m=32, seed=8)
    P = ra.AllocationProblem.from_numpy(prob, "cuda")
    info = P.solve(tol=1e-14, max_evals=3)
    P.close()
    assert info["status"] == ra.RA_ENOTCONV and info["evals"] == 3


@pytest.mark.parametrize("make,cap", [
    (lambda: W.config_hetero(n=100_000, m=8, seed=31), False),
    (lambda: W.config_hetero(n=60_000, m=16, seed=32), False),
    (lambda: W.random_small(80_000, 6, seed=33, kinds=(0, 1), r_scale=0.3), False),
    (lambda: W.config_hetero(n=100_000, m=8, seed=34), True),
], ids=["hetero-100k-m8-nocap", "hetero-60k-m16-nocap", "logpow-80k-m6-nocap", "hetero-100k-m8-cap"])
def test_prices_match_oracle_fp64(ra, oracle, make, cap):
    """Prices within 5e-5 relative of the oracle's where the dual optimum is
    unique (log and power utilities: strictly concave, so the prices of a
    Fisher-type market are unique).  The price error of a point whose dual
    value is eps above the minimum is of order sqrt(eps / curvature), so this
    needs a dual value within about 1e-12 of the minimum: FP64 per-job
    arithmetic, whose dual values are exact to about 1e-14.  The dual value
    at the GPU's prices, evaluated by the oracle, is checked against the
    oracle's minimum.  Certifying that gap also takes a lower bound as tight;
    where the solve reaches it, the oracle re-checks the certificate, and
    where ties at the optimum keep the bound above it (the kinked dual of
    few jobs per resource), the solve reports RA_ENOTCONV."""
    prob = make()
    P = ra.AllocationProblem.from_numpy(prob, "cuda", fp64_jobmath=True, job_cap=cap)
    info = P.solve(tol=1e-12, max_evals=3000)
    lam = P.prices.cpu().numpy()
    assert info["status"] in (ra.RA_OK, ra.RA_ENOTCONV), info
    if info["status"] == ra.RA_OK:
        _, _, scaled = P.certificate()
        g, lb, gap = certify(oracle, prob, P, cap)
        # a repaired allocation comes back in FP32 (the solver's bound is its
        # FP64 utility): the oracle re-checks it to that precision
        assert gap <= (1e-8 if 2 in list(scaled) else 1e-12), (g, lb, gap)
    P.close()
    ref = oracle.solve(prob, cap=cap, tol=1e-13, max_evals=4000)
    big = ref.lam > 1e-3 * ref.lam.max()
    rel = np.abs(lam - ref.lam) / np.where(big, ref.lam, ref.lam.max())
    assert rel.max() <= 5e-5, (rel.max(), info, ref.gap)
    g_gpu, _, _ = oracle.dual(prob, lam, cap=cap)
    assert g_gpu - ref.g <= 5e-12 * max(abs(ref.g), 1.0), (g_gpu, ref.g)


@pytest.mark.parametrize("update", ["lbfgs-diag", "lbfgs-scalar"])
def test_initial_matrix_choices_are_certified(ra, oracle, update):
    """Both initial inverse Hessians of the L-BFGS update (the diagonal
    lambda_j / r_j and the scalar s^T y / y^T y) reach the tolerance, and the
    oracle certifies the result; without the per-job cap the diagonal one
    takes fewer evaluations."""
    prob = W.config_large(n=150_000, m=32, seed=4)
    P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=False)
    info = P.solve(tol=1e-6, max_evals=800, update=update)
    assert info["status"] == ra.RA_OK, info
    g, lb, gap = certify(oracle, prob, P, cap=False)
    assert gap <= 1e-6, (g, lb, gap)
    if update == "lbfgs-diag":
        other = P.solve(tol=1e-6, max_evals=800, update="lbfgs-scalar")
        assert info["evals"] < other["evals"], (info, other)
    P.close()


def test_unknown_update_is_rejected(ra):
    prob = W.config_hetero(n=5_000, m=4, seed=2)
    P = ra.AllocationProblem.from_numpy(prob, "cuda")
    o = ra.ra_solve_opts_default()
    o.update = 7
    lam = torch.empty(prob.m, dtype=torch.float64, device="cuda")
    with pytest.raises(ra.RaError, match="update"):
        ra.ra_solve(P.handle, lam, opts=o)
    P.close()


@pytest.mark.parametrize("per_resource", [False, True], ids=["scalar-demand", "vector-demand"])
def test_demand_scaling_and_solve(ra, oracle, per_resource):
    """Per-job demands (Section 7.1) without the per-job cap: the library's
    scaling A / d equals NumPy's IEEE division bit for bit, and the solve of
    the scaled problem is certified by the oracle at the stated tolerance."""
    prob = W.config_hetero(n=100_000, m=8, seed=21)
    rng = np.random.default_rng(5)
    d = rng.uniform(0.5, 3.0, (prob.n, prob.m) if per_resource else prob.n).astype(np.float32)
    A = torch.from_numpy(prob.A).cuda()
    As = ra.ra_scale_by_demand(A, torch.from_numpy(d).cuda())
    ref = (prob.A / (d if per_resource else d[:, None])).astype(np.float32)
    assert np.array_equal(As.cpu().numpy(), ref)
    scaled = W.Problem(ref, prob.kind, prob.w, prob.param, prob.R)
    P = ra.AllocationProblem(As, torch.from_numpy(prob.kind).cuda(), torch.from_numpy(prob.w).cuda(),
                             torch.from_numpy(prob.param).cuda(), torch.from_numpy(prob.R).cuda(),
                             job_cap=False)
    info = P.solve(tol=1e-6)
    assert info["status"] == ra.RA_OK, info
    g, lb, gap = certify(oracle, scaled, P, cap=False)
    assert gap <= 1e-6, (g, lb, gap)
    P.close()
