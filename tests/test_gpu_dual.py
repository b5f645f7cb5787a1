"""GPU parity of the dual evaluation, initialisation and primal recovery
against the FP64 CPU oracle, through the C ABI (libra.so).

What is compared:
* g(lambda) (continuous in lambda, so unique): relative to the magnitude
  sum |lambda_j R_j| + sum_i |h_i|, 2e-6 with FP32 per-job arithmetic, 1e-11
  with FP64.
* per job, where the oracle finds the optimum unique (no other cost-curve
  point within 1e-5 relative of the supporting line, and for lin-cap/target
  utilities no switch within 1e-5): the resources used and jstar exactly,
  t and x within 2e-5 relative.
* jobs with a near tie may legitimately pick another optimum: the GPU's
  allocation must then be optimal (its net utility within tolerance of the
  oracle's) -- r is rebuilt from the oracle's unique part plus the GPU's
  choice on near-tie jobs and must match the GPU's r to 2e-6 R_j.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2104_00282_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TIE = 1e-5          # allocation ambiguity: another cost-curve point this close to the segment
TIE_ARGMIN = 1e-6   # argmin exemption: the two best effective prices this close


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


def _u(kind, w, p, t):
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(kind == 0, w * np.log(t),
               np.where(kind == 1, np.sign(p) * w * np.power(np.maximum(t, 0), p),
               np.where(kind == 2, w * np.minimum(t, p), w * np.minimum(t - p, 0.0))))


def dense_rows(n, m, j12, x12):
    X = np.zeros((n, m))
    rows = np.arange(n)
    for c in (0, 1):
        j = j12[c::2]
        x = x12[c::2]
        sel = j >= 0
        np.add.at(X, (rows[sel], j[sel]), x[sel])
    return X


def _canon(j, t):
    """Records list (P, Q) with P = -1 for the origin: move used resources first."""
    j = j.copy()
    t = t.copy()
    sw = (j[:, 0] < 0) & (j[:, 1] >= 0)
    j[sw] = j[sw][:, ::-1]
    t[sw] = t[sw][:, ::-1]
    return j, t


def compare_eval(ra, O, prob, lam, cap=True, fp64=False, check_lb=True):
    P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=cap, fp64_jobmath=fp64)
    try:
        g, q, U = P.eval_dual(lam, lower_bound=True)
        je, te = P.eval_records()
        rec = P.recover(lam)
        torch.cuda.synchronize()
        g = g.item()
        U = U.item()
        q = q.cpu().numpy()
        je = je.cpu().numpy().astype(np.int64).reshape(-1, 2)
        te = te.cpu().numpy().astype(np.float64).reshape(-1, 2)
        j12 = rec["j12"].cpu().numpy().astype(np.int64)
        x12 = rec["x12"].cpu().numpy().astype(np.float64)
        t_gpu = rec["t"].cpu().numpy().astype(np.float64)
        jstar = rec["jstar"].cpu().numpy()
    finally:
        P.close()
    n, m = prob.n, prob.m
    rows = np.arange(n)
    ora = O.jobs(prob, lam, cap=cap)
    lam = np.asarray(lam, np.float64)
    A = prob.A.astype(np.float64)
    kind, w, par = prob.kind, prob.w.astype(np.float64), prob.param.astype(np.float64)
    amb = (ora[:, 8] < TIE) | (ora[:, 9] < TIE)
    amb_ratio = ora[:, 7] < TIE_ARGMIN
    # t within the FP32 arithmetic's reach of a hull vertex: one side may keep a
    # sliver (< 1e-4) of the neighbouring resource; compare x, not the index set
    sliver = (ora[:, 4] >= 0) & (np.minimum(ora[:, 5], ora[:, 6]) < 1e-4)
    uniq = ~amb
    uniq_j = uniq & ~sliver
    # outputs are FP32: FP64 per-job arithmetic is still rounded once on output
    rt = 2e-7 if fp64 else 2e-5
    X_ora = np.zeros((n, m))
    for jc, xc in ((3, 5), (4, 6)):
        sel = ora[:, jc] >= 0
        X_ora[rows[sel], ora[sel, jc].astype(np.int64)] += ora[sel, xc]
    # the evaluation kernel's own choice (compact record: resources, throughputs)
    je, te = _canon(je, te)
    X_eval = np.zeros((n, m))
    for c in (0, 1):
        sel = je[:, c] >= 0
        X_eval[rows[sel], je[sel, c]] += te[sel, c] / A[rows[sel], je[sel, c]]
    assert np.array_equal(je[uniq_j, 0], ora[uniq_j, 3].astype(np.int64))
    assert np.array_equal(je[uniq_j, 1], ora[uniq_j, 4].astype(np.int64))
    tmask = ora[:, 9] >= TIE
    np.testing.assert_allclose(te.sum(1)[tmask & uniq], ora[tmask & uniq, 0], rtol=rt, atol=rt * 1e-3)
    # the recovery kernel: identical resources, close x (conditioned by the
    # segment: x = (t - a_P)/(a_Q - a_P)), close t, and jstar
    X_rec = dense_rows(n, m, j12, x12)
    assert np.array_equal(j12[0::2][uniq_j], ora[uniq_j, 3].astype(np.int64))
    assert np.array_equal(j12[1::2][uniq_j], ora[uniq_j, 4].astype(np.int64))
    j1, j2 = ora[:, 3].astype(np.int64), ora[:, 4].astype(np.int64)
    two = j2 >= 0
    kappa = np.ones(n)
    aP = A[rows[two], j1[two]]
    aQ = A[rows[two], j2[two]]
    kappa[two] = np.maximum(aP, aQ) / np.maximum(np.abs(aQ - aP), 1e-30)
    # x = (t - a_P)/(a_Q - a_P) amplifies t's error by kappa; t's FP32 error
    # reaches a few 1e-6 for power utilities (fast log/exp, exponent 1/(1-p))
    cond = (1e-15 if fp64 else 5e-6) * kappa
    lim = rt + rt * np.abs(X_ora) + cond[:, None]
    for X in (X_rec, X_eval):
        err = np.abs(X - X_ora)
        assert np.all(err[uniq] <= lim[uniq]), float((err[uniq] / lim[uniq]).max())
    np.testing.assert_allclose(t_gpu[tmask], ora[tmask, 0], rtol=rt, atol=rt * 1e-3)
    assert np.array_equal(jstar[~amb_ratio], ora[~amb_ratio, 2].astype(np.int64))
    # near ties: both kernels' allocations are optima of the job's subproblem
    if amb.any():
        for X in (X_eval, X_rec):
            Xa = X[amb]
            ta = (A[amb] * Xa).sum(1)
            ha = _u(kind[amb], w[amb], par[amb], ta) - Xa @ lam
            scale = np.abs(ora[amb, 1]) + np.abs(Xa @ lam) + 1.0
            assert np.all(ha >= ora[amb, 1] - rt * scale)
            if cap:
                assert np.all(Xa.sum(1) <= 1 + 1e-5)
    # r from the unique oracle part and the evaluation kernel's near-tie choices
    X_mix = np.where(amb[:, None], X_eval, X_ora)
    r_exp = X_mix.sum(0)
    r_gpu = prob.R - q
    tol_r = (1e-12 if fp64 else 2e-6) * np.maximum(np.maximum(prob.R, r_exp), 1.0)
    tol_r = tol_r + 2e-7 * X_eval[amb].sum(0)
    assert np.all(np.abs(r_gpu - r_exp) <= tol_r), (r_gpu, r_exp)
    # g is continuous: compare with the oracle directly
    g_ora = float(lam @ prob.R + ora[:, 1].sum())
    mag = float(np.abs(lam * prob.R).sum() + np.abs(ora[:, 1]).sum())
    assert abs(g - g_ora) <= (1e-11 if fp64 else 2e-6) * mag, (g, g_ora)
    if check_lb:
        r_lin = X_mix[kind >= 2].sum(0)
        s, s_lin = O.column_scales(prob.R, r_gpu, r_lin, cap)
        tt = (A * X_mix * np.where((kind >= 2)[:, None], s_lin[None, :], s[None, :])).sum(1)
        uu = _u(kind, w, par, tt)
        U_exp = float(uu.sum())
        if np.isinf(U_exp):      # a job left with no throughput: both -inf
            assert U == U_exp, (U, U_exp)
        else:
            assert abs(U - U_exp) <= (2e-7 if fp64 else 3e-6) * (np.abs(uu).sum() + 1.0), (U, U_exp)
    # the exempted argmin count is small (near ties of FP32-rounded ratios)
    # unless prices are zero, where free resources tie by construction
    if lam.min() > 0:
        assert int(amb_ratio.sum()) <= 10 + n // 1000, int(amb_ratio.sum())
    return dict(n_amb=int(amb.sum()), n_argmin_exempt=int(amb_ratio.sum()), g=g)


SHAPES = [(1, 4), (255, 3), (256, 8), (257, 32), (100_003, 1), (100_003, 4), (100_003, 5),
          (100_003, 8), (60_011, 13), (60_011, 16), (50_021, 17), (50_021, 32)]


@pytest.mark.parametrize("n,m", SHAPES)
@pytest.mark.parametrize("cap", [True, False])
def test_dual_eval_matches_oracle_fp32(ra, oracle, n, m, cap):
    prob = W.random_small(n, m, seed=n + m, r_scale=0.3)
    lam = W.random_prices(m, seed=m, lo=0.3, hi=3.0)
    compare_eval(ra, oracle, prob, lam, cap=cap)


@pytest.mark.parametrize("n,m", [(1000, 4), (3001, 8), (20_000, 13), (20_000, 32)])
@pytest.mark.parametrize("cap", [True, False])
def test_dual_eval_matches_oracle_fp64(ra, oracle, n, m, cap):
    prob = W.random_small(n, m, seed=7 * n + m)
    lam = W.random_prices(m, seed=m + 1)
    compare_eval(ra, oracle, prob, lam, cap=cap, fp64=True)


def test_zero_and_tiny_prices_with_cap(ra, oracle):
    prob = W.random_small(40_000, 8, seed=3)
    lam = W.random_prices(8, seed=4)
    lam[[1, 5]] = 0.0
    lam[2] = 1e-12
    compare_eval(ra, oracle, prob, lam, cap=True)
    lam[:] = 0.0                          # all free: every job takes its most efficient resource
    compare_eval(ra, oracle, prob, lam, cap=True)


def test_hetero_recipe_full_size(ra, oracle):
    prob = W.config_hetero(n=1_000_000, m=8, seed=0)
    lam = oracle.init_prices(prob)
    compare_eval(ra, oracle, prob, lam)
    compare_eval(ra, oracle, prob, lam * W.random_prices(8, seed=1, lo=0.7, hi=1.4))


@pytest.mark.parametrize("cap", [False, True])
def test_large_recipe_many_tiles_per_cta(ra, oracle, cap):
    """The large recipe at m = 32 with about ten 256-job tiles per CTA (and a
    ragged tail): every ring stage is reused and its mbarrier phase flips
    several times within one evaluation, as at n = 1e7."""
    prob = W.config_large(n=1_200_007, m=32, seed=12)
    lam = oracle.init_prices(prob, cap=cap)
    r = compare_eval(ra, oracle, prob, lam, cap=cap)
    assert r["n_argmin_exempt"] <= 200


@pytest.mark.parametrize("cap", [False, True])
@pytest.mark.parametrize("fp64", [False, True])
def test_alpha_fair_utilities(ra, oracle, cap, fp64):
    """Power utilities with p < 0 (-w t^p, alpha-fair with alpha = 1 - p in
    [1.5, 5]) beside log utilities."""
    prob = W.alpha_fair(n=60_011, m=8, seed=3)
    lam = oracle.init_prices(prob, cap=cap)
    compare_eval(ra, oracle, prob, lam * W.random_prices(8, seed=4, lo=0.7, hi=1.4), cap=cap,
                 fp64=fp64)


def test_plain_small_recipe_fp64(ra, oracle):
    prob = W.config_plain_small()
    lam = oracle.init_prices(prob)
    compare_eval(ra, oracle, prob, lam, fp64=True)


def test_init_prices_match_oracle(ra, oracle):
    for prob, cap in ((W.config_hetero(n=200_003, m=8, seed=5), True),
                      (W.random_small(50_000, 32, seed=6, r_scale=0.05), True),
                      (W.random_small(50_000, 5, seed=6, r_scale=0.5), False),
                      (W.config_plain_small(), True)):
        P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=cap)
        lam = P.init_prices().cpu().numpy()
        P.close()
        np.testing.assert_allclose(lam, oracle.init_prices(prob, cap=cap), rtol=2e-5)


def test_dual_eval_is_deterministic(ra):
    prob = W.config_large(n=300_000, m=32, seed=2)
    P = ra.AllocationProblem.from_numpy(prob, "cuda")
    lam = torch.tensor(W.random_prices(32, seed=9), dtype=torch.float64, device="cuda")
    outs = [tuple(x.cpu().numpy().copy() for x in P.eval_dual(lam, lower_bound=True)) for _ in range(3)]
    P.close()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


def test_near_tie_count_and_flags(ra, oracle):
    prob = W.random_small(30_000, 4, seed=12)
    # duplicate column 1 into column 2 with a doubled price: every job ties
    prob.A[:, 2] = prob.A[:, 1] * 2
    lam = np.array([5.0, 1.0, 2.0, 5.0])
    P = ra.AllocationProblem.from_numpy(prob, "cuda")
    rec = P.recover(lam)
    P.close()
    ora = oracle.jobs(prob, lam)
    flags = rec["near_tie"].cpu().numpy().astype(bool)
    assert rec["n_near_ties"] == int(flags.sum())
    assert np.all(flags[ora[:, 7] < 1e-7])
    assert not np.any(flags[ora[:, 7] > 1e-4])


def test_invalid_arguments_are_rejected(ra):
    dev = "cuda"
    A = torch.rand(100, 4, device=dev)
    kind = torch.zeros(100, dtype=torch.uint8, device=dev)
    w = torch.ones(100, device=dev)
    p = torch.zeros(100, device=dev)
    R = torch.full((4,), 10.0, dtype=torch.float64, device=dev)
    with pytest.raises(ra.RaError) as e:
        ra.ra_problem_create(A[:, :0].contiguous(), kind, w, p, R[:0])
    assert e.value.status == ra.RA_EINVAL
    A1 = torch.rand(101, 1, device=dev)
    with pytest.raises(ra.RaError) as e:
        ra.ra_problem_create(A1[1:], kind, w, p, R[:1])   # 4-byte offset: misaligned
    assert e.value.status == ra.RA_EINVAL
    for bad in ("A", "w", "p", "kind"):
        A2, w2, p2, k2 = A.clone(), w.clone(), p.clone(), kind.clone()
        if bad == "A":
            A2[3, 1] = -1.0
        elif bad == "w":
            w2[5] = 0.0
        elif bad == "p":
            k2[7] = ra.RA_U_POWER
            p2[7] = 1.5
        else:
            k2[9] = 9
        with pytest.raises(ra.RaError) as e:
            ra.ra_problem_create(A2, k2, w2, p2, R, ra.RA_VALIDATE)
        assert e.value.status == ra.RA_EINVAL
    h = ra.ra_problem_create(A, kind, w, p, R, ra.RA_VALIDATE)
    ra.ra_problem_destroy(h)


def test_expired_wait_is_reported(ra):
    """A bounded device wait that gives up (zero timeout: every wait expires
    at once) makes the evaluation's outputs NaN and the solve return
    RA_ETIMEOUT; with the default timeout the same problem solves again."""
    prob = W.random_small(100_003, 8, seed=21, r_scale=0.3)
    P = ra.AllocationProblem.from_numpy(prob, "cuda")
    lam = torch.tensor(W.random_prices(8, seed=22), dtype=torch.float64, device="cuda")
    try:
        ra.ra_set_wait_timeout(0.0)
        g, q, U = P.eval_dual(lam, lower_bound=True)
        torch.cuda.synchronize()
        assert np.isnan(g.item()) and np.all(np.isnan(q.cpu().numpy())) and np.isnan(U.item())
        with pytest.raises(ra.RaError) as e:
            P.solve(tol=1e-6, max_evals=50)
        assert e.value.status == ra.RA_ETIMEOUT
    finally:
        ra.ra_set_wait_timeout(2.0)
    info = P.solve(tol=1e-6, max_evals=200)
    P.close()
    assert info["status"] == ra.RA_OK
    with pytest.raises(ra.RaError):
        ra.ra_set_wait_timeout(-1.0)
