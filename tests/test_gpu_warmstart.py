"""Warm-start kernels (statistics, MLP forward, back-propagation, Adam and the
start-price choice) against the FP64 oracle in oracle/warmstart.py.

* Statistics: the order statistics are exact selections, so the GPU's
  logarithms match the oracle's to FP32 rounding; fractions and means match
  to FP32 rounding of FP64 sums.  Sizes cover n = 1, n below one 1024-thread
  pass, n just below and above the 16384-row sample, and zeros in A.
* Forward: FP32 against FP64 on rows spanning several 64-row tiles and a
  ragged tail.
* Gradient: every parameter tensor of one training step against the
  oracle's back-propagation, relative to the tensor's largest entry.
* Adam: parameters after several steps against the oracle's Adam run on the
  oracle's own gradients, and each step entry by entry against the oracle's
  Adam applied to the gradient the GPU step used.
* The committed network: on held-out problems its prices are kept and warm
  solves take at most 0.6 times the cold evaluations (median).
* Start prices: the choice between the network's prices and Eq.
  e-initialization follows the oracle's dual values.
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
def WS():
    from oracle import warmstart as M
    return M


def with_zeros(prob, frac=0.1, seed=0):
    rng = np.random.default_rng(seed)
    A = prob.A.copy()
    A[rng.random(A.shape) < frac] = 0.0
    A[:, 0] = np.maximum(A[:, 0], 0.05)       # keep a positive entry per row
    return W.Problem(A, prob.kind, prob.w, prob.param, prob.R)


FEAT_CASES = [
    (lambda: W.random_small(1, 4, seed=1), "n1"),
    (lambda: W.random_small(700, 3, seed=2), "n700"),
    (lambda: W.config_hetero(n=16_383, m=16, seed=3), "n16383"),
    (lambda: W.config_hetero(n=16_385, m=8, seed=4), "n16385"),
    (lambda: W.config_large(n=300_001, m=32, seed=5), "n300001"),
    (lambda: with_zeros(W.random_small(50_000, 5, seed=6)), "zeros"),
]


def check_features(WS, prob, f):
    ref = WS.features(prob.A, prob.kind, prob.w, prob.R)
    assert f.shape == ref.shape
    np.testing.assert_allclose(f, ref, rtol=2e-6, atol=2e-6)


@pytest.mark.parametrize("make,name", FEAT_CASES, ids=[c[1] for c in FEAT_CASES])
def test_features_match_oracle(ra, WS, make, name):
    prob = make()
    P = ra.AllocationProblem.from_numpy(prob, "cuda")
    f = P.features().cpu().numpy().astype(np.float64)
    P.close()
    check_features(WS, prob, f)


def test_batch_features_match_oracle(ra, WS):
    probs = [c[0]() for c in FEAT_CASES]
    B = ra.AllocationBatch(probs)
    f = B.features().cpu().numpy().astype(np.float64)
    B.close()
    off = 0
    for prob in probs:
        check_features(WS, prob, f[off:off + prob.m])
        off += prob.m


@pytest.mark.parametrize("rows", [1, 16, 200, 1000])
def test_forward_matches_oracle(ra, WS, rows):
    theta = W.mlp_init(seed=rows)
    X = np.random.default_rng(rows).normal(size=(rows, 26)).astype(np.float32)
    net = ra.WarmStartMLP(theta)
    y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    net.close()
    ref = WS.forward(theta.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(y, ref, rtol=1e-5, atol=1e-5 * (np.abs(ref).max() + 1))


@pytest.mark.parametrize("rows", [7, 300, 2000])
def test_gradients_match_oracle(ra, WS, rows):
    theta = W.mlp_init(seed=100 + rows)
    rng = np.random.default_rng(rows)
    X = rng.normal(size=(rows, 26)).astype(np.float32)
    t = rng.normal(size=rows).astype(np.float32)
    net = ra.WarmStartMLP(theta)
    loss = net.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), 1e-3)
    g = net.grads().astype(np.float64)
    net.close()
    L, ref = WS.loss_and_grads(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert float(loss.item()) == pytest.approx(L, rel=1e-5)
    off = 0
    for name, shape in WS.SHAPES:
        size = int(np.prod(shape))
        a, b = g[off:off + size], ref[off:off + size]
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= 2e-5 * scale + 1e-9, (name, np.abs(a - b).max(), scale)
        off += size


def test_adam_steps_match_oracle(ra, WS):
    theta0 = W.mlp_init(seed=7)
    rng = np.random.default_rng(7)
    X = rng.normal(size=(256, 26)).astype(np.float32)
    t = (np.tanh(X[:, 0]) - 0.5 * X[:, 1]).astype(np.float32)
    lr, steps = 1e-3, 8
    net = ra.WarmStartMLP(theta0)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    for _ in range(steps):
        net.train_step(Xd, td, lr)
    th_gpu = net.params().astype(np.float64)
    net.close()
    th = theta0.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for k in range(1, steps + 1):
        _, g = WS.loss_and_grads(th, X.astype(np.float64), t.astype(np.float64))
        th, m, v = WS.adam(th, g, m, v, k, lr)
    # each step moves a parameter by at most about lr; the two runs differ by
    # FP32 rounding of the gradients, which only matters where a gradient
    # component is near zero
    diff = np.abs(th_gpu - th)
    assert diff.max() <= 2 * steps * lr
    assert np.median(diff) <= 1e-3 * lr * steps
    L_gpu = WS.loss_and_grads(th_gpu, X.astype(np.float64), t.astype(np.float64))[0]
    L_ora = WS.loss_and_grads(th, X.astype(np.float64), t.astype(np.float64))[0]
    assert L_gpu == pytest.approx(L_ora, rel=1e-3)


def test_adam_update_is_elementwise(ra, WS):
    """Each Adam step, applied by the oracle to the gradient the GPU step used
    (ra_mlp_get_grads) and to the GPU's parameters before the step, gives the
    GPU's parameters after it, entry by entry, up to FP32 rounding."""
    theta0 = W.mlp_init(seed=5)
    rng = np.random.default_rng(5)
    X = rng.normal(size=(192, 26)).astype(np.float32)
    t = (np.tanh(X[:, 2]) + 0.3 * X[:, 5]).astype(np.float32)
    lr, steps = 3e-3, 6
    net = ra.WarmStartMLP(theta0)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    before = theta0.astype(np.float64)
    m = np.zeros_like(before)
    v = np.zeros_like(before)
    for k in range(1, steps + 1):
        net.train_step(Xd, td, lr)
        g = net.grads().astype(np.float64)
        after = net.params().astype(np.float64)
        want, m, v = WS.adam(before, g, m, v, k, lr)
        err = np.abs(after - want)
        bound = 1e-5 * lr + 2.5e-7 * np.abs(want)
        assert np.all(err <= bound), (k, int(np.argmax(err - bound)), float(err.max()))
        # and the step really moved the parameters where the gradient is not zero
        moved = np.abs(after - before)
        assert np.median(moved[np.abs(g) > 0]) > 0.1 * lr
        before = after
    net.close()


def test_committed_network_beats_the_cold_start(ra, WS):
    """The trained network shipped with the package, on held-out problems of
    its recipe (seed 1, never in the training corpus; no per-job cap): its
    prices beat Eq. e-initialization on g, and warm solves need far fewer
    evaluations than cold ones."""
    from paper_2104_00282_gb300 import warmstart
    net = warmstart.load()
    held_out = [(i, int(x)) for i, x in enumerate(W.warmstart_sizes(16, warmstart.EVAL_SEED))
                if x >= 30_000][:10]
    cold_e, warm_e, used_n = [], [], 0
    for i, n in held_out:
        A, kind, w, par, R = W.hetero_device(n, 16, warmstart.EVAL_SEED, i, "cuda")
        P = ra.AllocationProblem(A, kind, w, par, R, job_cap=False)
        cold = P.solve(tol=1e-6, max_evals=500, init_scale=False)
        lam0, used = P.warm_prices(net)
        warm = P.solve(tol=1e-6, max_evals=500, lam0=lam0, init_step=warmstart.WARM_INIT_STEP)
        P.close()
        assert cold["status"] == ra.RA_OK and warm["status"] == ra.RA_OK, (n, cold, warm)
        cold_e.append(cold["evals"])
        warm_e.append(warm["evals"])
        used_n += used
    net.close()
    assert used_n == len(held_out)
    assert np.median(warm_e) <= 0.6 * np.median(cold_e), (cold_e, warm_e)


def constant_net(ra, WS, log_price):
    """A network whose output is log_price for every input (W3 = 0, b3)."""
    P = {name: np.zeros(shape) for name, shape in WS.SHAPES}
    P["b3"][0] = log_price
    return ra.WarmStartMLP(WS.pack(P).astype(np.float32))


@pytest.mark.parametrize("cap", [True, False], ids=["job-cap", "no-job-cap"])
def test_start_price_choice_follows_oracle(ra, WS, oracle, cap):
    prob = W.config_hetero(n=60_000, m=8, seed=11)
    P = ra.AllocationProblem.from_numpy(prob, "cuda", job_cap=cap)
    lam_c = oracle.init_prices(prob, cap=cap)
    g_c = oracle.dual(prob, lam_c, cap=cap)[0]
    ref = oracle.solve(prob, cap=cap, tol=1e-7, max_evals=1000)
    seen = set()
    for price in (1e3, float(np.median(ref.lam[ref.lam > 0])) + 1e-3, float(lam_c.mean()) + 1e-3):
        net = constant_net(ra, WS, float(np.log(price)))
        lam0, used = P.warm_prices(net)
        lam0b, none = P.warm_prices(net, sync=False)   # the same choice, asked for later
        assert none is None and P.warm_used() == used
        assert torch.equal(lam0, lam0b)
        net.close()
        y = np.float64(np.float32(np.log(price)))
        lam_w = np.full(prob.m, max(np.exp(y) - 1e-3, 0.0))
        g_w = oracle.dual(prob, lam_w, cap=cap)[0]
        if abs(g_w - g_c) <= 1e-5 * abs(g_c):
            continue                               # too close to call in FP32
        assert used == (g_w < g_c), (price, g_w, g_c)
        seen.add(used)
        got = lam0.cpu().numpy()
        np.testing.assert_allclose(got, lam_w if used else lam_c, rtol=2e-5)
    P.close()
    assert False in seen                            # the fallback was exercised


def test_solve_reuses_the_warm_start_pass(ra):
    """ra_warmstart_prices' pass is also the first evaluation of a solve from
    the prices it returns: a solve called next with that buffer starts from
    it, and its result equals a solve from a copy of the same prices (which
    evaluates them itself) field by field."""
    from paper_2104_00282_gb300 import warmstart as WSG
    A, kind, w, param, R = W.hetero_device(120_000, 16, 7, 3, "cuda")
    P = ra.AllocationProblem(A, kind, w, param, R, job_cap=False)
    net = WSG.load()
    timing = ("eval_ms", "step_ms")
    lam0, used = P.warm_prices(net)
    assert used
    reused = {k: v for k, v in P.solve(tol=1e-6, lam0=lam0).items() if k not in timing}
    lam_r = P.prices.cpu().numpy().copy()
    plain = {k: v for k, v in P.solve(tol=1e-6, lam0=lam0.clone()).items() if k not in timing}
    lam_p = P.prices.cpu().numpy().copy()
    # anything run in between drops the reuse: the solve evaluates again
    lam0b, _ = P.warm_prices(net)
    P.eval_dual(lam0b)
    again = {k: v for k, v in P.solve(tol=1e-6, lam0=lam0b).items() if k not in timing}
    net.close()
    P.close()
    assert reused["status"] == ra.RA_OK
    assert reused == plain == again
    assert np.array_equal(lam_r, lam_p)
