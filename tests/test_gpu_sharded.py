"""One problem split by job range (ra_eval_partial, ra_combine_partials,
ra_solve_sharded), emulated on one GPU: the shards run on separate streams,
driven by host threads that exchange their sums through host barriers (no
kernel waits on another).  Compared with the unsharded entry points and
certified by the FP64 oracle on the whole problem."""
import threading

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


def _device(prob):
    return [torch.from_numpy(x).to("cuda") for x in (prob.A, prob.kind, prob.w, prob.param, prob.R)]


@pytest.mark.parametrize("S", [1, 2, 3])
@pytest.mark.parametrize("cap", [False, True])
def test_partials_combine_to_the_whole_evaluation(ra, oracle, S, cap):
    from paper_2104_00282_gb300 import sharded
    prob = W.random_small(300_007, 16, seed=S, r_scale=0.3)
    A, kind, w, par, R = _device(prob)
    lam = torch.tensor(W.random_prices(16, seed=7, lo=0.3, hi=3.0), dtype=torch.float64,
                       device="cuda")
    width = ra.RA_SHARD_WIDTH(16)
    parts = torch.empty(S * width, dtype=torch.float64, device="cuda")
    for k, (s, e) in enumerate(sharded.shard_bounds(prob.n, S)):
        P = sharded.shard_problem(A, kind, w, par, R, s, e, job_cap=cap)
        ra.ra_eval_partial(P.handle, lam, parts[k * width:(k + 1) * width])
        torch.cuda.synchronize()
        P.close()
    g = torch.empty(1, dtype=torch.float64, device="cuda")
    q = torch.empty(16, dtype=torch.float64, device="cuda")
    ra.ra_combine_partials(parts, 16, lam, R, g, q)
    Pw = ra.AllocationProblem(A, kind, w, par, R, job_cap=cap)
    g1, q1, _ = Pw.eval_dual(lam)
    torch.cuda.synchronize()
    Pw.close()
    lam_h = lam.cpu().numpy()
    g_ora, r_ora, _ = oracle.dual(prob, lam_h, cap=cap)
    mag = float(np.abs(lam_h * prob.R).sum()) + abs(g_ora)
    assert abs(g.item() - g1.item()) <= 2e-7 * mag
    assert abs(g.item() - g_ora) <= 2e-6 * mag
    assert np.allclose(q.cpu().numpy(), q1.cpu().numpy(), rtol=0, atol=2e-6 * prob.R.max())
    if S == 1:      # one shard: the very same sums
        assert g.item() == g1.item()


@pytest.mark.parametrize("cap", [False, True])
def test_sharded_solve_two_shards_on_one_gpu(ra, oracle, cap):
    from paper_2104_00282_gb300 import sharded
    prob = W.config_hetero(n=400_000, m=8, seed=21)
    A, kind, w, par, R = _device(prob)
    world = 2
    tg = sharded.ThreadGather(world)
    bounds = sharded.shard_bounds(prob.n, world)
    out = [None] * world

    def run(rank):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                P = sharded.shard_problem(A, kind, w, par, R, *bounds[rank], job_cap=cap, stream=s)
                lam, info = sharded.solve(P, prob.n, rank, world, tg.for_rank(rank), tol=1e-6,
                                          max_evals=400)
                cert = P.certificate()
                out[rank] = (lam.cpu().numpy(), info, cert)
                P.close()
        except Exception as e:  # reported below
            out[rank] = e
            tg.barrier.abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    for o in out:
        assert not isinstance(o, Exception), o
    (l0, i0, c0), (l1, i1, c1) = out
    # every shard ran the same update on the same combined sums (only the
    # device timings differ)
    timing = ("eval_ms", "step_ms")
    assert np.array_equal(l0, l1)
    assert {k: v for k, v in i0.items() if k not in timing} == \
        {k: v for k, v in i1.items() if k not in timing}
    assert i0["status"] == ra.RA_OK and i0["rel_gap"] <= 1e-6, i0
    # the whole problem's certificate, rebuilt by the oracle
    theta, lams, scaled = c0
    c = oracle.certify(prob, l0, theta, lams, scaled, cap)
    assert c["rel_gap"] <= 1e-6 and c["max_usage_over_R"] <= 1 + 1e-6, c
    # and the unsharded solve reaches the same optimum
    Pw = ra.AllocationProblem(A, kind, w, par, R, job_cap=cap)
    info = Pw.solve(tol=1e-6, max_evals=400)
    Pw.close()
    scale = max(abs(info["g"]), 1.0)
    assert abs(info["g"] - i0["g"]) <= 2e-6 * scale
