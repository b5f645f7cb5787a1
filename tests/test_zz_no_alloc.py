"""The allocation-free dual evaluation (ra_eval_dual_static) against the
regular entry point (ra_eval_dual), through the C ABI.

Callers that cannot allocate device memory -- serving loops that forbid
allocation (cudaMalloc may synchronise the device), hosts whose framework
owns all device memory through its own pool -- use ra_eval_dual_static,
whose scratch is a static array in the library.  The two entry points run
the same kernel with the same launch shape, so their results must agree bit
for bit, on two calls in a row that share the array.  This file is
collected last on purpose; it must pass alone in a fresh process and after
every other test.
"""
import ctypes

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


def _static_call(ra, A, kind, w, par, R, lam, flags):
    """Marshal straight onto the exported C symbol."""
    n, m = A.shape
    g = torch.empty(1, dtype=torch.float64, device="cuda")
    q = torch.empty(m, dtype=torch.float64, device="cuda")
    st = ra.lib().ra_eval_dual_static(
        ctypes.c_int64(n), ctypes.c_int32(m), ctypes.c_void_p(A.data_ptr()),
        ctypes.c_void_p(kind.data_ptr()), ctypes.c_void_p(w.data_ptr()),
        ctypes.c_void_p(par.data_ptr()), ctypes.c_void_p(R.data_ptr()),
        ctypes.c_void_p(lam.data_ptr()), ctypes.c_uint32(flags),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
        ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(q.data_ptr()))
    assert st == 0, ra.lib().ra_last_error().decode()
    return g, q


@pytest.mark.parametrize("n,m,cap", [(300_007, 32, True), (123_457, 8, False), (1000, 5, True)])
def test_static_scratch_matches_regular_entry_point(ra, n, m, cap):
    prob = W.random_small(n, m, seed=n % 97, r_scale=0.3)
    dev = "cuda"
    A = torch.from_numpy(prob.A).to(dev)
    kind = torch.from_numpy(prob.kind).to(dev)
    w = torch.from_numpy(prob.w).to(dev)
    par = torch.from_numpy(prob.param).to(dev)
    R = torch.from_numpy(prob.R).to(dev)
    flags = 0 if cap else ra.RA_NO_JOB_CAP
    P = ra.AllocationProblem(A, kind, w, par, R, job_cap=cap)
    for call in range(2):                              # two calls in a row share the array
        lam = torch.tensor(W.random_prices(m, seed=call, lo=0.3, hi=3.0), dtype=torch.float64,
                           device=dev)
        g_ref, q_ref, _ = P.eval_dual(lam)
        g, q = _static_call(ra, A, kind, w, par, R, lam, flags)
        torch.cuda.synchronize()
        g, q, g_ref, q_ref = g.item(), q.cpu().numpy(), g_ref.item(), q_ref.cpu().numpy()
        # the same kernel, launch shape and fixed reduction order: the same bits
        assert g == g_ref
        assert np.array_equal(q, q_ref)
    P.close()


def test_static_timeout_shows_as_nan(ra):
    """The call returns before its work is done, so an expired device wait
    cannot be returned as RA_ETIMEOUT; g and q become NaN instead.  A zero
    wait timeout makes every wait give up at once; the next call with the
    default timeout is complete again."""
    prob = W.random_small(200_003, 16, seed=5, r_scale=0.3)
    dev = "cuda"
    A, kind, w, par, R = (torch.from_numpy(x).to(dev) for x in
                          (prob.A, prob.kind, prob.w, prob.param, prob.R))
    lam = torch.tensor(W.random_prices(16, seed=3), dtype=torch.float64, device=dev)
    try:
        ra.ra_set_wait_timeout(0.0)
        g, q = _static_call(ra, A, kind, w, par, R, lam, 0)
        torch.cuda.synchronize()
        assert np.isnan(g.item()) and np.all(np.isnan(q.cpu().numpy()))
    finally:
        ra.ra_set_wait_timeout(2.0)
    g, q = _static_call(ra, A, kind, w, par, R, lam, 0)
    torch.cuda.synchronize()
    assert np.isfinite(g.item()) and np.all(np.isfinite(q.cpu().numpy()))


def test_static_entry_point_rejects_bad_arguments(ra):
    A = torch.rand(64, 40, device="cuda")          # m beyond the maximum
    kind = torch.zeros(64, dtype=torch.uint8, device="cuda")
    w = torch.ones(64, device="cuda")
    par = torch.zeros(64, device="cuda")
    R = torch.ones(40, dtype=torch.float64, device="cuda")
    lam = torch.ones(40, dtype=torch.float64, device="cuda")
    g = torch.empty(1, dtype=torch.float64, device="cuda")
    q = torch.empty(40, dtype=torch.float64, device="cuda")
    st = ra.lib().ra_eval_dual_static(64, 40, ctypes.c_void_p(A.data_ptr()),
                                      ctypes.c_void_p(kind.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                      ctypes.c_void_p(par.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                                      ctypes.c_void_p(lam.data_ptr()), 0, None,
                                      ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(q.data_ptr()))
    assert st == ra.RA_EINVAL
    assert b"m = 40" in ra.lib().ra_last_error()
