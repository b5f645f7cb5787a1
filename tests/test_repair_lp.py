"""The library's host LP solver (the dense bounded-variable simplex that the
allocation repair uses) against scipy's HiGHS, on the CPU.

The simplex source is compiled on its own into a test object that exports a
plain C entry point; libra.so itself does not export it.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest
from scipy.optimize import linprog

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2104_00282_gb300", "csrc", "ra_lp.cpp")


@pytest.fixture(scope="module")
def lp(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("lp") / "ra_lp_test.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-DRA_LP_TEST_EXPORT",
                    "-I" + os.path.dirname(SRC), SRC, "-o", out], check=True)
    L = ctypes.CDLL(out)
    P = ctypes.c_void_p
    L.ra_lp_test_solve.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P, ctypes.c_int, P, P]
    L.ra_lp_test_solve.restype = ctypes.c_int
    return L


def solve(L, A, b, c, ub, basis, max_iter=10_000):
    rows, cols = A.shape
    A = np.ascontiguousarray(A, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    c = np.ascontiguousarray(c, np.float64)
    ub = np.ascontiguousarray(ub, np.float64)
    basis = np.ascontiguousarray(basis, np.int32)
    x = np.zeros(cols)
    obj = np.zeros(1)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    st = L.ra_lp_test_solve(rows, cols, p(A), p(b), p(c), p(ub), p(basis), max_iter, p(x), p(obj))
    return st, x, float(obj[0])


@pytest.mark.parametrize("seed", range(12))
def test_inequality_lps_match_highs(lp, seed):
    """min c^T y, G y <= h, 0 <= y <= u (some u infinite), with slacks as the
    starting basis; bounded by construction (c >= 0 on unbounded columns)."""
    rng = np.random.default_rng(seed)
    m, k = int(rng.integers(2, 12)), int(rng.integers(2, 40))
    G = rng.uniform(-1, 1, (m, k))
    h = rng.uniform(0.1, 2.0, m)
    u = np.where(rng.random(k) < 0.6, rng.uniform(0.2, 3.0, k), np.inf)
    c = rng.uniform(-1, 1, k)
    c[np.isinf(u)] = np.abs(c[np.isinf(u)])
    A = np.hstack([G, np.eye(m)])
    st, x, obj = solve(lp, A, h, np.concatenate([c, np.zeros(m)]),
                       np.concatenate([u, np.full(m, np.inf)]), np.arange(k, k + m))
    ref = linprog(c, A_ub=G, b_ub=h, bounds=[(0, None if np.isinf(v) else v) for v in u],
                  method="highs")
    assert ref.status == 0 and st == 0
    assert obj == pytest.approx(ref.fun, rel=1e-9, abs=1e-10)
    y = x[:k]
    assert np.all(y >= -1e-12) and np.all(y <= u + 1e-12)
    assert np.all(G @ y <= h + 1e-9)


@pytest.mark.parametrize("seed", range(8))
def test_two_phase_repair_shaped_lps(lp, seed):
    """The repair's shape: rows  D theta + s - v = b  (rows with b < 0 are
    negated so that v starts basic), theta in [0, 1].  Phase 1 minimises the
    weighted overuse sum v_j / R_j; the result must equal HiGHS's minimum of
    the same objective."""
    rng = np.random.default_rng(100 + seed)
    m, k = int(rng.integers(2, 10)), int(rng.integers(3, 50))
    D = rng.uniform(-1, 1, (m, k)) * (rng.random((m, k)) < 0.4)
    b = rng.uniform(-1.0, 1.0, m)
    R = rng.uniform(0.5, 2.0, m)
    # columns: theta (k), s (m), v (m)
    A = np.hstack([D, np.eye(m), -np.eye(m)])
    neg = b < 0
    A[neg] *= -1
    rhs = np.abs(b)
    basis = np.where(neg, k + m + np.arange(m), k + np.arange(m))
    c = np.concatenate([np.zeros(k + m), 1.0 / R])
    ub = np.concatenate([np.ones(k), np.full(2 * m, np.inf)])
    st, x, obj = solve(lp, A, rhs, c, ub, basis)
    assert st == 0
    ref = linprog(c, A_eq=np.hstack([D, np.eye(m), -np.eye(m)]), b_eq=b,
                  bounds=[(0, 1)] * k + [(0, None)] * (2 * m), method="highs")
    assert ref.status == 0
    assert obj == pytest.approx(ref.fun, rel=1e-9, abs=1e-11)
    th = x[:k]
    assert np.all(th >= -1e-12) and np.all(th <= 1 + 1e-12)
    assert np.allclose(D @ th + x[k:k + m] - x[k + m:], b, atol=1e-9)
