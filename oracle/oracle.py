"""FP64 CPU oracle for the dual price-discovery method (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It imports nothing from the product
package: problems arrive as plain numpy arrays.

The per-job arithmetic lives in ``ra_oracle.c`` (FP64, OpenMP over jobs);
this module adds the price-discovery loop of Section 5 (Algorithm 2):

* dual value and subgradient  g(lam), q = R - r          (Section 3)
* feasible lower bound by column scaling  U(X~)            (Section 5)
* a bound on U(X~) from the evaluation's sums alone (no per-job cap;
  t u'(t) = lambda_j x_ij at each job's optimum, Section 4.1)
* initial prices                                             (Eq. e-initialization)
* L-BFGS price updates with bounds lam >= 0 -- scipy's L-BFGS-B
  (memory 10) serves as the quasi-Newton step (Section 5, "More efficient
  price updates"; Section 6.1 uses L-BFGS with memory 10)
* the projected subgradient update  lam+ = max(lam - a_k q, 0)  (Section 5)
* stopping on the duality gap  g(lam) - U(X~) <= eps  (Algorithm 2, step 2),
  made relative:  (g_best - U_best) / max(|U_best|, |g_best|, 1).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import time

import numpy as np

from . import build as _build

NOUT = 10
_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        P = ctypes.c_void_p
        L.ora_version.restype = i32
        L.ora_max_threads.restype = i32
        L.ora_job.argtypes = [i32, P, P, i32, d, d, i32, i32, P]
        L.ora_job.restype = None
        L.ora_dual.argtypes = [i64, i32, P, P, P, P, P, P, i32, i32, P, P, P, P, i32]
        L.ora_dual.restype = i32
        L.ora_scaled_utility.argtypes = [i64, i32, P, P, P, P, P, P, P, i32, i32, P, i32]
        L.ora_scaled_utility.restype = i32
        L.ora_init.argtypes = [i64, i32, P, P, P, P, P, i32, P, i32]
        L.ora_init.restype = i32
        L.ora_jobs.argtypes = [i64, i32, P, P, P, P, P, i32, i32, i64, P, P, i32]
        L.ora_jobs.restype = i32
        L.ora_cost.argtypes = [i32, P, P, d, P]
        L.ora_cost.restype = d
        L.ora_dual_blocks.argtypes = [i64, i32, P, P, P, P, P, i32, i32, P, i32]
        L.ora_dual_blocks.restype = i32
        L.ora_mixture_utility.argtypes = [i64, i32, P, P, P, P, i32, P, P, P, P, i32, i32, P, i32]
        L.ora_mixture_utility.restype = i32
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _arrays(prob):
    A = np.ascontiguousarray(prob.A, dtype=np.float32)
    kind = np.ascontiguousarray(prob.kind, dtype=np.uint8)
    w = np.ascontiguousarray(prob.w, dtype=np.float32)
    par = np.ascontiguousarray(prob.param, dtype=np.float32)
    R = np.ascontiguousarray(prob.R, dtype=np.float64)
    return A, kind, w, par, R


def max_threads() -> int:
    return int(lib().ora_max_threads())


# --------------------------------------------------------------------------- per job

def job(a, lam, kind, w, par, cap=True, method="hull"):
    """One subproblem (Eq. e-subproblem) from FP64 data.  Returns a dict with
    t, h, jstar, j1, j2, x1, x2 and the tie margins."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    out = np.zeros(NOUT)
    lib().ora_job(len(a), _p(a), _p(lam), int(kind), float(w), float(par), int(bool(cap)),
                  0 if method == "hull" else 1, _p(out))
    return _record(out)


def cost(a, lam, t):
    """(c(t), x): the parametric LP of Section 4.1 solved on the lower hull."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    x = np.zeros(len(a))
    c = lib().ora_cost(len(a), _p(a), _p(lam), float(t), _p(x))
    return float(c), x


def _record(o):
    return dict(t=o[0], h=o[1], jstar=int(o[2]), j1=int(o[3]), j2=int(o[4]), x1=o[5], x2=o[6],
                tie_ratio=o[7], tie_seg=o[8], tie_t=o[9])


def jobs(prob, lam, idx=None, cap=True, method="hull", nthreads=0):
    """Per-job records (array (k, 10)) for rows ``idx`` (all rows if None)."""
    A, kind, w, par, _ = _arrays(prob)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    if idx is None:
        cnt, ip = prob.n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        cnt, ip = len(idx), _p(idx)
    out = np.zeros((cnt, NOUT))
    rc = lib().ora_jobs(prob.n, prob.m, _p(A), _p(kind), _p(w), _p(par), _p(lam), int(bool(cap)),
                        0 if method == "hull" else 1, cnt, ip, _p(out), nthreads)
    assert rc == 0
    return out


# --------------------------------------------------------------------------- dual

def dual(prob, lam, cap=True, method="hull", nthreads=0, split=False):
    """(g, r, U): dual value g(lam) = lam^T R + sum_i h_i, usage r = sum_i x_i
    and the utility U(X) of the unscaled subproblem solutions (Section 3).
    With split, also r_lin: the part of r used by jobs with a linear utility
    (kinds 2 and 3)."""
    A, kind, w, par, R = _arrays(prob)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    g = np.zeros(1)
    r = np.zeros(prob.m)
    U = np.zeros(1)
    r_lin = np.zeros(prob.m)
    rc = lib().ora_dual(prob.n, prob.m, _p(A), _p(kind), _p(w), _p(par), _p(R), _p(lam),
                        int(bool(cap)), 0 if method == "hull" else 1, _p(g), _p(r), _p(U),
                        _p(r_lin), nthreads)
    assert rc == 0
    if split:
        return float(g[0]), r, float(U[0]), r_lin
    return float(g[0]), r, float(U[0])


BLOCK = 4096   # jobs per partial sum of the oracle's evaluation


def dual_blocks(prob, lam, cap=True, method="hull", nthreads=0):
    """Per-block sums of the dual evaluation, blocks of BLOCK jobs in job
    order: rows (sum h_i, sum u_i(t_i), r[m], r_lin[m]).  ``dual`` adds these
    rows in block order."""
    A, kind, w, par, _ = _arrays(prob)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    nb = (prob.n + BLOCK - 1) // BLOCK
    part = np.zeros((max(nb, 1), 2 * prob.m + 2))
    rc = lib().ora_dual_blocks(prob.n, prob.m, _p(A), _p(kind), _p(w), _p(par), _p(lam),
                               int(bool(cap)), 0 if method == "hull" else 1, _p(part), nthreads)
    assert rc == 0
    return part[:nb]


def column_scale(R, r, cap=True):
    """Column scaling that makes X diag(s) feasible (Section 5).  With the
    per-job cap, s_j = min(1, R_j / r_j): the paper's scaling down of the
    over-used columns.  Without the cap nothing bounds a job's x_i, so the
    under-used columns are scaled up too, s_j = R_j / r_j (1 where r_j = 0):
    X diag(s) then uses exactly R, and to first order its utility gains
    sum_j lambda_j (R_j - r_j), the term by which g exceeds U(X)."""
    R = np.asarray(R, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    s = np.ones_like(R)
    sel = (r > R) if cap else (r > 0)
    s[sel] = R[sel] / r[sel]
    return s


def column_scales(R, r, r_lin, cap=True):
    """(s, s_lin): column scaling with a separate factor for the jobs with a
    linear utility.  With the per-job cap both are the paper's min(1, R/r).
    Without it, the linear-utility jobs sit at their target t = T, where
    more throughput adds nothing (and below which each unit is worth at
    least its price), so while they use less than R_j they keep their
    allocation, s_lin = 1, and the other jobs are scaled to the capacity
    left, s = (R - r_lin) / (r - r_lin); a column that the linear jobs alone
    fill, or nearly alone use (other jobs below 1e-3 r, where r - r_lin
    would lose its digits to rounding), is scaled uniformly, s = s_lin =
    R / r."""
    R = np.asarray(R, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    r_lin = np.asarray(r_lin, dtype=np.float64)
    if cap:
        s = column_scale(R, r, True)
        return s, s.copy()
    s = column_scale(R, r, False)
    s_lin = s.copy()
    r_oth = r - r_lin
    room = r_lin < R
    s_lin[room] = 1.0
    use = room & (r_oth > 1e-3 * r)
    s[use] = (R[use] - r_lin[use]) / r_oth[use]
    s_lin[room & ~use] = s[room & ~use]       # (almost) only linear jobs: uniform
    return s, s_lin


def scaled_utility(prob, lam, s, cap=True, method="hull", nthreads=0, s_lin=None):
    """U(X~) with X the subproblem solutions at lam, column j of job i scaled
    by s_lin[j] for linear-utility jobs (when given) and s[j] otherwise
    (Section 5)."""
    A, kind, w, par, _ = _arrays(prob)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    sl = None if s_lin is None else np.ascontiguousarray(s_lin, dtype=np.float64)
    U = np.zeros(1)
    rc = lib().ora_scaled_utility(prob.n, prob.m, _p(A), _p(kind), _p(w), _p(par), _p(lam),
                                  _p(s), _p(sl) if sl is not None else None, int(bool(cap)),
                                  0 if method == "hull" else 1, _p(U), nthreads)
    assert rc == 0
    return float(U[0])


def lower_bound(prob, lam, cap=True, method="hull", nthreads=0, r=None, r_lin=None):
    """Feasible utility U(X~) at lam by column scaling (``column_scales``),
    with the scaling used (s, and s_lin for the linear-utility jobs)."""
    if r is None or r_lin is None:
        _, r, _, r_lin = dual(prob, lam, cap, method, nthreads, split=True)
    s, s_lin = column_scales(prob.R, r, r_lin, cap)
    return scaled_utility(prob, lam, s, cap, method, nthreads, s_lin=s_lin), (s, s_lin)


def own_lower_bound(prob, lam, nthreads=0):
    """Lower bound on the column-scaled utility U(X~) at lam without the
    per-job cap (``lower_bound`` with cap=False), formed from the evaluation's
    sums alone.  Without the cap job i uses one resource j, and at its
    subproblem optimum t_i u_i'(t_i) = (lam_j / A_ij) t_i = lam_j x_ij
    (Section 4.1).  Scaling t_i by s (ln s = l):

    * log:            w ln(s t) = w ln t + l (t u'(t))                 (exact)
    * power, p > 0:   s^p u(t) >= (1 + p l) u(t) = u(t) + l (t u'(t))   (e^y >= 1 + y, u >= 0)
    * power, p < 0:   s^p u(t) >= u(t) + l (t u'(t)) - (p l)^2 / 2 e^(|p l|) |u(t)|
                      (Taylor remainder of e^(p l); u < 0, |p| <= 64)
    * linear kinds:   kept whole or scaled up, which lowers no u.

    Summed over column j the first-order terms give lam_j (r_j - r_lin_j) l_j,
    so the bound is U(X) + sum_j lam_j (r_j - r_lin_j) ln s_j - L^2/2 e^(64 L)
    sum_{p_i<0} p_i^2 |u_i(t_i)|, L = max_j |ln s_j| over the scaled columns.
    A column that scales its linear-utility jobs down (s_lin < 1) admits no
    such bound: -inf.  Returns (bound, (s, s_lin))."""
    _, kind, w, par, R = _arrays(prob)
    lam = np.asarray(lam, np.float64)
    _, r, U, r_lin = dual(prob, lam, cap=False, nthreads=nthreads, split=True)
    s, s_lin = column_scales(R, r, r_lin, cap=False)
    if np.any((s_lin < 1.0) & (r_lin > 0.0)):
        return -np.inf, (s, s_lin)
    r_oth = r - r_lin
    scaled = (r_oth > 0.0) & (s != 1.0)
    ls = np.where(scaled, np.log(np.where(scaled, s, 1.0)), 0.0)
    L = float(np.max(np.abs(ls))) if prob.m else 0.0
    bound = U + float(np.sum(lam * r_oth * ls))
    neg = (kind == 1) & (par < 0)
    if np.any(neg):
        t = jobs(prob, lam, idx=np.flatnonzero(neg), cap=False, nthreads=nthreads)[:, 0]
        wn, pn = w[neg].astype(np.float64), par[neg].astype(np.float64)
        s2 = float(np.sum(pn * pn * np.abs(-wn * np.power(t, pn))))
        if s2 > 0.0:
            bound -= 0.5 * L * L * np.exp(64.0 * L) * s2
    return bound, (s, s_lin)


def init_prices(prob, cap=True, nthreads=0):
    """lam^1 of Eq. e-initialization."""
    A, kind, w, par, R = _arrays(prob)
    lam = np.zeros(prob.m)
    rc = lib().ora_init(prob.n, prob.m, _p(A), _p(kind), _p(w), _p(par), _p(R), int(bool(cap)),
                        _p(lam), nthreads)
    assert rc == 0
    return lam


def rel_gap(g, lb):
    return (g - lb) / max(abs(lb), abs(g), 1.0)


def mixture_utility(prob, theta, lams, sc_oth, sc_lin, cap=True, method="hull", nthreads=0):
    """U(sum_k theta_k X(lam_k) diag(sc_k)) in FP64 without forming X: column j
    of allocation k is scaled by sc_lin[k, j] for jobs with a linear utility
    and by sc_oth[k, j] otherwise."""
    A, kind, w, par, _ = _arrays(prob)
    theta = np.ascontiguousarray(theta, np.float64)
    lams = np.ascontiguousarray(lams, np.float64).reshape(len(theta), prob.m)
    so = np.ascontiguousarray(sc_oth, np.float64).reshape(len(theta), prob.m)
    sl = np.ascontiguousarray(sc_lin, np.float64).reshape(len(theta), prob.m)
    U = np.zeros(1)
    rc = lib().ora_mixture_utility(prob.n, prob.m, _p(A), _p(kind), _p(w), _p(par), len(theta),
                                   _p(theta), _p(lams), _p(so), _p(sl), int(bool(cap)),
                                   0 if method == "hull" else 1, _p(U), nthreads)
    assert rc == 0
    return float(U[0])


def sparse_allocation_check(prob, jk, xk):
    """FP64 utility and usage of an allocation given as per-job (resource,
    time fraction) pairs (resource -1 = unused): t_i = sum_k A[i, jk] xk,
    U = sum_i u_i(t_i), usage_j = sum of the fractions on resource j.
    Returns (U, usage, t)."""
    n, m = prob.n, prob.m
    jk = np.asarray(jk, np.int64).reshape(n, -1)
    xk = np.asarray(xk, np.float64).reshape(n, -1)
    valid = jk >= 0
    rows = np.broadcast_to(np.arange(n)[:, None], jk.shape)
    a = np.where(valid, prob.A[rows, np.where(valid, jk, 0)].astype(np.float64), 0.0)
    x = np.where(valid, xk, 0.0)
    t = (a * x).sum(1)
    usage = np.bincount(jk[valid], weights=x[valid], minlength=m)
    return utility_of(prob, t), usage, t


def certify(prob, lam_best, theta, lams, scaled, cap=True, nthreads=0, repaired=None):
    """FP64 re-check of a solver's result (Section 5's bounds): the dual value
    g at ``lam_best`` (an upper bound on U*), and the utility of the
    allocation behind the solver's lower bound -- the mixture sum_k theta_k
    X(lam_k), allocation k column-scaled (``column_scales``) where
    ``scaled[k]`` is 1 -- once more scaled by min(1, R/usage) so that it
    meets X^T 1 <= R exactly in FP64 (a lower bound on U*).  When the bound
    came from a repaired allocation (``scaled == [2]``), ``repaired`` holds
    that allocation as (jk, xk) pairs and is checked as given.  Returns a
    dict with g, U_lb, the relative gap, usage / R of the allocation before
    that last scaling (its worst entry is the solver's constraint
    violation), and the seconds taken."""
    t0 = time.perf_counter()
    R = np.asarray(prob.R, np.float64)
    lam_best = np.asarray(lam_best, np.float64)
    g, _, _ = dual(prob, lam_best, cap, nthreads=nthreads)
    if 2 in list(np.asarray(scaled)):
        jk, xk = repaired
        U0, usage, t = sparse_allocation_check(prob, jk, xk)
        ratio = np.where(R > 0, usage / np.where(R > 0, R, 1.0), np.where(usage > 0, np.inf, 0.0))
        f = column_scale(R, usage, cap=True)
        # the last scaling in FP64, applied to each job's throughput column by column
        jk_ = np.asarray(jk, np.int64).reshape(prob.n, -1)
        xk_ = np.asarray(xk, np.float64).reshape(prob.n, -1) * np.where(jk_ >= 0, f[np.maximum(jk_, 0)], 0.0)
        U, _, _ = sparse_allocation_check(prob, jk_, xk_)
        return dict(g=g, U_lb=U, rel_gap=rel_gap(g, U), usage_over_R=ratio,
                    max_usage_over_R=float(ratio.max()), seconds=time.perf_counter() - t0)
    theta = np.asarray(theta, np.float64)
    lams = np.asarray(lams, np.float64).reshape(len(theta), prob.m)
    keep = theta > 0
    theta, lams, scaled = theta[keep], lams[keep], np.asarray(scaled)[keep]
    so = np.ones_like(lams)
    sl = np.ones_like(lams)
    usage = np.zeros(prob.m)
    for k in range(len(theta)):
        _, r, _, r_lin = dual(prob, lams[k], cap, nthreads=nthreads, split=True)
        if scaled[k]:
            so[k], sl[k] = column_scales(R, r, r_lin, cap)
        usage += theta[k] * (so[k] * (r - r_lin) + sl[k] * r_lin)
    f = column_scale(R, usage, cap=True)
    U = mixture_utility(prob, theta, lams, so * f[None, :], sl * f[None, :], cap, nthreads=nthreads)
    ratio = np.where(R > 0, usage / np.where(R > 0, R, 1.0), np.where(usage > 0, np.inf, 0.0))
    return dict(g=g, U_lb=U, rel_gap=rel_gap(g, U), usage_over_R=ratio,
                max_usage_over_R=float(ratio.max()), seconds=time.perf_counter() - t0)


# --------------------------------------------------------------------------- solve

@dataclasses.dataclass
class Solution:
    lam: np.ndarray          # prices at the best dual value
    g: float                 # best (smallest) dual value = upper bound on U*
    U_lb: float              # best feasible utility = lower bound on U*
    lam_lb: np.ndarray       # prices whose scaled allocation gave U_lb
    s_lb: np.ndarray         # column scaling used for U_lb
    gap: float               # relative duality gap
    evals: int
    converged: bool
    seconds: float
    history: list


class _Converged(Exception):
    pass


def master_lower_bound(cands, R):
    """Lower bound from a convex combination of evaluated allocations.

    ``cands`` is a list of (U_k, r_k): the utility of an allocation X^k whose
    rows each solve the job constraints, and its usage r_k.  For weights
    theta >= 0, sum theta = 1 with sum_k theta_k r_k <= R, the allocation
    sum_k theta_k X^k is feasible for problem (e-res-alloc) and, since every
    u_i is concave, its utility is at least sum_k theta_k U_k.  The best such
    bound is an LP in theta (solved with scipy HiGHS).  Returns (bound, theta)
    or (-inf, None) when no combination is feasible."""
    from scipy.optimize import linprog
    if not cands:
        return -np.inf, None
    U = np.array([c[0] for c in cands], np.float64)
    Rm = np.array([c[1] for c in cands], np.float64)          # K x m
    ok = np.isfinite(U) & np.all(np.isfinite(Rm), axis=1)
    if not ok.any():
        return -np.inf, None
    U, Rm = U[ok], Rm[ok]
    R = np.asarray(R, np.float64)
    scale = np.where(R > 0, R, 1.0)
    # the LP solver meets constraints to its tolerance only: tighten the
    # limits by a margin larger than that tolerance, then verify exactly
    res = linprog(-U / max(np.abs(U).max(), 1.0), A_ub=(Rm / scale).T,
                  b_ub=R / scale * (1.0 - 1e-9), A_eq=np.ones((1, len(U))), b_eq=[1.0],
                  bounds=[(0, None)] * len(U), method="highs",
                  options=dict(primal_feasibility_tolerance=1e-10))
    if res.status != 0:
        return -np.inf, None
    theta = np.maximum(res.x, 0.0)
    theta /= theta.sum()
    if np.any(theta @ Rm > R):
        return -np.inf, None
    return float(theta @ U), theta


def solve(prob, cap=True, tol=1e-6, max_evals=400, method="hull", nthreads=0, lam0=None,
          update="lbfgs", lam_floor=None, history=False, repair=True, master=True,
          master_window=32):
    """Algorithm 2: evaluate g, q and U(X~) at each price vector, stop when the
    relative duality gap is <= tol, update the prices with L-BFGS (default) or
    the projected subgradient method.  With ``master`` the lower bound also
    uses ``master_lower_bound`` over the last ``master_window`` evaluations.
    When the loop ends above ``tol`` and ``repair`` is set, the tie-aware
    repair of ``repair_lower_bound`` is tried at the best prices."""
    m = prob.m
    lam = init_prices(prob, cap, nthreads) if lam0 is None else np.asarray(lam0, np.float64).copy()
    if lam_floor is None:
        # Without the per-job cap a zero price makes strictly increasing
        # utilities demand unbounded throughput, so prices stay positive.
        lam_floor = 0.0 if cap else 1e-9 * max(float(np.max(lam)), 1e-300)
    lam = np.maximum(lam, lam_floor)
    st = dict(g=np.inf, lam=lam.copy(), lb=-np.inf, lam_lb=lam.copy(), s_lb=np.ones(m), evals=0,
              hist=[])
    t0 = time.perf_counter()

    cands = []
    R = np.asarray(prob.R, np.float64)

    def evaluate(x):
        x = np.maximum(np.asarray(x, np.float64), lam_floor)
        g, r, Ux, r_lin = dual(prob, x, cap, method, nthreads, split=True)
        lb, (s, s_lin) = lower_bound(prob, x, cap, method, nthreads, r=r, r_lin=r_lin)
        st["evals"] += 1
        if master:
            cands.append((Ux, r.copy()))
            cands.append((lb, s * (r - r_lin) + s_lin * r_lin))
            if len(cands) > 2 * master_window:
                del cands[:2]
            if st["evals"] >= 2 and rel_gap(min(st["g"], g), max(st["lb"], lb)) > tol:
                mlb, _ = master_lower_bound(cands, R)
                if mlb > lb:
                    lb = mlb
        if g < st["g"]:
            st["g"], st["lam"] = g, x.copy()
        if lb > st["lb"]:
            st["lb"], st["lam_lb"], st["s_lb"] = lb, x.copy(), s
        if history:
            st["hist"].append((st["evals"], g, lb, rel_gap(st["g"], st["lb"])))
        if rel_gap(st["g"], st["lb"]) <= tol:
            raise _Converged
        if st["evals"] >= max_evals:
            raise _Converged
        return g, np.asarray(prob.R, np.float64) - r

    try:
        if update == "lbfgs":
            from scipy.optimize import minimize
            minimize(evaluate, lam, jac=True, method="L-BFGS-B",
                     bounds=[(lam_floor, None)] * m,
                     options=dict(maxcor=10, maxfun=max_evals, maxiter=max_evals, ftol=0.0,
                                  gtol=0.0, maxls=40))
        elif update == "subgradient":
            # lam^{k+1} = max(lam^k - a_k q^k, 0), a_k = a_0 / sqrt(k): a_k -> 0, sum a_k = inf
            g0, q = evaluate(lam)
            a0 = 0.1 * max(float(np.max(lam)), 1e-12) / max(float(np.max(np.abs(q))), 1e-300)
            k = 1
            while True:
                lam = np.maximum(lam - (a0 / np.sqrt(k)) * q, lam_floor)
                _, q = evaluate(lam)
                k += 1
        else:
            raise ValueError(update)
    except _Converged:
        pass
    if repair and rel_gap(st["g"], st["lb"]) > tol:
        # the column-scaled bound stalls when the optimum sits on ties
        for rel in (1e-10, 1e-8, 1e-6, 1e-4):
            lb, info = repair_lower_bound(prob, st["lam"], cap, rel, nthreads)
            if lb > st["lb"]:
                st["lb"], st["lam_lb"], st["s_lb"] = lb, st["lam"].copy(), info.get("s", st["s_lb"])
            if rel_gap(st["g"], st["lb"]) <= tol:
                break
    gap = rel_gap(st["g"], st["lb"])
    return Solution(st["lam"], st["g"], st["lb"], st["lam_lb"], st["s_lb"], gap, st["evals"],
                    gap <= tol, time.perf_counter() - t0, st["hist"])


# --------------------------------------------------------------------------- primal

def allocation(prob, lam, cap=True, method="hull", nthreads=0):
    """Dense X (n x m, FP64) of the subproblem solutions at lam (Section 3,
    "Recovering an optimal allocation from optimal prices")."""
    rec = jobs(prob, lam, cap=cap, method=method, nthreads=nthreads)
    X = np.zeros((prob.n, prob.m))
    rows = np.arange(prob.n)
    for jc, xc in ((3, 5), (4, 6)):
        sel = rec[:, jc] >= 0
        X[rows[sel], rec[sel, jc].astype(np.int64)] += rec[sel, xc]
    return X, rec


def utility_of(prob, t):
    """U(t) = sum_i u_i(t_i) in FP64 (Section 2.2)."""
    w = prob.w.astype(np.float64)
    par = prob.param.astype(np.float64)
    t = np.asarray(t, np.float64)
    u = np.empty_like(t)
    k = prob.kind
    with np.errstate(divide="ignore"):
        m0 = k == 0
        u[m0] = w[m0] * np.log(t[m0])
        m1 = k == 1
        u[m1] = np.sign(par[m1]) * w[m1] * np.power(t[m1], par[m1])
        m2 = k == 2
        u[m2] = w[m2] * np.minimum(t[m2], par[m2])
        m3 = k == 3
        u[m3] = w[m3] * np.minimum(t[m3] - par[m3], 0.0)
    return float(np.sum(u))


# --------------------------------------------------------------------------- repair

def _u_vec(kind, w, par, t):
    with np.errstate(divide="ignore", invalid="ignore"):
        if kind == 0:
            return w * np.log(t)
        if kind == 1:
            return np.sign(par) * w * np.power(t, par)
        if kind == 2:
            return w * np.minimum(t, par)
        return w * np.minimum(t - par, 0.0)


def job_alternatives(a, lam, kind, w, par, cap=True, rel=1e-9):
    """All extreme optimal allocations of one subproblem, within a relative
    value tolerance: every pair (P, Q) of the points (0,0), (a_j, lam_j)
    (Section 4.1) with both ends of its maximising t-interval.  Returns a
    list of (t, x) with x a dense m-vector."""
    a = np.asarray(a, np.float64)
    lam = np.asarray(lam, np.float64)
    m = len(a)
    cand = []
    pts = [(-1, 0.0, 0.0)] + [(j, a[j], lam[j]) for j in range(m) if a[j] > 0]
    for (Q, aQ, lQ) in pts[1:]:
        starts = pts if cap else pts[:1]
        for (P, aP, lP) in starts:
            if not aP < aQ:
                continue
            alpha = (lQ - lP) / (aQ - aP)
            beta = lP - alpha * aP
            hi = aQ if cap else np.inf
            ts = []
            if kind in (0, 1):
                if alpha <= 0:
                    ts = [hi]
                else:
                    t = w / alpha if kind == 0 else (w * abs(par) / alpha) ** (1.0 / (1.0 - par))
                    ts = [min(max(t, aP), hi)]
            else:
                if w < alpha * (1 - rel):
                    ts = [aP]
                elif w <= alpha * (1 + rel):
                    ts = [aP, min(max(par, aP), hi)]
                elif alpha < 0:
                    ts = [hi]
                elif alpha <= rel * w:
                    ts = [min(max(par, aP), hi), hi]
                else:
                    ts = [min(max(par, aP), hi)]
            for t in ts:
                if not np.isfinite(t):
                    continue
                v = float(_u_vec(kind, w, par, t)) - (alpha * t + beta)
                x = np.zeros(m)
                if cap:
                    xQ = (t - aP) / (aQ - aP)
                    x[Q] = xQ
                    if P >= 0:
                        x[P] = (aQ - t) / (aQ - aP)
                else:
                    x[Q] = t / aQ
                cand.append((v, t, x))
    if not cand:
        return [(0.0, np.zeros(m))]
    best = max(c[0] for c in cand)
    scale = max(abs(best), 1e-12)
    keep = []
    for v, t, x in cand:
        if v >= best - rel * scale and not any(np.allclose(x, y, rtol=0, atol=1e-13) for _, y in keep):
            keep.append((t, x))
    return keep


def repair_lower_bound(prob, lam, cap=True, rel=1e-9, nthreads=0, max_flex=20000):
    """Feasible utility at prices lam when subproblems have several optimal
    solutions (the paper is silent here; Section 3 only says any optimal
    allocation solves every job's subproblem at lam*).

    Jobs whose solution is unique within ``rel`` keep it.  For the others the
    optimal extreme allocations are enumerated and an LP (scipy HiGHS) picks
    convex weights that (A) minimise the total relative overuse
    sum_j max(r_j - R_j, 0)/R_j and then (B) maximise the linearised utility
    sum_k theta_k u(t_k).  Remaining overuse is removed by column scaling.
    Returns (U_lb, info) with U_lb the exact utility of the repaired X~."""
    from scipy.optimize import linprog
    rec = jobs(prob, lam, cap=cap, nthreads=nthreads)
    flex = np.flatnonzero((rec[:, 8] <= rel * 10) | (rec[:, 9] <= rel * 10))
    if len(flex) > max_flex:
        return -np.inf, dict(n_flex=len(flex), status="too many flexible jobs")
    n, m = prob.n, prob.m
    R = np.asarray(prob.R, np.float64)
    X, _ = allocation(prob, lam, cap=cap, nthreads=nthreads)
    t_all = rec[:, 0].copy()
    alts = []
    for i in flex:
        alts.append(job_alternatives(prob.A[i].astype(np.float64), lam, int(prob.kind[i]),
                                     float(prob.w[i]), float(prob.param[i]), cap, rel))
    fixed = np.ones(n, bool)
    fixed[flex] = False
    r_fixed = X[fixed].sum(axis=0)
    nv = sum(len(a_) for a_ in alts)
    if nv == 0:
        s = column_scale(R, r_fixed, cap)
        return (utility_of(prob, (prob.A.astype(np.float64) * X * s).sum(1)),
                dict(n_flex=0, n_alt=0, s=s, X=X))
    # variables: theta (nv), v (m)
    Mx = np.zeros((m, nv))
    uvec = np.zeros(nv)
    Aeq = np.zeros((len(alts), nv + m))
    col = 0
    for k, (i, al) in enumerate(zip(flex, alts)):
        for (t, x) in al:
            Mx[:, col] = x
            uvec[col] = float(_u_vec(int(prob.kind[i]), float(prob.w[i]), float(prob.param[i]),
                                     max(t, 1e-300)))
            Aeq[k, col] = 1.0
            col += 1
    Aub = np.hstack([Mx, -np.eye(m)])
    bub = R - r_fixed
    beq = np.ones(len(alts))
    bounds = [(0, None)] * (nv + m)
    resA = linprog(np.concatenate([np.zeros(nv), 1.0 / R]), A_ub=Aub, b_ub=bub, A_eq=Aeq, b_eq=beq,
                   bounds=bounds, method="highs")
    if resA.status != 0:
        return -np.inf, dict(n_flex=len(flex), status=resA.message)
    vstar = resA.x[nv:]
    bounds_b = [(0, None)] * nv + [(0, vj * (1 + 1e-9) + 1e-12) for vj in vstar]
    resB = linprog(np.concatenate([-uvec, np.zeros(m)]), A_ub=Aub, b_ub=bub, A_eq=Aeq, b_eq=beq,
                   bounds=bounds_b, method="highs")
    theta = (resB.x if resB.status == 0 else resA.x)[:nv]
    Xr = X.copy()
    col = 0
    for i, al in zip(flex, alts):
        xi = np.zeros(m)
        for (t, x) in al:
            xi += theta[col] * x
            col += 1
        Xr[i] = xi
    r = Xr.sum(axis=0)
    s = column_scale(R, r, cap)
    Af = prob.A.astype(np.float64)
    t_rep = (Af * Xr * s[None, :]).sum(axis=1)
    return utility_of(prob, t_rep), dict(n_flex=len(flex), n_alt=nv, s=s, X=Xr)


def allocation_stats(X, tol=1e-9):
    """Fractions of jobs using two resources and of jobs with positive slack
    1 - 1^T x_i (the statistics quoted in Section 6.2)."""
    nz = (X > tol).sum(axis=1)
    slack = 1.0 - X.sum(axis=1)
    return dict(two_resources=float(np.mean(nz == 2)), one_resource=float(np.mean(nz == 1)),
                positive_slack=float(np.mean(slack > 1e-6)))
