"""Seeded synthetic workloads for the fungible resource-allocation problem.

This module only draws random problem data; it contains none of the price
discovery arithmetic.  Both the CUDA path and the FP64 CPU oracle consume
the arrays it produces, so it is the one piece of code they share.

A problem is (Section 2.4, problem (e-res-alloc)):

* ``A``     -- n x m efficiency matrix, FP32, row-major; row i is a_i^T
               (Section 2.1, "Throughput").
* ``kind``  -- n uint8 utility kinds:
               0 = log        u(t) = w log t            (Eq. e-log-util, weighted)
               1 = power      u(t) = w t^p, 0 < p < 1, or -w t^p, p < 0
                                (Section 2.2, "Power utilities"; alpha-fair)
               2 = lin-cap    u(t) = w min(t, T)        (target-priority plus w T)
               3 = target     u(t) = w min(t - T, 0)    (Eq. e-target-priority-util)
* ``w``     -- n FP32 weights (priorities), w > 0.
* ``param`` -- n FP32: the exponent p for kind 1, the target/cap T for kinds
               2 and 3, ignored (0) for kind 0.
* ``R``     -- m FP64 resource limits.

Every generator takes an explicit seed; the same (recipe, sizes, seed)
always yields bit-identical arrays on any machine (numpy PCG64 streams);
``hetero_device`` alone draws on the GPU with torch's seeded generator.
"""
from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

U_LOG, U_POWER, U_LINCAP, U_TARGET = 0, 1, 2, 3


@dataclasses.dataclass
class Problem:
    A: np.ndarray       # (n, m) float32, C-contiguous
    kind: np.ndarray    # (n,) uint8
    w: np.ndarray       # (n,) float32
    param: np.ndarray   # (n,) float32
    R: np.ndarray       # (m,) float64
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.A.shape[0])

    @property
    def m(self) -> int:
        return int(self.A.shape[1])

    def subset(self, idx) -> "Problem":
        """Rows ``idx`` with R scaled by the kept fraction of jobs."""
        idx = np.asarray(idx)
        frac = len(idx) / max(self.n, 1)
        return Problem(np.ascontiguousarray(self.A[idx]), self.kind[idx].copy(),
                       self.w[idx].copy(), self.param[idx].copy(),
                       self.R * frac, self.name + "[subset]")

    def nbytes(self) -> int:
        return self.A.nbytes + self.kind.nbytes + self.w.nbytes + self.param.nbytes


def _rng(recipe: int, seed: int, idx: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([recipe, idx, seed])))


def _lognormal_columns(rng, n, m, sigma, s_lo, s_hi):
    """A_ij = s_j * exp(sigma * z_ij), z ~ N(0,1), s_j ~ U[s_lo, s_hi] (FP32)."""
    s = rng.uniform(s_lo, s_hi, size=m).astype(np.float32)
    A = rng.standard_normal(size=(n, m), dtype=np.float32)
    A *= np.float32(sigma)
    np.exp(A, out=A)
    A *= s[None, :]
    return A


def _utility_mix(rng, n, fractions):
    """Per-job kinds drawn independently with the given (log, power, lincap) probabilities."""
    u = rng.random(n)
    kind = np.zeros(n, dtype=np.uint8)
    edge = 0.0
    for k, f in enumerate(fractions):
        lo, edge = edge, edge + f
        kind[(u >= lo) & (u < edge)] = k
    kind[u >= edge] = len(fractions) - 1
    return kind


def config_plain_small(n: int = 1000, m: int = 4, seed: int = 0) -> Problem:
    """Plain method, FP64 check case: A ~ U[0.1, 1], all log utilities,
    w ~ U[0.5, 2], R_j = 0.25 n."""
    rng = _rng(1, seed)
    A = rng.uniform(0.1, 1.0, size=(n, m)).astype(np.float32)
    w = rng.uniform(0.5, 2.0, size=n).astype(np.float32)
    kind = np.zeros(n, dtype=np.uint8)
    param = np.zeros(n, dtype=np.float32)
    R = np.full(m, 0.25 * n, dtype=np.float64)
    return Problem(A, kind, w, param, R, f"plain-small n={n} m={m}")


def config_hetero(n: int = 1_000_000, m: int = 8, seed: int = 0, recipe: int = 2,
                  idx: int = 0) -> Problem:
    """Heterogeneous hardware: A_ij = s_j exp(0.5 z), s_j ~ U[0.5, 4];
    50 % log and 50 % power (p ~ U[0.2, 0.8]); w ~ U[0.5, 2];
    R_j ~ U[0.1, 0.4] n."""
    rng = _rng(recipe, seed, idx)
    A = _lognormal_columns(rng, n, m, 0.5, 0.5, 4.0)
    kind = _utility_mix(rng, n, (0.5, 0.5))
    w = rng.uniform(0.5, 2.0, size=n).astype(np.float32)
    p = rng.uniform(0.2, 0.8, size=n).astype(np.float32)
    param = np.where(kind == U_POWER, p, np.float32(0)).astype(np.float32)
    R = rng.uniform(0.1, 0.4, size=m) * n
    return Problem(A, kind, w, param, R.astype(np.float64), f"hetero n={n} m={m}")


def config_large(n: int = 10_000_000, m: int = 32, seed: int = 0) -> Problem:
    """Large single problem: A_ij = s_j exp(0.75 z), s_j ~ U[0.25, 8];
    40 % log, 40 % power (p ~ U[0.2, 0.8]), 20 % linear with cap
    (T ~ U[1, 10]); w ~ U[0.5, 2]; R_j ~ U[0.05, 0.3] n."""
    rng = _rng(3, seed)
    A = _lognormal_columns(rng, n, m, 0.75, 0.25, 8.0)
    kind = _utility_mix(rng, n, (0.4, 0.4, 0.2))
    w = rng.uniform(0.5, 2.0, size=n).astype(np.float32)
    p = rng.uniform(0.2, 0.8, size=n).astype(np.float32)
    T = rng.uniform(1.0, 10.0, size=n).astype(np.float32)
    param = np.where(kind == U_POWER, p, np.where(kind == U_LINCAP, T, np.float32(0)))
    R = rng.uniform(0.05, 0.3, size=m) * n
    return Problem(A, kind, w, param.astype(np.float32), R.astype(np.float64),
                   f"large n={n} m={m}")


def batched_shapes(P: int = 4096, seed: int = 0, n_lo: int = 100, n_hi: int = 200_000,
                   m_choices=(4, 8, 16, 32)):
    """(n_k, m_k) for P independent problems: n log-uniform in [n_lo, n_hi],
    m uniform over ``m_choices``."""
    rng = _rng(4, seed)
    n = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=P))).astype(np.int64)
    m = rng.choice(np.asarray(m_choices, dtype=np.int64), size=P)
    return n, m


def batched_problem(k: int, n: int, m: int, seed: int = 0) -> Problem:
    """Problem k of the batched workload: heterogeneous-hardware recipe."""
    return config_hetero(n=int(n), m=int(m), seed=seed, recipe=40, idx=k)


def batched_workload(P: int = 4096, seed: int = 0, threads: int | None = None):
    """The P problems of the batched workload (shapes from ``batched_shapes``),
    generated on a thread pool; each problem has its own seeded stream, so
    the result does not depend on the thread count."""
    from concurrent.futures import ThreadPoolExecutor
    n, m = batched_shapes(P, seed)
    threads = threads or min(32, os.cpu_count() or 1)
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda k: batched_problem(k, n[k], m[k], seed), range(P)))


def warmstart_problem(k: int, seed: int = 0, m: int = 16, n_lo: int = 10_000,
                      n_hi: int = 1_000_000) -> Problem:
    """Problem k of the warm-start corpus: n log-uniform in [n_lo, n_hi], m = 16,
    heterogeneous-hardware recipe."""
    rng = _rng(5, seed, k)
    n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    return config_hetero(n=n, m=m, seed=seed, recipe=50, idx=k)


def paper_medium(n: int = 1_000_000, utility: str = "log", seed: int = 0) -> Problem:
    """Section 6.2 medium problem: (a_i)_1 ~ U(0.1,0.3), (a_i)_2 ~ U(0.1,0.5),
    (a_i)_3 ~ U(0.3,0.8), (a_i)_4 ~ U(0.6,1.0); R = (8e5, 1e5, 1e4, 1e3) at
    n = 1e6 (scaled by n / 1e6).  ``utility`` is "log" (u = log t, w = 1) or
    "target" (target-priority with t_des = 0.2 and w in {1, 2} with
    probability 1/2 each)."""
    rng = _rng(6, seed)
    lo = np.array([0.1, 0.1, 0.3, 0.6])
    hi = np.array([0.3, 0.5, 0.8, 1.0])
    A = (lo + (hi - lo) * rng.random((n, 4))).astype(np.float32)
    R = np.array([8e5, 1e5, 1e4, 1e3]) * (n / 1e6)
    if utility == "log":
        kind = np.zeros(n, dtype=np.uint8)
        w = np.ones(n, dtype=np.float32)
        param = np.zeros(n, dtype=np.float32)
    elif utility == "target":
        kind = np.full(n, U_TARGET, dtype=np.uint8)
        w = np.where(rng.random(n) < 0.5, 1.0, 2.0).astype(np.float32)
        param = np.full(n, 0.2, dtype=np.float32)
    else:
        raise ValueError(utility)
    return Problem(A, kind, w, param, R.astype(np.float64), f"paper-medium-{utility} n={n}")


def paper_code_example(n: int = 1_000_000, m: int = 4, seed: int = 0) -> Problem:
    """Section 6.1 code example: A ~ U[0, 1], R = U[0, 1] n + 1e3, log utility."""
    rng = _rng(7, seed)
    A = rng.random((n, m), dtype=np.float32)
    R = rng.random(m) * n + 1e3
    return Problem(A, np.zeros(n, np.uint8), np.ones(n, np.float32),
                   np.zeros(n, np.float32), R.astype(np.float64), f"paper-example n={n} m={m}")


def random_small(n: int, m: int, seed: int, kinds=(0, 1, 2, 3), r_scale: float = 0.3) -> Problem:
    """Small mixed problems for exhaustive checks: A ~ U[0.05, 1] (FP32),
    kinds uniform over ``kinds``, w ~ U[0.5, 2], p ~ U[0.2, 0.8],
    T ~ U[0.1, 1], R_j ~ U[0.5, 1.5] r_scale n."""
    rng = _rng(8, seed)
    A = rng.uniform(0.05, 1.0, size=(n, m)).astype(np.float32)
    kind = np.asarray(kinds, dtype=np.uint8)[rng.integers(0, len(kinds), size=n)]
    w = rng.uniform(0.5, 2.0, size=n).astype(np.float32)
    p = rng.uniform(0.2, 0.8, size=n).astype(np.float32)
    T = rng.uniform(0.1, 1.0, size=n).astype(np.float32)
    param = np.where(kind == U_POWER, p, np.where(kind >= U_LINCAP, T, 0)).astype(np.float32)
    R = rng.uniform(0.5, 1.5, size=m) * r_scale * n
    return Problem(A, kind, w, param, R.astype(np.float64), f"random-small n={n} m={m}")


def alpha_fair(n: int, m: int = 8, seed: int = 0, alpha_lo: float = 1.5,
               alpha_hi: float = 5.0) -> Problem:
    """Alpha-fair utilities (Section 2.2): A_ij = s_j exp(0.5 z), s_j ~ U[0.5, 4];
    30 % log utilities (alpha = 1), 70 % t^(1-alpha) / (1-alpha) with alpha ~
    U[alpha_lo, alpha_hi] (kind 1 with p = 1 - alpha < 0 and weight 1/|p|),
    each times a priority ~ U[0.5, 2]; R_j ~ U[0.1, 0.4] n."""
    rng = _rng(12, seed)
    A = _lognormal_columns(rng, n, m, 0.5, 0.5, 4.0)
    kind = _utility_mix(rng, n, (0.3, 0.7))
    prio = rng.uniform(0.5, 2.0, size=n)
    p = 1.0 - rng.uniform(alpha_lo, alpha_hi, size=n)
    w = np.where(kind == U_POWER, prio / np.abs(p), prio).astype(np.float32)
    param = np.where(kind == U_POWER, p, 0.0).astype(np.float32)
    R = rng.uniform(0.1, 0.4, size=m) * n
    return Problem(A, kind, w, param, R.astype(np.float64), f"alpha-fair n={n} m={m}")


def random_prices(m: int, seed: int, lo: float = 0.2, hi: float = 3.0) -> np.ndarray:
    """A seeded FP64 price vector lambda ~ U[lo, hi]^m."""
    return _rng(9, seed).uniform(lo, hi, size=m)


MLP_SHAPES = [(26, 256), (256,), (256, 256), (256,), (256,), (1,)]   # W1 b1 W2 b2 W3 b3
MLP_FAN_IN = [26, 26, 256, 256, 256, 256]


def mlp_init(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters of the warm-start network (flat FP32 vector in
    the library's layout): every tensor ~ U[-1/sqrt(fan_in), 1/sqrt(fan_in)]."""
    rng = _rng(10, seed)
    parts = []
    for shape, fan in zip(MLP_SHAPES, MLP_FAN_IN):
        b = 1.0 / math.sqrt(fan)
        parts.append(rng.uniform(-b, b, size=shape).astype(np.float32).ravel())
    return np.concatenate(parts)


def device_seed(recipe: int, seed: int, idx: int = 0) -> int:
    """63-bit seed of a torch generator for (recipe, seed, idx)."""
    state = np.random.SeedSequence([recipe, idx, seed]).generate_state(2, np.uint32)
    return int((int(state[0]) << 31) ^ int(state[1]))


def hetero_device(n: int, m: int, seed: int, idx: int, device, recipe: int = 50):
    """The heterogeneous-hardware recipe of ``config_hetero`` drawn directly on
    a CUDA device with a seeded torch generator (for corpora too large to
    generate on the host; reproducible for a given torch version and GPU):
    A_ij = s_j exp(0.5 z), s_j ~ U[0.5, 4]; 50 % log and 50 % power utilities
    (p ~ U[0.2, 0.8]); w ~ U[0.5, 2]; R_j ~ U[0.1, 0.4] n.  Returns device
    tensors (A, kind, w, param, R)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(device_seed(recipe, seed, idx))
    s = 0.5 + 3.5 * torch.rand(m, generator=g, device=device)
    A = torch.randn(n, m, generator=g, device=device).mul_(0.5).exp_().mul_(s)
    kind = (torch.rand(n, generator=g, device=device) >= 0.5).to(torch.uint8)
    w = 0.5 + 1.5 * torch.rand(n, generator=g, device=device)
    p = 0.2 + 0.6 * torch.rand(n, generator=g, device=device)
    param = torch.where(kind == U_POWER, p, torch.zeros_like(p))
    R = (0.1 + 0.3 * torch.rand(m, generator=g, device=device, dtype=torch.float64)) * n
    return A.contiguous(), kind, w.contiguous(), param.contiguous(), R


def warmstart_sizes(P: int, seed: int = 0, n_lo: int = 10_000, n_hi: int = 1_000_000) -> np.ndarray:
    """n of the P problems of a warm-start corpus: log-uniform in [n_lo, n_hi]."""
    rng = _rng(11, seed)
    return np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=P))).astype(np.int64)
