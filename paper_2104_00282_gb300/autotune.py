"""Autotuner of the batched evaluation's launch shape (ra_batch_create_shaped).

The knobs: chunk_tiles (256-job tiles of one problem a CTA takes per visit),
whole_tiles (problems of at most this many tiles are one chunk -- one CTA
evaluates the whole small problem, the small-problem path) and ctas_per_sm
(the persistent grid per width class).  Each candidate is timed on the
caller's own problems (one complete batched solve after a warm-up solve,
CUDA events), and the fastest is cached in a JSON file keyed by the GPU, the
width classes present and a histogram of the problem sizes (n buckets of a
factor 4), so a later call with the same kind of workload reuses it.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import torch

from . import ra

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "_tuned", "batch_shapes.json")
CANDIDATES = [(c, w, k) for c in (8, 16, 32, 64) for w in (0, 4, 16) for k in (0, 2)]


def workload_key(tensors, job_cap):
    """(GPU name, width classes present, n histogram in factor-4 buckets, cap mode)."""
    name = torch.cuda.get_device_name()
    ms = sorted({4 << (0 if m <= 4 else 1 if m <= 8 else 2 if m <= 16 else 3)
                 for m in (int(t[0].shape[1]) for t in tensors)})
    hist = {}
    for t in tensors:
        b = int(math.log(max(int(t[0].shape[0]), 1), 4))
        hist[b] = hist.get(b, 0) + 1
    hk = ",".join(f"{b}:{hist[b]}" for b in sorted(hist))
    return f"{name}|m{ms}|n4^{{{hk}}}|cap{int(job_cap)}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def time_shape(tensors, shape, job_cap, tol, max_evals):
    """Device time of one batched solve with this shape (after one warm-up
    solve), and the per-problem times to tolerance."""
    B = ra.AllocationBatch.from_tensors(tensors, job_cap=job_cap, shape=shape)
    try:
        B.solve(tol=tol, max_evals=max_evals)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        infos, secs = B.solve(tol=tol, max_evals=max_evals)
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1), infos, secs
    finally:
        B.close()


def tune(tensors, job_cap=True, tol=1e-6, max_evals=500, use_cache=True, log=None):
    """Best (chunk_tiles, whole_tiles, ctas_per_sm) for these problems (device
    tensors (A, kind, w, param, R) per problem) and the timing of every
    candidate tried."""
    key = workload_key(tensors, job_cap)
    cache = _load()
    if use_cache and key in cache:
        e = cache[key]
        return tuple(e["shape"]), e
    trials = []
    for shape in CANDIDATES:
        ms, infos, secs = time_shape(tensors, shape, job_cap, tol, max_evals)
        p99 = float(sorted(secs)[max(0, int(0.99 * len(secs)) - 1)] * 1e3)
        trials.append({"shape": list(shape), "ms": ms,
                       "p50_ms": float(statistics.median(secs) * 1e3), "p99_ms": p99})
        if log:
            log(f"shape {shape}: {ms:.2f} ms")
    best = min(trials, key=lambda t: t["ms"])
    entry = {"shape": best["shape"], "ms": best["ms"], "trials": trials}
    cache[key] = entry
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return tuple(best["shape"]), entry
