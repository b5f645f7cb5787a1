"""One allocation problem split by job range across devices or processes.

Given the prices, the jobs are independent (Section 3, "Evaluating the dual
function"): each shard -- one rank, one GPU -- holds a contiguous range of the
jobs, evaluates them with the library's kernels, and the shards exchange one
small vector per evaluation (RA_SHARD_WIDTH(m) FP64 sums: sum of h_i, U(X),
the lagged lower bound, a status word, r and r_lin).  The sums are added in
rank order on every rank, and every rank runs the same FP64 price update, so
the prices stay bitwise identical everywhere.  This module only marshals:
the all-gather is torch.distributed's (NCCL on GPUs), called back by
ra_solve_sharded on the library's stream.
"""
from __future__ import annotations

import threading

import torch

from . import ra

ALIGN = 256   # shard boundaries fall on multiples of 256 jobs (16-byte aligned pointers)


def shard_bounds(n, world, align=ALIGN):
    """[start, stop) of each of `world` contiguous job ranges: equal sizes
    rounded down to a multiple of `align`, the last range taking the rest."""
    if world < 1 or n < 1:
        raise ValueError("need n >= 1 and world >= 1")
    base = (n // world) // align * align
    if world > 1 and base == 0:
        raise ValueError(f"{n} jobs are too few for {world} shards of >= {align} jobs")
    return [(r * base, n if r == world - 1 else (r + 1) * base) for r in range(world)]


def shard_problem(A, kind, w, param, R, start, stop, job_cap=False, fp64_jobmath=False,
                  stream=None):
    """The AllocationProblem of jobs [start, stop) of device tensors (A n x m;
    R is the whole problem's)."""
    return ra.AllocationProblem(A[start:stop], kind[start:stop], w[start:stop],
                                param[start:stop], R, job_cap=job_cap,
                                fp64_jobmath=fp64_jobmath, stream=stream)


def torch_gather(group=None):
    """All-gather through torch.distributed: every rank's send into recv
    (rank order), on torch's current stream."""
    import torch.distributed as dist

    def gather(send, recv):
        try:
            dist.all_gather_into_tensor(recv, send, group=group)
        except (RuntimeError, NotImplementedError):
            world = recv.numel() // send.numel()
            dist.all_gather(list(recv.view(world, -1).unbind(0)), send, group=group)
    return gather


class ThreadGather:
    """All-gather among `world` threads of one process that drive shards on
    the same GPU: each thread waits for its own stream, publishes its send
    buffer, and copies every thread's buffer into its recv.  Only host
    barriers order the threads; no kernel waits on another."""

    def __init__(self, world, timeout=120.0):
        self.world = world
        self.barrier = threading.Barrier(world, timeout=timeout)
        self.bufs = [None] * world

    def for_rank(self, rank):
        def gather(send, recv):
            torch.cuda.current_stream().synchronize()
            self.bufs[rank] = send
            self.barrier.wait()
            c = send.numel()
            for s in range(self.world):
                recv[s * c:(s + 1) * c].copy_(self.bufs[s])
            torch.cuda.current_stream().synchronize()
            self.barrier.wait()
        return gather


class Exchange:
    """The buffers and the C callback that ra_solve_sharded calls once per
    evaluation."""

    def __init__(self, m, world, device, gather):
        self.world = world
        width = ra.RA_SHARD_WIDTH(m)
        self.send = torch.zeros(width, dtype=torch.float64, device=device)
        self.recv = torch.zeros(world * width, dtype=torch.float64, device=device)
        self.gather = gather
        self.error = None
        self.fn = ra.ALLGATHER_FN(self._call)   # keep the callback alive

    def _call(self, ctx, count, stream):
        try:
            with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
                self.gather(self.send[:count], self.recv[:self.world * count])
            return 0
        except Exception as e:  # reported by ra_solve_sharded as a failed exchange
            self.error = e
            return 1


def solve(shard, n_total, rank, world, gather, tol=1e-6, max_evals=500, lam0=None,
          init_step=None, lbfgs_mem=10, master_lb=True):
    """ra_solve_sharded for this rank's shard; returns (prices, info)."""
    ex = Exchange(shard.m, world, shard.A.device, gather)
    o = ra.ra_solve_opts_default()
    o.tol_rel = tol
    o.max_evals = max_evals
    o.lbfgs_mem = lbfgs_mem
    o.master_lb = 1 if master_lb else 0
    o.use_graph = 0
    o.repair_window = 0
    if init_step is not None:
        o.init_step = init_step
    lam = torch.empty(shard.m, dtype=torch.float64, device=shard.A.device)
    if lam0 is not None:
        lam0 = torch.as_tensor(lam0, dtype=torch.float64, device=shard.A.device).contiguous()
    try:
        info = ra.ra_solve_sharded(shard.handle, n_total, rank, world, ex.send, ex.recv, ex.fn,
                                   lam, opts=o, lam0=lam0)
    except ra.RaError:
        if ex.error is not None:
            raise ex.error
        raise
    shard.prices = lam
    return lam, info


def eval_dual(shard, lam, m, world, gather, R):
    """g and q of the whole problem at lam from this rank's shard."""
    width = ra.RA_SHARD_WIDTH(m)
    dev = shard.A.device
    part = torch.empty(width, dtype=torch.float64, device=dev)
    lam = torch.as_tensor(lam, dtype=torch.float64, device=dev).contiguous()
    ra.ra_eval_partial(shard.handle, lam, part)
    parts = torch.empty(world * width, dtype=torch.float64, device=dev)
    gather(part, parts)
    g = torch.empty(1, dtype=torch.float64, device=dev)
    q = torch.empty(m, dtype=torch.float64, device=dev)
    ra.ra_combine_partials(parts, m, lam, R, g, q)
    return g, q
