"""Thin Python binding of the libra C ABI (``include/ra.h``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device arrays are torch CUDA tensors; work is enqueued on the
stream given at problem creation (torch's current stream by default).  The
binding raises if ``libra.so`` has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libra.so")

RA_OK, RA_EINVAL, RA_ENOMEM, RA_ECUDA, RA_ENOTCONV, RA_ETIMEOUT, RA_EUNBOUNDED = range(7)
RA_U_LOG, RA_U_POWER, RA_U_LINCAP, RA_U_TARGET = range(4)
RA_JOB_CAP, RA_NO_JOB_CAP, RA_FP64_JOBMATH, RA_VALIDATE = 0x0, 0x1, 0x2, 0x4
RA_MAX_M = 32
RA_MLP_STATS, RA_MLP_IN, RA_MLP_HIDDEN, RA_MLP_PARAMS = 13, 26, 256, 72961
RA_MLP_PRICE_OFFSET = 1e-3


class RaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libra status {status}: {msg}")
        self.status = status


class ra_solve_opts(ctypes.Structure):
    _fields_ = [("tol_rel", ctypes.c_double), ("max_evals", ctypes.c_int32),
                ("lbfgs_mem", ctypes.c_int32), ("update", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("lam_floor", ctypes.c_double),
                ("master_lb", ctypes.c_int32), ("repair_window", ctypes.c_int32),
                ("init_step", ctypes.c_double), ("init_scale", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class ra_batch_shape(ctypes.Structure):
    _fields_ = [("chunk_tiles", ctypes.c_int32), ("whole_tiles", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class ra_repair_opts(ctypes.Structure):
    _fields_ = [("tie_rel", ctypes.c_double), ("max_flex", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class ra_repair_info(ctypes.Structure):
    _fields_ = [("n_flex", ctypes.c_int64), ("n_alt", ctypes.c_int32),
                ("lp_status", ctypes.c_int32), ("tie_cut", ctypes.c_double),
                ("overuse", ctypes.c_double), ("U", ctypes.c_double),
                ("max_usage_over_R", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ra_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("evals", ctypes.c_int32),
                ("ls_fail", ctypes.c_int32), ("g", ctypes.c_double), ("U_lb", ctypes.c_double),
                ("rel_gap", ctypes.c_double), ("gap_per_job", ctypes.c_double),
                ("repairs", ctypes.c_int32), ("n_flex", ctypes.c_int32),
                ("eval_ms", ctypes.c_double), ("step_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        L.ra_problem_create.argtypes = [i64, i32, P, P, P, P, P, u32, P, ctypes.POINTER(P)]
        L.ra_problem_create.restype = i32
        L.ra_problem_destroy.argtypes = [P]
        L.ra_problem_destroy.restype = None
        L.ra_eval_dual.argtypes = [P, P, P, P, P]
        L.ra_eval_dual.restype = i32
        L.ra_eval_records.argtypes = [P, P, P]
        L.ra_eval_records.restype = i32
        L.ra_init_prices.argtypes = [P, P]
        L.ra_init_prices.restype = i32
        L.ra_solve_opts_default.argtypes = [ctypes.POINTER(ra_solve_opts)]
        L.ra_solve_opts_default.restype = None
        L.ra_solve.argtypes = [P, ctypes.POINTER(ra_solve_opts), P, P, P,
                               ctypes.POINTER(ra_solve_info)]
        L.ra_solve.restype = i32
        L.ra_solve_certificate.argtypes = [P, P, P, P]
        L.ra_solve_certificate.restype = i32
        L.ra_solve_history.argtypes = [P, P, i32]
        L.ra_solve_history.restype = i32
        L.ra_recover_primal.argtypes = [P, P, P, P, P, P, P, P, P, ctypes.POINTER(i64)]
        L.ra_recover_primal.restype = i32
        L.ra_batch_rebalance.argtypes = [P, P, P, ctypes.c_double]
        L.ra_batch_rebalance.restype = i32
        L.ra_eval_partial.argtypes = [P, P, P]
        L.ra_eval_partial.restype = i32
        L.ra_combine_partials.argtypes = [i32, i32, P, P, P, P, P, P]
        L.ra_combine_partials.restype = i32
        L.ra_solve_sharded.argtypes = [P, i64, i32, i32, P, P, ALLGATHER_FN, P,
                                       ctypes.POINTER(ra_solve_opts), P, P,
                                       ctypes.POINTER(ra_solve_info)]
        L.ra_solve_sharded.restype = i32
        L.ra_repair_opts_default.argtypes = [ctypes.POINTER(ra_repair_opts)]
        L.ra_repair_opts_default.restype = None
        L.ra_recover_feasible.argtypes = [P, P, ctypes.POINTER(ra_repair_opts), P, P, P,
                                          ctypes.POINTER(ra_repair_info)]
        L.ra_recover_feasible.restype = i32
        L.ra_eval_dual_static.argtypes = [i64, i32, P, P, P, P, P, P, u32, P, P, P]
        L.ra_eval_dual_static.restype = i32
        L.ra_scale_by_demand.argtypes = [i64, i32, P, P, i32, P, P]
        L.ra_scale_by_demand.restype = i32
        L.ra_batch_create.argtypes = [i32, P, P, P, P, P, P, P, u32, P, ctypes.POINTER(P)]
        L.ra_batch_create.restype = i32
        L.ra_batch_create_shaped.argtypes = [i32, P, P, P, P, P, P, P, u32,
                                             ctypes.POINTER(ra_batch_shape), P, ctypes.POINTER(P)]
        L.ra_batch_create_shaped.restype = i32
        L.ra_batch_destroy.argtypes = [P]
        L.ra_batch_destroy.restype = None
        L.ra_batch_prices.argtypes = [P]
        L.ra_batch_prices.restype = i64
        L.ra_batch_solve.argtypes = [P, ctypes.POINTER(ra_solve_opts), P, P, P, P]
        L.ra_batch_solve.restype = i32
        L.ra_mlp_create.argtypes = [P, P, ctypes.POINTER(P)]
        L.ra_mlp_create.restype = i32
        L.ra_mlp_destroy.argtypes = [P]
        L.ra_mlp_destroy.restype = None
        for name in ("ra_mlp_get_params", "ra_mlp_set_params", "ra_mlp_get_grads"):
            getattr(L, name).argtypes = [P, P]
            getattr(L, name).restype = i32
        L.ra_mlp_forward.argtypes = [P, P, i32, P]
        L.ra_mlp_forward.restype = i32
        L.ra_mlp_train_step.argtypes = [P, P, P, i32, ctypes.c_float, P]
        L.ra_mlp_train_step.restype = i32
        L.ra_warmstart_features.argtypes = [P, P]
        L.ra_warmstart_features.restype = i32
        L.ra_batch_features.argtypes = [P, P]
        L.ra_batch_features.restype = i32
        L.ra_warmstart_prices.argtypes = [P, P, P, ctypes.POINTER(i32)]
        L.ra_warmstart_prices.restype = i32
        L.ra_warmstart_used.argtypes = [P, ctypes.POINTER(i32)]
        L.ra_warmstart_used.restype = i32
        L.ra_status_string.argtypes = [i32]
        L.ra_status_string.restype = ctypes.c_char_p
        L.ra_last_error.argtypes = []
        L.ra_last_error.restype = ctypes.c_char_p
        L.ra_version.restype = ctypes.c_char_p
        L.ra_set_wait_timeout.argtypes = [ctypes.c_double]
        L.ra_set_wait_timeout.restype = i32
        _lib = L
    return _lib


def _check(status, ok=(RA_OK,)):
    if status not in ok:
        raise RaError(status, lib().ra_last_error().decode())
    return status


def _ptr(t, dtype=None, numel=None):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"tensor has {t.numel()} elements, need {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ----------------------------------------------------------------------------- C ABI, same names

def ra_problem_create(A, kind, w, param, R, flags=0, stream=None):
    n, m = A.shape
    h = ctypes.c_void_p()
    _check(lib().ra_problem_create(n, m, _ptr(A, torch.float32), _ptr(kind, torch.uint8, n),
                                   _ptr(w, torch.float32, n), _ptr(param, torch.float32, n),
                                   _ptr(R, torch.float64, m), flags, _stream(stream),
                                   ctypes.byref(h)))
    return h


def ra_problem_destroy(h):
    lib().ra_problem_destroy(h)


def ra_eval_dual(h, lam, g=None, q=None, U_lb=None):
    _check(lib().ra_eval_dual(h, _ptr(lam, torch.float64), _ptr(g, torch.float64),
                              _ptr(q, torch.float64), _ptr(U_lb, torch.float64)))


def ra_eval_records(h, j12, t12):
    _check(lib().ra_eval_records(h, _ptr(j12, torch.int32), _ptr(t12, torch.float32)))


def ra_init_prices(h, lam1):
    _check(lib().ra_init_prices(h, _ptr(lam1, torch.float64)))


def ra_solve_opts_default():
    o = ra_solve_opts()
    lib().ra_solve_opts_default(ctypes.byref(o))
    return o


def ra_solve(h, lam_out, opts=None, lam0=None, lam_lb=None, allow_notconv=True):
    info = ra_solve_info()
    o = opts if opts is not None else ra_solve_opts_default()
    ok = (RA_OK, RA_ENOTCONV) if allow_notconv else (RA_OK,)
    _check(lib().ra_solve(h, ctypes.byref(o), _ptr(lam0, torch.float64),
                          _ptr(lam_out, torch.float64), _ptr(lam_lb, torch.float64),
                          ctypes.byref(info)), ok)
    return info.as_dict()


RA_MAX_CERT = 64
RA_HIST_COLS = 6


def ra_solve_certificate(h, m):
    """(theta, lam (k x m), scaled) describing the allocation behind U_lb."""
    import numpy as np
    theta = np.zeros(RA_MAX_CERT)
    lam = np.zeros((RA_MAX_CERT, m))
    scaled = np.zeros(RA_MAX_CERT, np.int32)
    k = lib().ra_solve_certificate(h, ctypes.c_void_p(theta.ctypes.data),
                                   ctypes.c_void_p(lam.ctypes.data),
                                   ctypes.c_void_p(scaled.ctypes.data))
    if k < 0:
        raise RaError(RA_ECUDA, lib().ra_last_error().decode())
    return theta[:k], lam[:k], scaled[:k]


def ra_solve_history(h, cap=512):
    import numpy as np
    buf = np.zeros((cap, RA_HIST_COLS))
    k = lib().ra_solve_history(h, ctypes.c_void_p(buf.ctypes.data), cap)
    if k < 0:
        raise RaError(RA_ECUDA, lib().ra_last_error().decode())
    return buf[:k]


def ra_recover_primal(h, lam, jstar=None, j12=None, x12=None, t=None, X=None, U=None,
                      near_tie=None, count_ties=True):
    cnt = ctypes.c_int64(0)
    _check(lib().ra_recover_primal(h, _ptr(lam, torch.float64), _ptr(jstar, torch.int32),
                                   _ptr(j12, torch.int32), _ptr(x12, torch.float32),
                                   _ptr(t, torch.float32), _ptr(X, torch.float32),
                                   _ptr(U, torch.float64), _ptr(near_tie, torch.uint8),
                                   ctypes.byref(cnt) if count_ties else None))
    return int(cnt.value)


def RA_SHARD_WIDTH(m):
    return 4 + 2 * m


ALLGATHER_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p)


def ra_batch_rebalance(h, lam, R_total, step):
    _check(lib().ra_batch_rebalance(h, _ptr(lam, torch.float64), _ptr(R_total, torch.float64),
                                    float(step)))


def ra_eval_partial(h, lam, part):
    _check(lib().ra_eval_partial(h, _ptr(lam, torch.float64), _ptr(part, torch.float64)))


def ra_combine_partials(parts, m, lam, R, g=None, q=None, stream=None):
    S = parts.numel() // RA_SHARD_WIDTH(m)
    _check(lib().ra_combine_partials(S, m, _ptr(parts, torch.float64), _ptr(lam, torch.float64),
                                     _ptr(R, torch.float64), _ptr(g, torch.float64),
                                     _ptr(q, torch.float64), _stream(stream)))


def ra_solve_sharded(h, n_total, rank, world, send, recv, fn, lam_out, opts=None, lam0=None,
                     allow_notconv=True):
    o = opts or ra_solve_opts_default()
    info = ra_solve_info()
    ok = (RA_OK, RA_ENOTCONV) if allow_notconv else (RA_OK,)
    _check(lib().ra_solve_sharded(h, n_total, rank, world, _ptr(send, torch.float64),
                                  _ptr(recv, torch.float64), fn, None, ctypes.byref(o),
                                  _ptr(lam0, torch.float64), _ptr(lam_out, torch.float64),
                                  ctypes.byref(info)), ok)
    return info.as_dict()


def ra_recover_feasible(h, lam, jk=None, xk=None, X=None, tie_rel=None, max_flex=None):
    o = ra_repair_opts()
    lib().ra_repair_opts_default(ctypes.byref(o))
    if tie_rel is not None:
        o.tie_rel = tie_rel
    if max_flex is not None:
        o.max_flex = max_flex
    info = ra_repair_info()
    _check(lib().ra_recover_feasible(h, _ptr(lam, torch.float64), ctypes.byref(o),
                                     _ptr(jk, torch.int32), _ptr(xk, torch.float32),
                                     _ptr(X, torch.float32), ctypes.byref(info)))
    return info.as_dict()


def ra_scale_by_demand(A, d, A_out=None, stream=None):
    """A_out = A / d for per-job demands (include/ra.h): d of n entries (one
    demand per job) or n x m (per resource).  Returns A_out."""
    n, m = A.shape
    per_res = 1 if d.dim() == 2 else 0
    out = torch.empty_like(A) if A_out is None else A_out
    _check(lib().ra_scale_by_demand(n, m, _ptr(A, torch.float32), _ptr(d, torch.float32, n * m if per_res else n),
                                    per_res, _ptr(out, torch.float32), _stream(stream)))
    return out


def ra_eval_dual_static(A, kind, w, param, R, lam, g, q, flags=0, stream=None):
    """ra_eval_dual without a problem object and without device allocation
    (static scratch inside libra.so; see include/ra.h)."""
    n, m = A.shape
    _check(lib().ra_eval_dual_static(n, m, _ptr(A, torch.float32), _ptr(kind, torch.uint8, n),
                                     _ptr(w, torch.float32, n), _ptr(param, torch.float32, n),
                                     _ptr(R, torch.float64, m), _ptr(lam, torch.float64, m), flags,
                                     _stream(stream), _ptr(g, torch.float64, 1),
                                     _ptr(q, torch.float64, m)))


def ra_batch_create(n, m, A_ptrs, kind_ptrs, w_ptrs, param_ptrs, R_ptrs, flags=0, stream=None,
                    shape=None):
    """n, m: P sizes; *_ptrs: P device addresses (ints) laid out as for
    ra_problem_create; shape: optional (chunk_tiles, whole_tiles, ctas_per_sm)."""
    P = len(n)
    arr = lambda ctype, vals: (ctype * P)(*vals)
    h = ctypes.c_void_p()
    sh = None
    if shape is not None:
        sh = ctypes.byref(ra_batch_shape(int(shape[0]), int(shape[1]), int(shape[2]), 0))
    _check(lib().ra_batch_create_shaped(P, arr(ctypes.c_int64, n), arr(ctypes.c_int32, m),
                                        arr(ctypes.c_void_p, A_ptrs), arr(ctypes.c_void_p, kind_ptrs),
                                        arr(ctypes.c_void_p, w_ptrs), arr(ctypes.c_void_p, param_ptrs),
                                        arr(ctypes.c_void_p, R_ptrs), flags, sh, _stream(stream),
                                        ctypes.byref(h)))
    return h


def ra_batch_destroy(h):
    lib().ra_batch_destroy(h)


def ra_batch_prices(h):
    return int(lib().ra_batch_prices(h))


def ra_batch_solve(h, P, lam_out, opts=None, lam0=None, allow_notconv=True):
    """Returns (list of P info dicts, numpy seconds to each problem's stop)."""
    import numpy as np
    infos = (ra_solve_info * P)()
    secs = np.zeros(P)
    o = opts if opts is not None else ra_solve_opts_default()
    ok = (RA_OK, RA_ENOTCONV) if allow_notconv else (RA_OK,)
    _check(lib().ra_batch_solve(h, ctypes.byref(o), _ptr(lam0, torch.float64),
                                _ptr(lam_out, torch.float64), ctypes.cast(infos, ctypes.c_void_p),
                                ctypes.c_void_p(secs.ctypes.data)), ok)
    return [infos[k].as_dict() for k in range(P)], secs


def ra_mlp_create(theta=None, stream=None):
    """theta: host numpy float32 vector of RA_MLP_PARAMS, or None (zeros)."""
    import numpy as np
    h = ctypes.c_void_p()
    buf = None
    if theta is not None:
        buf = np.ascontiguousarray(theta, dtype=np.float32)
        assert buf.size == RA_MLP_PARAMS
    _check(lib().ra_mlp_create(ctypes.c_void_p(buf.ctypes.data) if buf is not None else None,
                               _stream(stream), ctypes.byref(h)))
    return h


def ra_mlp_destroy(h):
    lib().ra_mlp_destroy(h)


def _mlp_host(fn, h):
    import numpy as np
    out = np.zeros(RA_MLP_PARAMS, np.float32)
    _check(fn(h, ctypes.c_void_p(out.ctypes.data)))
    return out


def ra_mlp_get_params(h):
    return _mlp_host(lib().ra_mlp_get_params, h)


def ra_mlp_get_grads(h):
    return _mlp_host(lib().ra_mlp_get_grads, h)


def ra_mlp_set_params(h, theta):
    import numpy as np
    buf = np.ascontiguousarray(theta, dtype=np.float32)
    assert buf.size == RA_MLP_PARAMS
    _check(lib().ra_mlp_set_params(h, ctypes.c_void_p(buf.ctypes.data)))


def ra_mlp_forward(h, feats, rows, log_lambda):
    _check(lib().ra_mlp_forward(h, _ptr(feats, torch.float32, rows * RA_MLP_IN), rows,
                                _ptr(log_lambda, torch.float32, rows)))


def ra_mlp_train_step(h, feats, target, rows, lr, loss=None):
    _check(lib().ra_mlp_train_step(h, _ptr(feats, torch.float32, rows * RA_MLP_IN),
                                   _ptr(target, torch.float32, rows), rows, float(lr),
                                   _ptr(loss, torch.float32, 1)))


def ra_warmstart_features(h, feats):
    _check(lib().ra_warmstart_features(h, _ptr(feats, torch.float32)))


def ra_batch_features(h, feats):
    _check(lib().ra_batch_features(h, _ptr(feats, torch.float32)))


def ra_warmstart_prices(h, net, lam0, sync=True):
    flag = ctypes.c_int32(-1)
    _check(lib().ra_warmstart_prices(h, net, _ptr(lam0, torch.float64),
                                     ctypes.byref(flag) if sync else None))
    return int(flag.value) if sync else None


def ra_set_wait_timeout(seconds):
    _check(lib().ra_set_wait_timeout(float(seconds)))


def ra_version():
    return lib().ra_version().decode()


# ----------------------------------------------------------------------------- convenience

class AllocationProblem:
    """Problem (e-res-alloc) bound to device tensors, in the spirit of the
    paper's ``AllocationProblem`` (Section 6.1): ``solve()`` then ``prices``
    and ``X``.  Tensors must stay alive with the object."""

    def __init__(self, A, kind, w, param, R, job_cap=True, fp64_jobmath=False, validate=False,
                 stream=None):
        dev = A.device
        self.A = A.contiguous()
        self.kind = kind.to(dev, torch.uint8).contiguous()
        self.w = w.to(dev, torch.float32).contiguous()
        self.param = param.to(dev, torch.float32).contiguous()
        self.R = R.to(dev, torch.float64).contiguous()
        self.n, self.m = self.A.shape
        flags = (0 if job_cap else RA_NO_JOB_CAP) | (RA_FP64_JOBMATH if fp64_jobmath else 0)
        flags |= RA_VALIDATE if validate else 0
        self.stream = stream
        self.handle = ra_problem_create(self.A, self.kind, self.w, self.param, self.R, flags, stream)
        self.prices = None
        self.info = None

    @classmethod
    def from_numpy(cls, prob, device="cuda", **kw):
        t = lambda a: torch.from_numpy(a).to(device)
        return cls(t(prob.A), t(prob.kind), t(prob.w), t(prob.param), t(prob.R), **kw)

    def eval_dual(self, lam, lower_bound=False):
        dev = self.A.device
        lam = torch.as_tensor(lam, dtype=torch.float64, device=dev).contiguous()
        g = torch.empty(1, dtype=torch.float64, device=dev)
        q = torch.empty(self.m, dtype=torch.float64, device=dev)
        U = torch.empty(1, dtype=torch.float64, device=dev) if lower_bound else None
        ra_eval_dual(self.handle, lam, g, q, U)
        return g, q, U

    def eval_records(self):
        """(j12, t12) chosen by the last eval_dual(..., lower_bound=True)."""
        j12 = torch.empty(2 * self.n, dtype=torch.int32, device=self.A.device)
        t12 = torch.empty(2 * self.n, dtype=torch.float32, device=self.A.device)
        ra_eval_records(self.handle, j12, t12)
        return j12, t12

    def init_prices(self):
        lam = torch.empty(self.m, dtype=torch.float64, device=self.A.device)
        ra_init_prices(self.handle, lam)
        return lam

    def solve(self, tol=1e-6, max_evals=500, lam0=None, update="lbfgs", use_graph=True,
              lbfgs_mem=10, master_lb=True, init_step=None, repair_window=None, init_scale=None):
        o = ra_solve_opts_default()
        if init_scale is not None:
            o.init_scale = 1 if init_scale else 0
        o.master_lb = 1 if master_lb else 0
        if repair_window is not None:
            o.repair_window = repair_window
        if init_step is not None:
            o.init_step = init_step
        o.tol_rel = tol
        o.max_evals = max_evals
        o.lbfgs_mem = lbfgs_mem
        o.update = {"lbfgs": 0, "subgradient": 1, "lbfgs-scalar": 2, "lbfgs-diag": 3}[update]
        o.use_graph = 1 if use_graph else 0
        lam = torch.empty(self.m, dtype=torch.float64, device=self.A.device)
        lam_lb = torch.empty(self.m, dtype=torch.float64, device=self.A.device)
        if lam0 is not None:
            lam0 = torch.as_tensor(lam0, dtype=torch.float64, device=self.A.device).contiguous()
        self.info = ra_solve(self.handle, lam, o, lam0, lam_lb)
        self.prices = lam
        self.prices_lb = lam_lb
        return self.info

    def certificate(self):
        """(theta, lam, scaled): the allocation behind the last solve's U_lb is
        sum_k theta_k X(lam_k), column-scaled where scaled[k] == 1; scaled ==
        [2] marks the repaired allocation recover_feasible(lam[0]) returns."""
        return ra_solve_certificate(self.handle, self.m)

    def history(self):
        """Rows (evaluation, g, best U_lb, relative gap, master-LP bound, LP
        pivots) of the last solve."""
        return ra_solve_history(self.handle)

    def verbose_log(self, every=5):
        """The paper's verbose lines (Section 6.1): per-job utility, dual value, gap."""
        h = self.history()
        lines = []
        for k, (ev, g, ub, gap) in enumerate(h[:, :4]):
            if k % every == 0:
                lines.append(f"iteration {int(ev):02d} | utility={ub / self.n:.6g} | "
                             f"dual_value={g / self.n:.6g} | gap={gap:.2e}")
        if len(h):
            lines.append(f"Converged in {int(h[-1][0]):03d} evaluations, with residual "
                         f"{(h[-1][1] - h[-1][2]) / self.n:.6g}")
        return lines

    def features(self):
        """Warm-start network input, (m, 26) FP32 on the device."""
        f = torch.empty((self.m, RA_MLP_IN), dtype=torch.float32, device=self.A.device)
        ra_warmstart_features(self.handle, f)
        return f

    def warm_prices(self, net, sync=True):
        """(lambda0, used_warm): the network's prices if their dual value is not
        larger than the cold start's, else Eq. e-initialization.  With
        sync=False nothing waits for the choice (used_warm is None; ask
        warm_used() later)."""
        lam0 = torch.empty(self.m, dtype=torch.float64, device=self.A.device)
        used = ra_warmstart_prices(self.handle, net.handle, lam0, sync)
        return lam0, (bool(used) if sync else None)

    def warm_used(self):
        """Whether the last warm_prices kept the network's prices (synchronises)."""
        v = ctypes.c_int32(0)
        _check(lib().ra_warmstart_used(self.handle, ctypes.byref(v)))
        return bool(v.value)

    def recover(self, lam=None, dense=False):
        lam = self.prices if lam is None else torch.as_tensor(lam, dtype=torch.float64,
                                                             device=self.A.device).contiguous()
        dev = self.A.device
        out = dict(jstar=torch.empty(self.n, dtype=torch.int32, device=dev),
                   j12=torch.empty(2 * self.n, dtype=torch.int32, device=dev),
                   x12=torch.empty(2 * self.n, dtype=torch.float32, device=dev),
                   t=torch.empty(self.n, dtype=torch.float32, device=dev),
                   U=torch.empty(1, dtype=torch.float64, device=dev),
                   near_tie=torch.empty(self.n, dtype=torch.uint8, device=dev))
        if dense:
            out["X"] = torch.empty(self.n * self.m, dtype=torch.float32, device=dev)
        out["n_near_ties"] = ra_recover_primal(self.handle, lam, out["jstar"], out["j12"],
                                               out["x12"], out["t"], out.get("X"), out["U"],
                                               out["near_tie"])
        return out

    @property
    def X(self):
        return self.recover(dense=True)["X"].view(self.n, self.m)

    def recover_feasible(self, lam=None, dense=False, tie_rel=None, max_flex=None):
        """A feasible allocation at lam (default: the last solve's best
        prices) with the jobs at ties re-mixed (ra_recover_feasible): jk, xk
        (4 (resource, fraction) pairs per job), X when dense, and info."""
        lam = self.prices if lam is None else torch.as_tensor(lam, dtype=torch.float64,
                                                             device=self.A.device).contiguous()
        dev = self.A.device
        out = dict(jk=torch.empty(4 * self.n, dtype=torch.int32, device=dev),
                   xk=torch.empty(4 * self.n, dtype=torch.float32, device=dev))
        if dense:
            out["X"] = torch.empty(self.n * self.m, dtype=torch.float32, device=dev)
        out["info"] = ra_recover_feasible(self.handle, lam, out["jk"], out["xk"], out.get("X"),
                                          tie_rel=tie_rel, max_flex=max_flex)
        return out

    def close(self):
        if getattr(self, "handle", None):
            ra_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _pack(arrays, align_elems=16):
    """Concatenate 1-D numpy arrays with every segment starting on a multiple
    of align_elems elements; returns (buffer, offsets)."""
    import numpy as np
    offs, pos = [], 0
    for a in arrays:
        offs.append(pos)
        pos += (a.size + align_elems - 1) // align_elems * align_elems
    buf = np.zeros(max(pos, align_elems), dtype=arrays[0].dtype)
    for a, o in zip(arrays, offs):
        buf[o:o + a.size] = a.ravel()
    return buf, offs


class AllocationBatch:
    """P independent problems solved together (batched price discovery).
    Each problem's arrays live in one packed device buffer per field, every
    segment 16-byte aligned."""

    def __init__(self, problems, job_cap=True, device="cuda", stream=None, pinned=False,
                 shape=None):
        import numpy as np
        self.P = len(problems)
        self.n = [int(p.A.shape[0]) for p in problems]
        self.m = [int(p.A.shape[1]) for p in problems]
        host = {}
        for f, dt in (("A", np.float32), ("kind", np.uint8), ("w", np.float32),
                      ("param", np.float32), ("R", np.float64)):
            buf, offs = _pack([np.ascontiguousarray(getattr(p, f), dtype=dt).ravel() for p in problems])
            t = torch.from_numpy(buf)
            if pinned:
                t = t.pin_memory()
            host[f] = (t, offs)
        self.dev = {f: t.to(device, non_blocking=pinned) for f, (t, _) in host.items()}
        self.offs = {f: o for f, (_, o) in host.items()}
        self.h2d_bytes = sum(t.numel() * t.element_size() for t, _ in host.values())
        esz = {"A": 4, "kind": 1, "w": 4, "param": 4, "R": 8}
        ptrs = {f: [self.dev[f].data_ptr() + o * esz[f] for o in self.offs[f]] for f in esz}
        self.flags = 0 if job_cap else RA_NO_JOB_CAP
        self.stream = stream
        self.shape = shape
        self.handle = ra_batch_create(self.n, self.m, ptrs["A"], ptrs["kind"], ptrs["w"],
                                      ptrs["param"], ptrs["R"], self.flags, stream, shape)
        self.m_total = ra_batch_prices(self.handle)
        self.lam_off = np.concatenate([[0], np.cumsum(self.m)[:-1]]).astype(np.int64)
        self.prices = None

    @classmethod
    def from_tensors(cls, tensors, job_cap=True, stream=None, shape=None):
        """Batch over device tensors (A, kind, w, param, R) per problem, used in
        place (they must stay alive with the batch; each is kept referenced)."""
        import numpy as np
        self = cls.__new__(cls)
        self.P = len(tensors)
        self.n = [int(t[0].shape[0]) for t in tensors]
        self.m = [int(t[0].shape[1]) for t in tensors]
        self.tensors = [tuple(x.contiguous() for x in t) for t in tensors]
        self.dev = {"A": self.tensors[0][0]}
        self.flags = 0 if job_cap else RA_NO_JOB_CAP
        self.stream = stream
        cols = list(zip(*self.tensors))
        ptrs = [[x.data_ptr() for x in col] for col in cols]
        self.shape = shape
        self.handle = ra_batch_create(self.n, self.m, *ptrs, self.flags, stream, shape)
        self.m_total = ra_batch_prices(self.handle)
        self.lam_off = np.concatenate([[0], np.cumsum(self.m)[:-1]]).astype(np.int64)
        self.prices = None
        return self

    def solve(self, tol=1e-6, max_evals=500, lam0=None, use_graph=True, master_lb=True,
              lbfgs_mem=10, init_step=None):
        o = ra_solve_opts_default()
        if init_step is not None:
            o.init_step = init_step
        o.tol_rel = tol
        o.max_evals = max_evals
        o.use_graph = 1 if use_graph else 0
        o.master_lb = 1 if master_lb else 0
        o.lbfgs_mem = lbfgs_mem
        dev = self.dev["A"].device
        lam = torch.empty(self.m_total, dtype=torch.float64, device=dev)
        if lam0 is not None:
            lam0 = torch.as_tensor(lam0, dtype=torch.float64, device=dev).contiguous()
        self.infos, self.seconds = ra_batch_solve(self.handle, self.P, lam, o, lam0)
        self.prices = lam
        return self.infos, self.seconds

    def features(self):
        """Warm-start network input of every problem, (sum m, 26) FP32."""
        f = torch.empty((self.m_total, RA_MLP_IN), dtype=torch.float32, device=self.dev["A"].device)
        ra_batch_features(self.handle, f)
        return f

    def prices_of(self, k):
        o = int(self.lam_off[k])
        return self.prices[o:o + self.m[k]]

    def close(self):
        if getattr(self, "handle", None):
            ra_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WarmStartMLP:
    """The warm-start network (parameters, Adam state and activations on the
    device); training and inference run in libra's kernels."""

    def __init__(self, theta=None, stream=None):
        self.stream = stream
        self.handle = ra_mlp_create(theta, stream)

    def params(self):
        return ra_mlp_get_params(self.handle)

    def set_params(self, theta):
        ra_mlp_set_params(self.handle, theta)

    def grads(self):
        return ra_mlp_get_grads(self.handle)

    def forward(self, feats):
        feats = feats.contiguous()
        rows = feats.shape[0]
        out = torch.empty(rows, dtype=torch.float32, device=feats.device)
        ra_mlp_forward(self.handle, feats, rows, out)
        return out

    def train_step(self, feats, target, lr):
        rows = feats.shape[0]
        loss = torch.empty(1, dtype=torch.float32, device=feats.device)
        ra_mlp_train_step(self.handle, feats.contiguous(), target.contiguous(), rows, lr, loss)
        return loss

    def close(self):
        if getattr(self, "handle", None):
            ra_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
