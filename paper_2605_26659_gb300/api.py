"""Thin Python binding of libfinom (include/finom.h), same names as the C ABI.

Argument marshalling only: device arrays are torch CUDA tensors (float64,
contiguous) passed as raw pointers; every computation runs in the CUDA
library.  There is no CPU fallback: if libfinom.so cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfinom.so")

(FINOM_OK, FINOM_EINVAL, FINOM_ENOMEM, FINOM_ECUDA, FINOM_EDEVICE_TIMEOUT, FINOM_ENOTSUP, FINOM_EPENDING,
 FINOM_ECANCELED) = range(8)
F64, F32_LOG = 0, 1
_PREC = {"f64": F64, "fp64": F64, "float64": F64, F64: F64,
         "f32_log": F32_LOG, "fp32_log": F32_LOG, "f32": F32_LOG, F32_LOG: F32_LOG}


class FinomError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"finom status {status}: {msg}")
        self.status = status


class FinomResult(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_double), ("marginal_err", ctypes.c_double),
                ("marginal_err_loop", ctypes.c_double), ("dual", ctypes.c_double),
                ("iters", ctypes.c_int64), ("converged", ctypes.c_int32), ("status", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FinomServerDone(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("kind", ctypes.c_int32), ("status", ctypes.c_int32),
                ("result", FinomResult), ("latency_s", ctypes.c_double), ("queue_s", ctypes.c_double)]


_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_I32 = ctypes.c_int32

_SIGS = {
    "finom_version": ([], ctypes.c_int),
    "finom_last_error": ([], ctypes.c_char_p),
    "finom_plan": ([_P, _I64, _P, _I64, _D, ctypes.c_int, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "finom_plan_destroy": ([_P], ctypes.c_int),
    "finom_plan_info": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_D),
                         ctypes.POINTER(_I32)], ctypes.c_int),
    "finom_dividing_index": ([_P, _P, _P, _P], ctypes.c_int),
    "finom_kv": ([_P, _P, _P, _P], ctypes.c_int),
    "finom_ktu": ([_P, _P, _P, _P], ctypes.c_int),
    "finom_kv_log": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "finom_ktu_log": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "finom_solve": ([_P, _P, _P, _D, _I64, _P, _P, _I32, ctypes.POINTER(FinomResult), _P], ctypes.c_int),
    "finom_solve_begin": ([_P, _P, _P, _D, _I64, _P, _P, _P], ctypes.c_int),
    "finom_solve_step": ([_P, _I64, _P], ctypes.c_int),
    "finom_solve_poll": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64), _P], ctypes.c_int),
    "finom_solve_end": ([_P, _P, _P, ctypes.POINTER(FinomResult), _P], ctypes.c_int),
    "finom_cost": ([_P, _P, _P, _P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D), _P], ctypes.c_int),
    "finom_kv_log_noalloc": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "finom_plan_2d": ([_P, _P, _I64, _P, _P, _I64, _D, ctypes.c_int, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "finom_plan_shape": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64), ctypes.POINTER(_I64)], ctypes.c_int),
    "finom_plan_nd": ([_I32, _P, _P, _P, _D, ctypes.c_int, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "finom_plan_axes": ([_P, ctypes.POINTER(_I32), _P], ctypes.c_int),
    "finom_plan_batch": ([_P, _P, _P, _P, _I64, _P, ctypes.c_int, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "finom_plan_instances": ([_P, ctypes.POINTER(_I64)], ctypes.c_int),
    "finom_plan_batch_elems": ([_P, _P, _P, _P, _I64, _P, ctypes.c_int, _I32, _P, ctypes.POINTER(_P)],
                               ctypes.c_int),
    "finom_tune_set_batch": ([ctypes.c_int, _I32], ctypes.c_int),
    "finom_tune_get_batch": ([ctypes.c_int, ctypes.POINTER(_I32)], ctypes.c_int),
    "finom_solve_batch": ([_P, _P, _P, _D, _I64, _P, _P, _P, _P], ctypes.c_int),
    "finom_solve_batch_begin": ([_P, _P, _P, _D, _I64, _P], ctypes.c_int),
    "finom_solve_batch_step": ([_P, _I64, _P], ctypes.c_int),
    "finom_solve_batch_end": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "finom_solve_trace": ([_P, _P, _P, _I64, _I64, _P, _P, ctypes.POINTER(_I64), _P], ctypes.c_int),
    "finom_solve_eps_scaling": ([_P, _P, _P, _D, _I64, _D, _D, _D, _P, _P, ctypes.POINTER(FinomResult), _P],
                                ctypes.c_int),
    "finom_transport_row": ([_P, _P, _P, _I64, _P, _P], ctypes.c_int),
    "finom_transport_col": ([_P, _P, _P, _I64, _P, _P], ctypes.c_int),
    "finom_barycentric": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "finom_plan_set_elems": ([_P, _I32, _P], ctypes.c_int),
    "finom_plan_elems": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64)], ctypes.c_int),
    "finom_tune_set": ([ctypes.c_int, _I32, _I32], ctypes.c_int),
    "finom_tune_get": ([ctypes.c_int, _I32, ctypes.POINTER(_I32)], ctypes.c_int),
    "finom_autotune": ([ctypes.c_int, _I32, _I32, ctypes.POINTER(_I32), _P, _P], ctypes.c_int),
    "finom_server_create": ([_I64, _I32, ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
    "finom_server_submit_1d": ([_P, _P, _I64, _P, _I64, _P, _P, _D, _D, _I64, ctypes.POINTER(_I64)], ctypes.c_int),
    "finom_server_submit_2d": ([_P, _P, _P, _I64, _P, _P, _I64, _P, _P, _D, _D, _I64, ctypes.POINTER(_I64)],
                               ctypes.c_int),
    "finom_server_step": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32)], ctypes.c_int),
    "finom_server_result": ([_P, _I64, ctypes.POINTER(FinomServerDone), _P, _P], ctypes.c_int),
    "finom_server_cancel": ([_P, _I64], ctypes.c_int),
    "finom_server_set_eps_scaling": ([_P, _I32, _D, _D], ctypes.c_int),
    "finom_server_set_policy": ([_P, _I32], ctypes.c_int),
    "finom_server_set_batching": ([_P, _I64], ctypes.c_int),
    "finom_server_destroy": ([_P], ctypes.c_int),
}


def load(path: str | None = None):
    """Load libfinom.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    p = path or LIB_PATH
    if path is None and not _build.up_to_date():
        _build.build()
    if not os.path.exists(p):
        raise FinomError(-1, f"libfinom.so not found at {p}; run paper_2605_26659_gb300/build.py")
    lib = ctypes.CDLL(p)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    cache = os.environ.get("FINOM_TUNE_CACHE")
    if cache and os.path.exists(cache):
        from . import autotune
        autotune.apply(cache)
    return lib


def _check(rc):
    if rc != FINOM_OK:
        raise FinomError(rc, _lib.finom_last_error().decode())


def _dev(t, n=None, dtype=None, name="array"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} entries, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


@dataclass
class Plan:
    handle: ctypes.c_void_p
    N: int
    M: int
    eps: float
    precision: int
    device: int
    dim: int = 1
    nx: int = 0          # 2D: grid side along x (N)
    ny: int = 0          # 2D: grid side along y (M)
    batch: int = 0       # batch plans: number of instances

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.finom_plan_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def finom_version():
    return load().finom_version()


def finom_plan(x, y, eps, precision="f32_log", stream=None) -> Plan:
    import torch
    load()
    N, M = x.numel(), y.numel()
    h = ctypes.c_void_p()
    _check(_lib.finom_plan(_dev(x, N, torch.float64, "x"), N, _dev(y, M, torch.float64, "y"), M,
                           float(eps), _PREC[precision], _stream(stream), ctypes.byref(h)))
    return Plan(h, N, M, float(eps), _PREC[precision], x.device.index or 0)


def finom_plan_2d(x1, x2, y1, y2, eps, precision="f32_log", stream=None) -> Plan:
    """Plan for the grids x1 (x) y1 and x2 (x) y2.  Grid arrays of the other
    calls are flat, column-major: point (k, i) at k + N*i."""
    import torch
    load()
    N, M = x1.numel(), y1.numel()
    h = ctypes.c_void_p()
    _check(_lib.finom_plan_2d(_dev(x1, N, torch.float64, "x1"), _dev(x2, N, torch.float64, "x2"), N,
                              _dev(y1, M, torch.float64, "y1"), _dev(y2, M, torch.float64, "y2"), M,
                              float(eps), _PREC[precision], _stream(stream), ctypes.byref(h)))
    return Plan(h, N * M, N * M, float(eps), _PREC[precision], x1.device.index or 0, 2, N, M)


def finom_plan_nd(xs, ys, eps, precision="f32_log", stream=None) -> Plan:
    """Plan for the d-dimensional grids x^1 (x) ... (x) x^d (mu) and
    y^1 (x) ... (x) y^d (nu): xs, ys are sequences of d device float64
    tensors (axis k of each grid).  Grid arrays of the other calls are flat
    with axis 0 fastest."""
    import torch
    load()
    d = len(xs)
    if len(ys) != d:
        raise ValueError("xs and ys need the same number of axes")
    n = (ctypes.c_int64 * d)(*[int(x.numel()) for x in xs])
    px = (ctypes.c_void_p * d)(*[_dev(x, int(x.numel()), torch.float64, f"xs[{k}]") for k, x in enumerate(xs)])
    py = (ctypes.c_void_p * d)(*[_dev(y, int(n[k]), torch.float64, f"ys[{k}]") for k, y in enumerate(ys)])
    h = ctypes.c_void_p()
    _check(_lib.finom_plan_nd(d, ctypes.cast(n, ctypes.c_void_p), ctypes.cast(px, ctypes.c_void_p),
                              ctypes.cast(py, ctypes.c_void_p), float(eps), _PREC[precision], _stream(stream),
                              ctypes.byref(h)))
    G = 1
    for v in n:
        G *= v
    return Plan(h, G, G, float(eps), _PREC[precision], xs[0].device.index or 0, d, int(n[0]), G // int(n[0]))


def finom_plan_axes(plan: Plan):
    d = _I32()
    n = (ctypes.c_int64 * 8)()
    _check(_lib.finom_plan_axes(plan.handle, ctypes.byref(d), ctypes.cast(n, ctypes.c_void_p)))
    return list(n[:d.value])


def finom_plan_shape(plan: Plan):
    d, n, m = _I32(), _I64(), _I64()
    _check(_lib.finom_plan_shape(plan.handle, ctypes.byref(d), ctypes.byref(n), ctypes.byref(m)))
    return d.value, n.value, m.value


def finom_plan_batch(x, offx, y, offy, eps, precision="f32_log", stream=None, elems=0) -> Plan:
    """Batch of independent 1D problems: x, y concatenated (device float64),
    offx, offy: B + 1 offsets (host sequences), eps: B values (host); elems:
    points per thread of the packing (0: the tuning table's batch entry)."""
    import numpy as np
    import torch
    load()
    ox = np.ascontiguousarray(offx, dtype=np.int64)
    oy = np.ascontiguousarray(offy, dtype=np.int64)
    ep = np.ascontiguousarray(eps, dtype=np.float64)
    B = len(ep)
    if len(ox) != B + 1 or len(oy) != B + 1:
        raise ValueError("offx and offy need B + 1 entries")
    h = ctypes.c_void_p()
    _check(_lib.finom_plan_batch_elems(_dev(x, int(ox[-1]), torch.float64, "x"), ox.ctypes.data,
                                       _dev(y, int(oy[-1]), torch.float64, "y"), oy.ctypes.data, B,
                                       ep.ctypes.data, _PREC[precision], int(elems), _stream(stream),
                                       ctypes.byref(h)))
    return Plan(h, int(ox[-1]), int(oy[-1]), float(ep[0]), _PREC[precision], x.device.index or 0, batch=B)


def finom_plan_instances(plan: Plan):
    b = _I64()
    _check(_lib.finom_plan_instances(plan.handle, ctypes.byref(b)))
    return b.value


def finom_solve_batch(plan: Plan, u, v, tol, maxit, f=None, g=None, stream=None):
    """Solve every instance; returns (f, g, list of per-instance result dicts)."""
    import torch
    dev = torch.device("cuda", plan.device)
    if f is None:
        f = torch.empty(plan.N, dtype=torch.float64, device=dev)
    if g is None:
        g = torch.empty(plan.M, dtype=torch.float64, device=dev)
    res = (FinomResult * plan.batch)()
    _check(_lib.finom_solve_batch(plan.handle, _dev(u, plan.N, torch.float64, "u"),
                                  _dev(v, plan.M, torch.float64, "v"), float(tol), int(maxit),
                                  _dev(f, plan.N, torch.float64, "f"), _dev(g, plan.M, torch.float64, "g"),
                                  ctypes.cast(res, ctypes.c_void_p), _stream(stream)))
    return f, g, [r.as_dict() for r in res]


def finom_solve_batch_begin(plan: Plan, u, v, tol, maxit, stream=None):
    import torch
    _check(_lib.finom_solve_batch_begin(plan.handle, _dev(u, plan.N, torch.float64, "u"),
                                        _dev(v, plan.M, torch.float64, "v"), float(tol), int(maxit),
                                        _stream(stream)))


def finom_solve_batch_step(plan: Plan, iterations, stream=None):
    _check(_lib.finom_solve_batch_step(plan.handle, int(iterations), _stream(stream)))


def finom_solve_batch_end(plan: Plan, f=None, g=None, stream=None):
    import torch
    dev = torch.device("cuda", plan.device)
    if f is None:
        f = torch.empty(plan.N, dtype=torch.float64, device=dev)
    if g is None:
        g = torch.empty(plan.M, dtype=torch.float64, device=dev)
    res = (FinomResult * plan.batch)()
    _check(_lib.finom_solve_batch_end(plan.handle, _dev(f, plan.N), _dev(g, plan.M),
                                      ctypes.cast(res, ctypes.c_void_p), _stream(stream)))
    return f, g, [r.as_dict() for r in res]


def finom_solve_trace(plan: Plan, u, v, maxit, every=10, stream=None):
    """Loop-head marginal error against GPU time: returns (iterations, err, ms)
    as numpy arrays, one entry per `every` iterations."""
    import numpy as np
    import torch
    K = (int(maxit) + int(every) - 1) // int(every)
    err = np.zeros(K)
    ms = np.zeros(K)
    n = _I64()
    _check(_lib.finom_solve_trace(plan.handle, _dev(u, plan.N, torch.float64, "u"), _dev(v, plan.M, torch.float64, "v"),
                                  int(maxit), int(every), err.ctypes.data, ms.ctypes.data, ctypes.byref(n),
                                  _stream(stream)))
    k = n.value
    its = np.minimum((np.arange(k) + 1) * int(every), int(maxit) - 1)
    return its, err[:k], ms[:k]


def finom_solve_eps_scaling(plan: Plan, u, v, tol, maxit, eps0, factor=0.5, tol_stage=1e-4, stream=None):
    """finom_solve preceded by warm-started solves at eps0, eps0*factor, ...;
    returns (f, g, result dict)."""
    import torch
    dev = torch.device("cuda", plan.device)
    f = torch.empty(plan.N, dtype=torch.float64, device=dev)
    g = torch.empty(plan.M, dtype=torch.float64, device=dev)
    res = FinomResult()
    _check(_lib.finom_solve_eps_scaling(plan.handle, _dev(u, plan.N, torch.float64, "u"),
                                        _dev(v, plan.M, torch.float64, "v"), float(tol), int(maxit), float(eps0),
                                        float(factor), float(max(tol_stage, tol)), _dev(f, plan.N),
                                        _dev(g, plan.M), ctypes.byref(res), _stream(stream)))
    return f, g, res.as_dict()


def finom_transport_row(plan: Plan, f, g, i, out=None, stream=None):
    """Row i of the transport plan (M entries)."""
    import torch
    out = _out(plan.M, plan, out)
    _check(_lib.finom_transport_row(plan.handle, _dev(f, plan.N, torch.float64, "f"),
                                    _dev(g, plan.M, torch.float64, "g"), int(i), _dev(out, plan.M), _stream(stream)))
    return out


def finom_transport_col(plan: Plan, f, g, j, out=None, stream=None):
    """Column j of the transport plan (N entries)."""
    import torch
    out = _out(plan.N, plan, out)
    _check(_lib.finom_transport_col(plan.handle, _dev(f, plan.N, torch.float64, "f"),
                                    _dev(g, plan.M, torch.float64, "g"), int(j), _dev(out, plan.N), _stream(stream)))
    return out


def finom_barycentric(plan: Plan, f, g, stream=None):
    """Barycentric projections (tx on x, ty on y) of the transport plan."""
    import torch
    tx, ty = _out(plan.N, plan, None), _out(plan.M, plan, None)
    _check(_lib.finom_barycentric(plan.handle, _dev(f, plan.N, torch.float64, "f"),
                                  _dev(g, plan.M, torch.float64, "g"), _dev(tx, plan.N), _dev(ty, plan.M),
                                  _stream(stream)))
    return tx, ty


def finom_plan_set_elems(plan: Plan, elems, stream=None):
    """Force the kernel's points per thread (1, 2, 4 or 8) on a 1D plan."""
    _check(_lib.finom_plan_set_elems(plan.handle, int(elems), _stream(stream)))


def finom_plan_elems(plan: Plan):
    """(points per thread, tiles) of a plan."""
    e, t = _I32(), _I64()
    _check(_lib.finom_plan_elems(plan.handle, ctypes.byref(e), ctypes.byref(t)))
    return e.value, t.value


def finom_tune_set(precision, log2_bucket, elems):
    load()
    _check(_lib.finom_tune_set(_PREC[precision], int(log2_bucket), int(elems)))


def finom_tune_get(precision, log2_bucket):
    load()
    e = _I32()
    _check(_lib.finom_tune_get(_PREC[precision], int(log2_bucket), ctypes.byref(e)))
    return e.value


def finom_tune_set_batch(precision, elems):
    load()
    _check(_lib.finom_tune_set_batch(_PREC[precision], int(elems)))


def finom_tune_get_batch(precision):
    load()
    e = _I32()
    _check(_lib.finom_tune_get_batch(_PREC[precision], ctypes.byref(e)))
    return e.value


def finom_autotune(precision, log2_bucket, iters=64, stream=None):
    """Time the tile kinds E = -1 (64-point tiles), 1, 2, 4, 8 on a synthetic
    problem of 2^log2_bucket merged points, install the fastest; returns
    (best, {E: us per iteration})."""
    load()
    best = _I32()
    t = (ctypes.c_double * 5)()
    _check(_lib.finom_autotune(_PREC[precision], int(log2_bucket), int(iters), ctypes.byref(best),
                               ctypes.cast(t, ctypes.c_void_p), _stream(stream)))
    return best.value, dict(zip((-1, 1, 2, 4, 8), list(t)))


def finom_plan_destroy(plan: Plan):
    if plan.handle:
        _check(_lib.finom_plan_destroy(plan.handle))
        plan.handle = None


def finom_plan_info(plan: Plan):
    n, m, e, p = _I64(), _I64(), _D(), _I32()
    _check(_lib.finom_plan_info(plan.handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(e), ctypes.byref(p)))
    return n.value, m.value, e.value, p.value


def finom_dividing_index(plan: Plan, stream=None):
    import torch
    dev = torch.device("cuda", plan.device)
    z = torch.empty(plan.N, dtype=torch.int32, device=dev)
    zt = torch.empty(plan.M, dtype=torch.int32, device=dev)
    _check(_lib.finom_dividing_index(plan.handle, _dev(z), _dev(zt), _stream(stream)))
    return z, zt


def _out(n, plan, out):
    import torch
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=torch.device("cuda", plan.device))
    return out


def finom_kv(plan: Plan, v, out=None, stream=None):
    import torch
    out = _out(plan.N, plan, out)
    _check(_lib.finom_kv(plan.handle, _dev(v, plan.M, torch.float64, "v"), _dev(out, plan.N), _stream(stream)))
    return out


def finom_ktu(plan: Plan, u, out=None, stream=None):
    import torch
    out = _out(plan.M, plan, out)
    _check(_lib.finom_ktu(plan.handle, _dev(u, plan.N, torch.float64, "u"), _dev(out, plan.M), _stream(stream)))
    return out


def finom_kv_log(plan: Plan, a, b, out=None, stream=None):
    import torch
    out = _out(plan.N, plan, out)
    _check(_lib.finom_kv_log(plan.handle, _dev(a, plan.N, torch.float64, "a"),
                             _dev(b, plan.M, torch.float64, "b"), _dev(out, plan.N), _stream(stream)))
    return out


def finom_ktu_log(plan: Plan, a, b, out=None, stream=None):
    import torch
    out = _out(plan.M, plan, out)
    _check(_lib.finom_ktu_log(plan.handle, _dev(a, plan.N, torch.float64, "a"),
                              _dev(b, plan.M, torch.float64, "b"), _dev(out, plan.M), _stream(stream)))
    return out


def finom_solve(plan: Plan, u, v, tol, maxit, f=None, g=None, warm=False, stream=None):
    """Run the Sinkhorn loop; returns (f, g, result dict)."""
    import torch
    dev = torch.device("cuda", plan.device)
    if f is None:
        f = torch.empty(plan.N, dtype=torch.float64, device=dev)
    if g is None:
        g = torch.empty(plan.M, dtype=torch.float64, device=dev)
    res = FinomResult()
    _check(_lib.finom_solve(plan.handle, _dev(u, plan.N, torch.float64, "u"), _dev(v, plan.M, torch.float64, "v"),
                            float(tol), int(maxit), _dev(f, plan.N, torch.float64, "f"),
                            _dev(g, plan.M, torch.float64, "g"), 1 if warm else 0, ctypes.byref(res),
                            _stream(stream)))
    return f, g, res.as_dict()


def finom_solve_begin(plan: Plan, u, v, tol, maxit, f0=None, g0=None, stream=None):
    import torch
    fp = _dev(f0, plan.N, torch.float64, "f0") if f0 is not None else None
    gp = _dev(g0, plan.M, torch.float64, "g0") if g0 is not None else None
    _check(_lib.finom_solve_begin(plan.handle, _dev(u, plan.N, torch.float64, "u"),
                                  _dev(v, plan.M, torch.float64, "v"), float(tol), int(maxit), fp, gp,
                                  _stream(stream)))


def finom_solve_step(plan: Plan, iterations, stream=None):
    _check(_lib.finom_solve_step(plan.handle, int(iterations), _stream(stream)))


def finom_solve_poll(plan: Plan, stream=None):
    d, it = _I32(), _I64()
    _check(_lib.finom_solve_poll(plan.handle, ctypes.byref(d), ctypes.byref(it), _stream(stream)))
    return bool(d.value), it.value


def finom_solve_end(plan: Plan, f=None, g=None, stream=None):
    import torch
    dev = torch.device("cuda", plan.device)
    if f is None:
        f = torch.empty(plan.N, dtype=torch.float64, device=dev)
    if g is None:
        g = torch.empty(plan.M, dtype=torch.float64, device=dev)
    res = FinomResult()
    _check(_lib.finom_solve_end(plan.handle, _dev(f, plan.N), _dev(g, plan.M), ctypes.byref(res), _stream(stream)))
    return f, g, res.as_dict()


def finom_cost(plan: Plan, u, v, f, g, stream=None):
    import torch
    w1, err = _D(), _D()
    _check(_lib.finom_cost(plan.handle, _dev(u, plan.N, torch.float64, "u"), _dev(v, plan.M, torch.float64, "v"),
                           _dev(f, plan.N, torch.float64, "f"), _dev(g, plan.M, torch.float64, "g"),
                           ctypes.byref(w1), ctypes.byref(err), _stream(stream)))
    return w1.value, err.value


def finom_kv_log_noalloc(plan: Plan, a, b, out=None, stream=None):
    """finom_kv_log without device allocation inside the library (static scratch)."""
    import torch
    out = _out(plan.N, plan, out)
    _check(_lib.finom_kv_log_noalloc(plan.handle, _dev(a, plan.N, torch.float64, "a"),
                                     _dev(b, plan.M, torch.float64, "b"), _dev(out, plan.N), _stream(stream)))
    return out


# ---------------------------------------------------------------------------
# serving loop (host arrays in, host arrays out)

def _host(a, n, name):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"{name} must have {n} entries, got {a.size}")
    return a


class Server:
    """finom_server_*: continuous batching of 1D and 2D solves on one GPU."""

    def __init__(self, mem_budget_bytes, max_active=16, precision="f32_log"):
        load()
        h = ctypes.c_void_p()
        _check(_lib.finom_server_create(int(mem_budget_bytes), int(max_active), _PREC[precision],
                                        ctypes.byref(h)))
        self.handle = h
        self._shape = {}

    def submit_1d(self, x, y, u, v, eps, tol, maxit):
        import numpy as np
        N, M = np.size(x), np.size(y)
        x, y, u, v = _host(x, N, "x"), _host(y, M, "y"), _host(u, N, "u"), _host(v, M, "v")
        rid = ctypes.c_int64()
        _check(_lib.finom_server_submit_1d(self.handle, x.ctypes.data, N, y.ctypes.data, M, u.ctypes.data,
                                           v.ctypes.data, float(eps), float(tol), int(maxit), ctypes.byref(rid)))
        self._shape[rid.value] = (N, M)
        return rid.value

    def submit_2d(self, x1, x2, y1, y2, U, V, eps, tol, maxit):
        """U, V: (N, M) arrays, point (k, i) at [k, i] (passed column-major)."""
        import numpy as np
        N, M = np.size(x1), np.size(y1)
        x1, x2, y1, y2 = _host(x1, N, "x1"), _host(x2, N, "x2"), _host(y1, M, "y1"), _host(y2, M, "y2")
        U = _host(np.asarray(U).ravel(order="F"), N * M, "U")
        V = _host(np.asarray(V).ravel(order="F"), N * M, "V")
        rid = ctypes.c_int64()
        _check(_lib.finom_server_submit_2d(self.handle, x1.ctypes.data, x2.ctypes.data, N, y1.ctypes.data,
                                           y2.ctypes.data, M, U.ctypes.data, V.ctypes.data, float(eps),
                                           float(tol), int(maxit), ctypes.byref(rid)))
        self._shape[rid.value] = (N * M, N * M, (N, M))
        return rid.value

    def step(self):
        """One scheduling round; returns (pending, active, finished)."""
        a, b, c = _I32(), _I32(), _I32()
        _check(_lib.finom_server_step(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def result(self, rid):
        """(done dict, f, g) of a finished request, or None while it is pending.
        2D potentials come back as (N, M) arrays."""
        import numpy as np
        shp = self._shape.get(rid)
        if shp is None:
            raise KeyError(rid)
        f = np.empty(shp[0])
        g = np.empty(shp[1])
        d = FinomServerDone()
        rc = _lib.finom_server_result(self.handle, int(rid), ctypes.byref(d), f.ctypes.data, g.ctypes.data)
        if rc == FINOM_EPENDING:
            return None
        _check(rc)
        del self._shape[rid]
        out = {"id": d.id, "kind": d.kind, "status": d.status, "latency_s": d.latency_s, "queue_s": d.queue_s}
        out.update(d.result.as_dict())
        if len(shp) == 3:
            f = f.reshape(shp[2], order="F")
            g = g.reshape(shp[2], order="F")
        return out, f, g

    def set_policy(self, policy):
        """'fifo' (arrival order) or 'smallest' (smallest queued request first)."""
        _check(_lib.finom_server_set_policy(self.handle, {"fifo": 0, "smallest": 1}[policy]))

    def set_batching(self, max_points):
        """Batch 1D requests with N + M <= max_points (0: off)."""
        _check(_lib.finom_server_set_batching(self.handle, int(max_points)))

    def set_eps_scaling(self, stages, factor=0.5, tol_stage=1e-4):
        _check(_lib.finom_server_set_eps_scaling(self.handle, int(stages), float(factor), float(tol_stage)))

    def cancel(self, rid):
        _check(_lib.finom_server_cancel(self.handle, int(rid)))

    def run(self, ids):
        """Step until every request in ids has finished; returns {id: (done, f, g)}."""
        out = {}
        ids = list(ids)
        while len(out) < len(ids):
            self.step()
            for r in ids:
                if r not in out:
                    got = self.result(r)
                    if got is not None:
                        out[r] = got
        return out

    def close(self):
        if self.handle:
            _lib.finom_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
