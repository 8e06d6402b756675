"""ctypes loader of the plain-C serial FINOM oracle (test infrastructure).

Compiles ``oracle/finom_serial.c`` with gcc (``-O2 -fPIC -shared``, IEEE
semantics kept) into ``oracle/_build/libfinomref.so`` on first use.  Only
``tests/``, ``__graft_entry__`` and ``bench.py`` may import this module.
"""
from __future__ import annotations

import ctypes
import math
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "finom_serial.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfinomref.so")

_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the serial oracle")
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run([cc, "-O2", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        I64, D = ctypes.c_int64, ctypes.c_double
        L.finom_ref_dividing_index.argtypes = [_dp, I64, _dp, I64, _ip]
        L.finom_ref_dividing_index.restype = None
        L.finom_ref_log_apply.argtypes = [_dp, I64, _dp, I64, D, _dp, _dp, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]
        L.finom_ref_log_apply.restype = None
        L.finom_ref_marginal_error.argtypes = [_dp, I64, _dp, I64, D, _dp, _dp, _dp]
        L.finom_ref_marginal_error.restype = D
        L.finom_ref_cost.argtypes = [_dp, I64, _dp, I64, D, _dp, _dp]
        L.finom_ref_cost.restype = D
        L.finom_ref_sinkhorn.argtypes = [_dp, I64, _dp, I64, _dp, _dp, D, D, I64, ctypes.c_int,
                                         _dp, _dp, ctypes.POINTER(D)]
        L.finom_ref_sinkhorn.restype = I64
        L.finom_ref_log_apply2d.argtypes = [_dp, _dp, _dp, _dp, I64, I64, D, _dp, _dp]
        L.finom_ref_log_apply2d.restype = None
        L.finom_ref_marginal_error2d.argtypes = [_dp, _dp, _dp, _dp, I64, I64, D, _dp, _dp, _dp]
        L.finom_ref_marginal_error2d.restype = D
        L.finom_ref_cost2d.argtypes = [_dp, _dp, _dp, _dp, I64, I64, D, _dp, _dp]
        L.finom_ref_cost2d.restype = D
        L.finom_ref_sinkhorn2d.argtypes = [_dp, _dp, _dp, _dp, I64, I64, _dp, _dp, D, D, I64,
                                           ctypes.c_int, _dp, _dp, ctypes.POINTER(D)]
        L.finom_ref_sinkhorn2d.restype = I64
        _lib = L
    return _lib


def _a(v):
    return np.ascontiguousarray(v, dtype=np.float64)


def dividing_index(x, y):
    x, y = _a(x), _a(y)
    z = np.zeros(len(x), dtype=np.int64)
    lib().finom_ref_dividing_index(x, len(x), y, len(y), z)
    return z


def log_apply(x, y, eps, b, with_cost=False):
    """log sum_j exp((b_j - |x_i - y_j|)/eps) per row i (and the cost-weighted version)."""
    x, y, b = _a(x), _a(y), _a(b)
    out = np.empty(len(x))
    cost = np.empty(len(x)) if with_cost else None
    lib().finom_ref_log_apply(x, len(x), y, len(y), float(eps), b, out, None, None,
                              cost.ctypes.data if with_cost else None)
    return (out, cost) if with_cost else out


def marginal_error(x, y, eps, f, g, v):
    x, y = _a(x), _a(y)
    return lib().finom_ref_marginal_error(x, len(x), y, len(y), float(eps), _a(f), _a(g), _a(v))


def cost(x, y, eps, f, g):
    x, y = _a(x), _a(y)
    return lib().finom_ref_cost(x, len(x), y, len(y), float(eps), _a(f), _a(g))


def sinkhorn(x, y, u, v, eps, tol, maxit, f0=None, g0=None):
    """Algorithm 1 (absorbed log arithmetic); returns (f, g, iters, err)."""
    x, y, u, v = _a(x), _a(y), _a(u), _a(v)
    warm = f0 is not None and g0 is not None
    f = _a(f0).copy() if warm else np.empty(len(x))
    g = _a(g0).copy() if warm else np.empty(len(y))
    err = ctypes.c_double()
    it = lib().finom_ref_sinkhorn(x, len(x), y, len(y), u, v, float(eps), float(tol), int(maxit),
                                  1 if warm else 0, f, g, ctypes.byref(err))
    return f, g, int(it), err.value


# ------------------------------------------------------------------ 2D
# Grid arrays are numpy (N, M) arrays G[k, i] (point (x_k, y_i)); the C side
# takes them column-major (k + N i), i.e. G.ravel(order="F").

def _g(G):
    return np.ascontiguousarray(np.asarray(G, dtype=np.float64).ravel(order="F"))


def _grid(flat, N, M):
    return flat.reshape((N, M), order="F")


def log_apply2d(x1, y1, x2, y2, eps, B):
    """log sum_{l,j} exp((B[l,j] - |x1_k - x2_l| - |y1_i - y2_j|)/eps) on grid 1 (N x M)."""
    x1, y1, x2, y2 = _a(x1), _a(y1), _a(x2), _a(y2)
    N, M = len(x1), len(y1)
    out = np.empty(N * M)
    lib().finom_ref_log_apply2d(x1, y1, x2, y2, N, M, float(eps), _g(B), out)
    return _grid(out, N, M)


def marginal_error2d(x1, y1, x2, y2, eps, A, B, V):
    x1, y1, x2, y2 = _a(x1), _a(y1), _a(x2), _a(y2)
    return lib().finom_ref_marginal_error2d(x1, y1, x2, y2, len(x1), len(y1), float(eps), _g(A),
                                            _g(B), _g(V))


def cost2d(x1, y1, x2, y2, eps, A, B):
    x1, y1, x2, y2 = _a(x1), _a(y1), _a(x2), _a(y2)
    return lib().finom_ref_cost2d(x1, y1, x2, y2, len(x1), len(y1), float(eps), _g(A), _g(B))


def sinkhorn2d(x1, y1, x2, y2, U, V, eps, tol, maxit, A0=None, B0=None):
    """Algorithm 2 (absorbed log arithmetic); returns (A, B, iters, err), A, B as (N, M)."""
    x1, y1, x2, y2 = _a(x1), _a(y1), _a(x2), _a(y2)
    N, M = len(x1), len(y1)
    warm = A0 is not None and B0 is not None
    A = _g(A0).copy() if warm else np.empty(N * M)
    B = _g(B0).copy() if warm else np.empty(N * M)
    err = ctypes.c_double()
    it = lib().finom_ref_sinkhorn2d(x1, y1, x2, y2, N, M, _g(U), _g(V), float(eps), float(tol),
                                    int(maxit), 1 if warm else 0, A, B, ctypes.byref(err))
    return _grid(A, N, M), _grid(B, N, M), int(it), err.value


# ------------------------------------------------------------------ d-D
# Grids of the d-dimensional tensor-product case are flat float64 arrays
# with axis 0 fastest.  A product with K = K_d (x) ... (x) K_1 is one pass of
# 1D stabilised products per axis (log_apply along every line), the
# separable form of Sec. 3 taken to d axes.

def _lines(n, k):
    """Flat grid indices of every line along axis k (one row per line)."""
    n = list(n)
    G = int(np.prod(n))
    inner = int(np.prod(n[:k])) if k else 1
    nk = n[k]
    nl = G // nk
    l = np.arange(nl)
    base = (l % inner) + (l // inner) * inner * nk
    return base[:, None] + inner * np.arange(nk)[None, :]


def log_apply_nd(xs, ys, eps, B):
    """log sum_j exp((B_j - sum_k |x^k_{i_k} - y^k_{j_k}|)/eps) on the first
    grid for log-weights B (cost units) on the second, axis by axis."""
    xs = [_a(a) for a in xs]
    ys = [_a(a) for a in ys]
    n = [len(a) for a in xs]
    W = _a(B).copy()
    for k in range(len(n)):
        rows = _lines(n, k)
        out = np.empty_like(W)
        for r in rows:
            out[r] = eps * log_apply(xs[k], ys[k], eps, W[r])
        W = out
    return W / eps


def sinkhorn_nd(xs, ys, U, V, eps, tol, maxit, A0=None, B0=None):
    """Algorithm 2 on d-dimensional grids (absorbed log arithmetic, psi
    first, loop-head check || diag(psi) K^T phi - v ||_1 <= tol or maxit);
    start Phi = Psi = 1 / prod(n).  Returns (A, B, iters, err), flat."""
    U, V = _a(U), _a(V)
    G = len(U)
    warm = A0 is not None and B0 is not None
    A = _a(A0).copy() if warm else np.full(G, eps * math.log(1.0 / G))
    B = _a(B0).copy() if warm else np.full(G, eps * math.log(1.0 / G))
    it = 0
    while True:
        lt = log_apply_nd(ys, xs, eps, A)   # log K^T phi on the second grid
        e = math.fsum(np.abs(np.exp(B / eps + lt) - V).tolist())
        if it >= maxit or e <= tol:
            break
        with np.errstate(divide="ignore"):
            B = np.where(V > 0, eps * (np.log(np.where(V > 0, V, 1.0)) - lt), -np.inf)
        lt = log_apply_nd(xs, ys, eps, B)
        with np.errstate(divide="ignore"):
            A = np.where(U > 0, eps * (np.log(np.where(U > 0, U, 1.0)) - lt), -np.inf)
        it += 1
    return A, B, it, e


def cost_nd_potentials(xs, ys, eps, A, B):
    """<C, Gamma> for Gamma = exp((A_i + B_j - C_ij)/eps), axis by axis: for
    every axis k the sum over the plan of |x^k - y^k|, from 1D products with
    the cost-weighted kernel on axis k (log_apply's cost output)."""
    xs = [_a(a) for a in xs]
    ys = [_a(a) for a in ys]
    n = [len(a) for a in xs]
    A, B = _a(A), _a(B)
    total = 0.0
    for k in range(len(n)):
        W = B.copy()
        for j in range(len(n)):
            rows = _lines(n, j)
            out = np.empty_like(W)
            for r in rows:
                lo, c = log_apply(xs[j], ys[j], eps, W[r], with_cost=True)
                out[r] = eps * (c if j == k else lo)
            W = out
        with np.errstate(invalid="ignore"):
            t = np.where(np.isfinite(A) & np.isfinite(W), np.exp((A + W) / eps), 0.0)
        total += math.fsum(t.tolist())
    return total


def marginal_error_nd(xs, ys, eps, A, B, V):
    lt = log_apply_nd(ys, xs, eps, A)
    return math.fsum(np.abs(np.exp(_a(B) / eps + lt) - _a(V)).tolist())
