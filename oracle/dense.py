"""Dense FP64 CPU oracle for entropic Wasserstein-1 Sinkhorn (test infrastructure).

This module is test infrastructure, not product code.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and reference
legs) may import it; the CUDA library never calls into it and shares no code
with it.

Everything here is the plain definition, evaluated densely in float64:

* the L1 cost matrix of Sec. 1 (eq. ``w1Definition``) and of Sec. 3.1 for
  tensor-product meshes ordered column-major (eq. ``2d-block-entry``);
* the kernel ``K = exp(-C / eps)`` (Sec. 2.1) and its stabilised form
  ``diag(e^{a/eps}) K diag(e^{b/eps})`` (Remark ``log-domain-stabilization``);
* the Sinkhorn iteration of eq. ``iteration`` (psi first, then phi), started
  from ``phi = 1/N``, ``psi = 1/M`` and stopped at the loop head when the
  marginal error ``|| diag(psi) K^T phi - v ||_1`` is ``<= tol`` or the
  iteration count reaches ``maxit`` (Algorithm 1);
* the primal cost ``<C, Gamma>`` of the entropic plan.

The iteration is evaluated in the log domain with a max-shifted log-sum-exp,
which is the stabilisation of the Remark taken to its limit (absorb after
every half step).  ``sinkhorn_linear`` is the unstabilised linear-domain form
of eq. ``iteration``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import logsumexp

__all__ = [
    "cost_1d", "cost_2d", "kernel", "kv_dense", "ktu_dense", "log_apply_dense",
    "SinkhornResult", "sinkhorn_log", "sinkhorn_linear", "marginal_error",
    "transport_cost", "plan_from_potentials", "barycentric", "kron_2d", "cost_nd",
]


def _log(a):
    """Natural log with log(0) = -inf and no warning (zero masses)."""
    a = np.asarray(a, dtype=np.float64)
    out = np.full(a.shape, -np.inf)
    pos = a > 0
    out[pos] = np.log(a[pos])
    return out


def cost_1d(x, y):
    """C_ij = |x_i - y_j| (Sec. 1, eq. w1Definition, 1D L1 cost)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return np.abs(x[:, None] - y[None, :])


def cost_2d(x1, y1, x2, y2):
    """L1 cost between the grids x1 x y1 and x2 x y2 (Sec. 3.1).

    Grid points are numbered column-major: point (x1_k, y1_i) of the first
    mesh has index ``k + N*i`` and point (x2_l, y2_j) of the second has index
    ``l + N*j`` (N = len(x1) = len(x2)).  The entry is
    ``|x1_k - x2_l| + |y1_i - y2_j|`` (eq. 2d-block-entry).
    """
    x1 = np.asarray(x1, dtype=np.float64)
    x2 = np.asarray(x2, dtype=np.float64)
    y1 = np.asarray(y1, dtype=np.float64)
    y2 = np.asarray(y2, dtype=np.float64)
    N, M = len(x1), len(y1)
    assert len(x2) == N and len(y2) == M
    X1 = np.tile(x1, M)      # k runs fastest
    Y1 = np.repeat(y1, N)
    X2 = np.tile(x2, M)
    Y2 = np.repeat(y2, N)
    return np.abs(X1[:, None] - X2[None, :]) + np.abs(Y1[:, None] - Y2[None, :])


def grid_coords(axes):
    """Coordinates of the points of the tensor-product grid of the given axis
    node arrays, one row per axis, points numbered with axis 0 fastest
    (index i_0 + n_0 (i_1 + n_1 (i_2 + ...)))."""
    axes = [np.asarray(a, dtype=np.float64) for a in axes]
    n = [len(a) for a in axes]
    G = int(np.prod(n))
    idx = np.arange(G)
    out = np.empty((len(axes), G))
    inner = 1
    for k, a in enumerate(axes):
        out[k] = a[(idx // inner) % n[k]]
        inner *= n[k]
    return out


def cost_nd(xs, ys):
    """L1 cost between the d-dimensional tensor-product grids of the axes xs
    (first measure) and ys (second), sum_k |x^k - y^k| (the separable cost of
    Sec. 3, in d dimensions), points numbered with axis 0 fastest."""
    X, Y = grid_coords(xs), grid_coords(ys)
    C = np.zeros((X.shape[1], Y.shape[1]))
    for k in range(X.shape[0]):
        C += np.abs(X[k][:, None] - Y[k][None, :])
    return C


def kernel(C, eps):
    """K = exp(-C / eps) (Sec. 2.1)."""
    return np.exp(-np.asarray(C, dtype=np.float64) / eps)


def kv_dense(C, v, eps):
    """K v with K = exp(-C/eps), the dense O(NM) product (Sec. 2.3)."""
    return kernel(C, eps) @ np.asarray(v, dtype=np.float64)


def ktu_dense(C, u, eps):
    """K^T u, the dense O(NM) product (Sec. 2.3)."""
    return kernel(C, eps).T @ np.asarray(u, dtype=np.float64)


def log_apply_dense(C, a, b, eps):
    """log( diag(e^{a/eps}) K diag(e^{b/eps}) 1 ), computed by log-sum-exp.

    This is the stabilised kernel of Remark log-domain-stabilization applied
    to the all-ones vector: entry i is ``log sum_j exp((a_i + b_j - C_ij)/eps)``.
    ``a`` and ``b`` are in cost units (the paper's absorption vectors).
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    Z = (a[:, None] + b[None, :] - np.asarray(C, dtype=np.float64)) / eps
    return logsumexp(Z, axis=1)


def plan_from_potentials(C, f, g, eps):
    """Gamma_ij = exp((f_i + g_j - C_ij)/eps) = phi_i k_ij psi_j (Sec. 2.1),
    with f = eps log phi and g = eps log psi."""
    return np.exp((f[:, None] + g[None, :] - C) / eps)


def barycentric(C, f, g, eps, x, y):
    """Barycentric projections of the plan Gamma returned by Algorithm 1:
    the image of x_i is the Gamma-weighted mean of the y_j in row i,
    sum_j Gamma_ij y_j / sum_j Gamma_ij, and that of y_j the weighted mean of
    the x_i in column j.  Returns (tx [N], ty [M])."""
    G = plan_from_potentials(C, np.asarray(f, dtype=np.float64), np.asarray(g, dtype=np.float64), eps)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return G @ y / G.sum(axis=1), G.T @ x / G.sum(axis=0)


def _col_logsum(C, f, g, eps):
    """log of the column sums of Gamma: g_j/eps + LSE_i((f_i - C_ij)/eps)."""
    return g / eps + logsumexp((f[:, None] - C) / eps, axis=0)


def marginal_error(C, f, g, v, eps):
    """|| diag(psi) K^T phi - v ||_1 (Algorithm 1 loop head; Sec. 4).

    Summed in a compensated way (math.fsum)."""
    col = np.exp(_col_logsum(C, f, g, eps))
    return math.fsum(np.abs(col - np.asarray(v, dtype=np.float64)).tolist())


def transport_cost(C, f, g, eps):
    """<C, Gamma> for Gamma = diag(phi) K diag(psi) (eq. w1Definition objective
    evaluated at the entropic plan), summed with math.fsum."""
    G = plan_from_potentials(C, f, g, eps)
    return math.fsum((C * G).ravel().tolist())


@dataclass
class SinkhornResult:
    f: np.ndarray          # eps * log(phi), cost units (-inf where u_i = 0)
    g: np.ndarray          # eps * log(psi)
    iters: int             # completed iterations (the paper's l at loop exit)
    err: float             # marginal error of the returned (phi, psi)
    converged: bool        # err <= tol was the exit reason
    w1: float              # <C, Gamma>
    err_history: list      # marginal error at every loop head


def sinkhorn_log(C, u, v, eps, tol, maxit, record=False, f0=None, g0=None):
    """Dense log-domain Sinkhorn (eq. iteration, Algorithm 1 control flow).

    Start: phi = 1/N, psi = 1/M (Algorithm 1), i.e. f = eps log(1/N),
    g = eps log(1/M), unless warm-start potentials are given.
    Loop head: stop when ``l >= maxit`` or the marginal error is ``<= tol``.
    Body: psi <- v / (K^T phi), then phi <- u / (K psi), written as
    ``g_j = eps log v_j - eps LSE_i((f_i - C_ij)/eps)`` and
    ``f_i = eps log u_i - eps LSE_j((g_j - C_ij)/eps)``.
    """
    C = np.asarray(C, dtype=np.float64)
    N, M = C.shape
    logu = _log(u)
    logv = _log(v)
    f = np.full(N, eps * math.log(1.0 / N)) if f0 is None else np.array(f0, dtype=np.float64)
    g = np.full(M, eps * math.log(1.0 / M)) if g0 is None else np.array(g0, dtype=np.float64)
    hist = []
    it = 0
    while True:
        err = marginal_error(C, f, g, v, eps)
        if record:
            hist.append(err)
        if it >= maxit or err <= tol:
            break
        g = eps * logv - eps * logsumexp((f[:, None] - C) / eps, axis=0)
        f = eps * logu - eps * logsumexp((g[None, :] - C) / eps, axis=1)
        it += 1
    return SinkhornResult(f=f, g=g, iters=it, err=err, converged=bool(err <= tol),
                          w1=transport_cost(C, f, g, eps), err_history=hist)


def sinkhorn_linear(C, u, v, eps, tol, maxit):
    """Unstabilised Sinkhorn of eq. iteration in linear float64.

    phi = psi = 1/N start, psi <- v / (K^T phi), phi <- u / (K psi), marginal
    error at the loop head.  Returns (phi, psi, iters, err)."""
    K = kernel(C, eps)
    N, M = K.shape
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    phi = np.full(N, 1.0 / N)
    psi = np.full(M, 1.0 / M)
    it = 0
    while True:
        err = math.fsum(np.abs(psi * (K.T @ phi) - v).tolist())
        if it >= maxit or err <= tol:
            break
        psi = v / (K.T @ phi)
        phi = u / (K @ psi)
        it += 1
    return phi, psi, it, err


def kron_2d(Kx, Ky):
    """K = K_y (x) K_x (eq. 2d-kron), numpy's Kronecker product."""
    return np.kron(Ky, Kx)
