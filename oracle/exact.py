"""Exact (unregularised) and closed-form references for W1 (test infrastructure).

This module is test infrastructure, not product code.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` may import it.

* ``w1_lp``            -- the linear program of eq. ``w1Definition`` (Sec. 1)
  solved by scipy's HiGHS: min <C, Gamma> over Gamma >= 0 with
  Gamma 1 = u and Gamma^T 1 = v.
* ``w1_closed_form_1d`` -- in 1D the same optimum equals
  integral |F_mu(t) - F_nu(t)| dt (F = cumulative distribution functions),
  evaluated exactly on the merged support.
* ``entropic_2x2``     -- the entropic plan of eq. ``regularized problem`` for
  N = M = 2 in closed form: Gamma = diag(phi) K diag(psi) forces
  g11 g22 / (g12 g21) = k11 k22 / (k12 k21) =: kappa, and with the marginals
  this is a quadratic in g11.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["w1_lp", "w1_closed_form_1d", "entropic_2x2"]


def w1_lp(C, u, v):
    """Optimal value of min <C, G> s.t. G 1 = u, G^T 1 = v, G >= 0 (HiGHS)."""
    from scipy.optimize import linprog

    C = np.asarray(C, dtype=np.float64)
    N, M = C.shape
    A_eq = np.zeros((N + M, N * M))
    for i in range(N):
        A_eq[i, i * M:(i + 1) * M] = 1.0          # row sums
    for j in range(M):
        A_eq[N + j, j::M] = 1.0                    # column sums
    b_eq = np.concatenate([np.asarray(u, float), np.asarray(v, float)])
    res = linprog(C.ravel(), A_eq=A_eq, b_eq=b_eq, bounds=(0, None), method="highs")
    if not res.success:
        raise RuntimeError(res.message)
    return float(res.fun)


def w1_closed_form_1d(x, u, y, v):
    """integral over t of |F_mu(t) - F_nu(t)| for mu = sum u_i d_{x_i},
    nu = sum v_j d_{y_j} (u, v each summing to 1)."""
    pts = np.concatenate([np.asarray(x, float), np.asarray(y, float)])
    w = np.concatenate([np.asarray(u, float), -np.asarray(v, float)])
    order = np.argsort(pts, kind="mergesort")
    pts, w = pts[order], w[order]
    total = []
    F = 0.0
    for k in range(len(pts) - 1):
        F += w[k]
        total.append(abs(F) * (pts[k + 1] - pts[k]))
    return math.fsum(total)


def entropic_2x2(C, u, v, eps):
    """Closed-form entropic plan for 2 x 2 problems; returns (Gamma, <C,Gamma>)."""
    C = np.asarray(C, float)
    K = np.exp(-C / eps)
    kappa = K[0, 0] * K[1, 1] / (K[0, 1] * K[1, 0])
    u1, v1 = float(u[0]), float(v[0])
    lo, hi = max(0.0, u1 + v1 - 1.0), min(u1, v1)
    # (1-kappa) t^2 + (1 - u1 - v1 + kappa (u1 + v1)) t - kappa u1 v1 = 0
    a = 1.0 - kappa
    b = 1.0 - u1 - v1 + kappa * (u1 + v1)
    c = -kappa * u1 * v1
    if abs(a) < 1e-300:
        t = -c / b
    else:
        disc = math.sqrt(b * b - 4 * a * c)
        roots = [(-b + disc) / (2 * a), (-b - disc) / (2 * a)]
        cand = [t for t in roots if lo - 1e-15 <= t <= hi + 1e-15]
        t = cand[0]
    G = np.array([[t, u1 - t], [v1 - t, 1.0 - u1 - v1 + t]])
    return G, float((C * G).sum())
