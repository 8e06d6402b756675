"""Serial FINOM recurrences in float64 (test infrastructure).

This module is test infrastructure, not product code.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and reference
legs) may import it.  It shares no code with the CUDA library.

dense.py's plain N x M product is the oracle of record; this module restates
the paper's O(N + M) product from the splitting K = K_L + K_U of Sec. 2.2 -
2.3, with 0-based arrays, and is pinned to the dense definition and to the
worked example of Sec. 2.2:

* ``dividing_index``      -- Definition (dividing index), Sec. 2.2:
  zeta(i) = number of y_j with y_j <= x_i (so zeta(i) = 0 when x_i < y_1 and
  zeta(i) = M when x_i >= y_M); it splits row i of K into its lower block
  (columns j < zeta(i)) and its upper block (columns j >= zeta(i)).
* ``lower_representation`` / ``upper_representation`` -- the objects of the
  Theorems on the vector representations of K_L and K_U: the row ratios
  (eq. ``ratio``; 1 where the row is a structural zero) and the block-edge
  vectors eta_i, eta'_i, i.e. the entries a row gains over its neighbour.
* ``matvec_linear`` -- since each row of a block is its neighbour times the
  row ratio plus its block-edge entries, the block products are the running
  sums of two first-order linear recurrences, one scanned forward (K_L psi),
  one backward (K_U psi); their inflows are the block-edge dot products.  A
  generic scan (``_scan``) runs both; K psi is their sum.
* ``matvec_log`` -- the same two scans for the stabilised kernel of Remark
  ``log-domain-stabilization`` (row ratios and entries scaled by the
  absorption vectors), in log arithmetic (``_log_scan``).
* ``sinkhorn_log`` -- Algorithm 1's fixed-point iteration with that
  stabilisation applied after every half step, in log arithmetic.
* ``apply2d_log`` / ``sinkhorn2d_log`` -- Algorithm 2 with the stabilisation
  of Appendix A (eq. ``K'bpsi``): a column pass with a_x = 0, b_x = B(:, j)
  and a row pass with a_y = A(k, :), b_y = 0.

Ratios are taken in closed form, ``e^{-(x_{i+1}-x_i)/eps}``: in exact
arithmetic that is what the quotient of two kernel entries equals, and it
avoids the 0/0 that the quotient of two float64 underflows would give.
Pure-Python loops: for small inputs only (N, M up to a few thousand).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "dividing_index", "lower_representation", "upper_representation",
    "matvec_linear", "matvec_log", "sinkhorn_log", "apply2d_log",
    "sinkhorn2d_log", "logaddexp", "lse",
]

NEG_INF = -math.inf


def logaddexp(a, b):
    """log(e^a + e^b) with -inf handled."""
    if a == NEG_INF:
        return b
    if b == NEG_INF:
        return a
    m = max(a, b)
    return m + math.log1p(math.exp(-abs(a - b)))


def lse(vals):
    """log sum exp of a list (empty -> -inf)."""
    if len(vals) == 0:
        return NEG_INF
    m = max(vals)
    if m == NEG_INF:
        return NEG_INF
    return m + math.log(math.fsum(math.exp(t - m) for t in vals))


def dividing_index(x, y):
    """zeta(i) = #{j : y_j <= x_i} for sorted x, y (Definition, Sec. 2.2)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N, M = len(x), len(y)
    zeta = np.zeros(N, dtype=np.int64)
    j = 0
    for i in range(N):
        while j < M and y[j] <= x[i]:
            j += 1
        zeta[i] = j
    return zeta


def _kcheck(x, y, zeta, i, j, eps):
    """Entry of K_L: e^{-(x_i - y_j)/eps} for j < zeta(i) (0-based j), else 0."""
    return math.exp(-(x[i] - y[j]) / eps) if j < zeta[i] else 0.0


def _khat(x, y, zeta, i, j, eps):
    """Entry of K_U: e^{-(y_j - x_i)/eps} for j >= zeta(i) (0-based j), else 0."""
    return math.exp(-(y[j] - x[i]) / eps) if j >= zeta[i] else 0.0


def lower_representation(x, y, eps, zeta=None):
    """(r, eta) of Theorem (vector representation of K_L)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if zeta is None:
        zeta = dividing_index(x, y)
    N = len(x)
    r = []
    for i in range(N - 1):
        # denominator k~_{i,1} is a structural zero when row i of K_L is empty
        r.append(math.exp(-(x[i + 1] - x[i]) / eps) if zeta[i] >= 1 else 1.0)
    eta = []
    for i in range(N):
        lo = zeta[i - 1] if i >= 1 else 0
        eta.append([_kcheck(x, y, zeta, i, j, eps) for j in range(lo, zeta[i])])
    return r, eta


def upper_representation(x, y, eps, zeta=None):
    """(r', eta') of Theorem (vector representation of K_U)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if zeta is None:
        zeta = dividing_index(x, y)
    N, M = len(x), len(y)
    rp = []
    for i in range(N - 1):
        # denominator k^_{i+1,M} is a structural zero when row i+1 of K_U is empty
        rp.append(math.exp(-(x[i + 1] - x[i]) / eps) if zeta[i + 1] < M else 1.0)
    etap = []
    for i in range(N):
        hi = zeta[i + 1] if i + 1 < N else M
        etap.append([_khat(x, y, zeta, i, j, eps) for j in range(zeta[i], hi)])
    return rp, etap


def _scan(decay, inflow, backward=False):
    """Running sums of the first-order linear recurrence s_k = decay_k s_prev +
    inflow_k (s_prev = 0 before the first term), forward or backward; decay
    has one entry per step between neighbours (len(inflow) - 1)."""
    n = len(inflow)
    out = np.zeros(n)
    order = range(n - 1, -1, -1) if backward else range(n)
    prev = None
    for k in order:
        if prev is None:
            out[k] = inflow[k]
        else:
            out[k] = decay[min(k, prev)] * out[prev] + inflow[k]
        prev = k
    return out


def _log_scan(log_decay, log_inflow, backward=False):
    """``_scan`` in log arithmetic: s_k = log(e^{log_decay + s_prev} + e^{log_inflow_k})."""
    n = len(log_inflow)
    out = np.full(n, NEG_INF)
    order = range(n - 1, -1, -1) if backward else range(n)
    prev = None
    for k in order:
        carried = NEG_INF if prev is None or out[prev] == NEG_INF else log_decay[min(k, prev)] + out[prev]
        out[k] = logaddexp(carried, log_inflow[k])
        prev = k
    return out


def matvec_linear(x, y, eps, psi):
    """K psi = K_L psi + K_U psi, each block by a first-order recurrence
    (Sec. 2.3, eqs. decompose to p+q, p / q by dynamic programming).

    Row i of K_L is r_{i-1} times row i-1 plus its block-edge entries eta_i
    over the columns zeta(i-1) .. zeta(i)-1, so p = K_L psi is the forward
    scan with decays r and inflows eta_i . psi; K_U mirrors it (row i is
    r'_i times row i+1 plus eta'_i), a backward scan.  Returns (p+q, p, q)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    N, M = len(x), len(y)
    zeta = dividing_index(x, y)
    r, eta = lower_representation(x, y, eps, zeta)
    rp, etap = upper_representation(x, y, eps, zeta)
    # columns a row of a block gains over its neighbour
    lo_cols = [(zeta[i - 1] if i > 0 else 0, zeta[i]) for i in range(N)]
    up_cols = [(zeta[i], zeta[i + 1] if i + 1 < N else M) for i in range(N)]
    inflow_p = [math.fsum(a * b for a, b in zip(eta[i], psi[c0:c1])) for i, (c0, c1) in enumerate(lo_cols)]
    inflow_q = [math.fsum(a * b for a, b in zip(etap[i], psi[c0:c1])) for i, (c0, c1) in enumerate(up_cols)]
    p = _scan(r, inflow_p)
    q = _scan(rp, inflow_q, backward=True)
    return p + q, p, q


def matvec_log(x, y, eps, a, b):
    """log(K' 1) for K' = diag(e^{a/eps}) K diag(e^{b/eps}) (Remark
    log-domain-stabilization), by the two block scans in log arithmetic.

    Modified ratios: log r_i = (a_{i+1} - a_i)/eps + log r_i, and modified
    entries log k~'_ij = (a_i + b_j)/eps + log k~_ij (likewise for K_U).
    Returns (log(p+q), log p, log q)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    N, M = len(x), len(y)
    zeta = dividing_index(x, y)

    def log_kcheck(i, j):   # log of the absorbed lower-block entry
        return (a[i] + b[j] - (x[i] - y[j])) / eps

    def log_khat(i, j):     # log of the absorbed upper-block entry
        return (a[i] + b[j] - (y[j] - x[i])) / eps

    # block-edge inflows (log) and log row ratios of the absorbed blocks; a
    # ratio is 1 (log 0) where the row it divides by is a structural zero
    in_p = [lse([log_kcheck(i, j) for j in range(zeta[i - 1] if i > 0 else 0, zeta[i])]) for i in range(N)]
    in_q = [lse([log_khat(i, j) for j in range(zeta[i], zeta[i + 1] if i + 1 < N else M)]) for i in range(N)]
    lr = [(-(x[i + 1] - x[i]) / eps if zeta[i] >= 1 else 0.0) + (a[i + 1] - a[i]) / eps for i in range(N - 1)]
    lrp = [(-(x[i + 1] - x[i]) / eps if zeta[i + 1] < M else 0.0) + (a[i] - a[i + 1]) / eps for i in range(N - 1)]
    lp = _log_scan(lr, in_p)
    lq = _log_scan(lrp, in_q, backward=True)
    tot = np.array([logaddexp(lp[i], lq[i]) for i in range(N)])
    return tot, lp, lq


def _log(a):
    a = np.asarray(a, dtype=np.float64)
    out = np.full(a.shape, -np.inf)
    out[a > 0] = np.log(a[a > 0])
    return out


def sinkhorn_log(x, y, u, v, eps, tol, maxit):
    """Algorithm 1 with log-domain stabilisation absorbed after every half step.

    Absorption vectors a (x side) and b (y side) carry eps*log(phi) and
    eps*log(psi); after each absorption phi = psi = 1, so each half step is
    one stabilised product.  The product is evaluated with the column
    absorption only (row absorption zero) and the row factor e^{b/eps} is
    applied after, which is the same product and keeps zero masses (-inf
    potentials) out of the recurrence ratios.  Start: phi = 1/N, psi = 1/M.
    Loop head: marginal error || diag(psi) K^T phi - v ||_1 <= tol or l = maxit.
    Returns (a, b, iters, err)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N, M = len(x), len(y)
    logu, logv = _log(u), _log(v)
    a = np.full(N, eps * math.log(1.0 / N))
    b = np.full(M, eps * math.log(1.0 / M))
    zx, zy = np.zeros(N), np.zeros(M)
    it = 0
    while True:
        # log (K^T phi)_j: rows = y (transposed case), columns absorbed by a
        q, _, _ = matvec_log(y, x, eps, zy, a)
        err = math.fsum(abs(math.exp(bj / eps + t) - vj) for bj, t, vj in zip(b, q, v))
        if it >= maxit or err <= tol:
            break
        b = eps * (logv - q)               # psi = v / (K^T phi), absorbed
        qk, _, _ = matvec_log(x, y, eps, zx, b)
        a = eps * (logu - qk)              # phi = u / (K psi), absorbed
        it += 1
    return a, b, it, err


def apply2d_log(x1, y1, x2, y2, eps, A, B):
    """log(K' 1) on the first grid for K' = diag(e^{a/eps}) (K_y (x) K_x)
    diag(e^{b/eps}) (Appendix A, eq. K'bpsi), with a = vec(A), b = vec(B)
    (A, B of shape N x M, column-major grids).

    Column pass: log Q(:, j) = log(K_x e^{B(:, j)/eps}) -- the 1D stabilised
    product with a_x = 0, b_x = B(:, j).  Row pass: log P(k, :) =
    log(diag(e^{A(k,:)/eps}) K_y Q(k,:)^T) -- the 1D stabilised product with
    a_y = A(k, :), b_y = eps * log Q(k, :)."""
    N, M = len(x1), len(y1)
    logQ = np.empty((N, M))
    zeros_n = np.zeros(N)
    for j in range(M):
        logQ[:, j], _, _ = matvec_log(x1, x2, eps, zeros_n, B[:, j])
    logP = np.empty((N, M))
    for k in range(N):
        logP[k, :], _, _ = matvec_log(y1, y2, eps, A[k, :], eps * logQ[k, :])
    return logP


def sinkhorn2d_log(x1, y1, x2, y2, U, V, eps, tol, maxit):
    """Algorithm 2 with the Appendix A stabilisation (absorb every half step).

    U, V: N x M masses (column-major grids).  Start Phi = Psi = 1/(NM).
    Returns (A, B, iters, err) with A = eps log Phi, B = eps log Psi."""
    N, M = len(x1), len(y1)
    logU, logV = _log(U), _log(V)
    A = np.full((N, M), eps * math.log(1.0 / (N * M)))
    B = np.full((N, M), eps * math.log(1.0 / (N * M)))
    it = 0
    while True:
        # transposed product: grids swap roles
        lt = apply2d_log(x2, y2, x1, y1, eps, B, A)
        err = math.fsum(np.abs(np.exp(lt) - V).ravel().tolist())
        if it >= maxit or err <= tol:
            break
        B = B + eps * (logV - lt)
        lk = apply2d_log(x1, y1, x2, y2, eps, A, B)
        A = A + eps * (logU - lk)
        it += 1
    return A, B, it, err
