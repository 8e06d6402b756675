"""Pins of the plain-C serial oracle against the dense definition and the paper's example."""
import json
import math
import os

import numpy as np
import pytest

from oracle import dense, serial_c

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _problem(seed, N, M, ties=False):
    g = np.random.default_rng(seed)
    x = np.sort(g.uniform(0, 1, N))
    y = np.sort(g.uniform(0, 1, M))
    if ties:
        x = np.sort(np.round(x * 37) / 37)
        y = np.sort(np.round(y * 37) / 37)
    u = g.uniform(0, 1, N); u /= u.sum()
    v = g.uniform(0, 1, M); v /= v.sum()
    return x, y, u, v


def test_worked_example_dividing_index():
    with open(os.path.join(GOLDEN, "worked_example.json")) as fh:
        ex = json.load(fh)
    assert serial_c.dividing_index(ex["x"], ex["y"]).tolist() == ex["zeta"]


@pytest.mark.parametrize("seed,ties", [(0, False), (1, True), (2, True)])
def test_log_apply_equals_dense(seed, ties):
    x, y, u, v = _problem(seed, 131, 97, ties)
    eps = 0.01
    b = np.random.default_rng(seed).normal(0, 0.02, len(y))
    b[3] = -np.inf
    got, c = serial_c.log_apply(x, y, eps, b, with_cost=True)
    C = dense.cost_1d(x, y)
    want = dense.log_apply_dense(C, np.zeros(len(x)), b, eps)
    np.testing.assert_allclose(got, want, atol=1e-12, rtol=0)
    # cost-weighted: log sum_j C_ij exp((b_j - C_ij)/eps)
    with np.errstate(divide="ignore"):
        Z = np.log(C) + (b[None, :] - C) / eps
    from scipy.special import logsumexp
    np.testing.assert_allclose(c, logsumexp(Z, axis=1), atol=1e-11, rtol=0)


def test_cost_and_marginal_error_equal_dense():
    x, y, u, v = _problem(5, 80, 64)
    eps = 0.02
    C = dense.cost_1d(x, y)
    res = dense.sinkhorn_log(C, u, v, eps, tol=0.0, maxit=12)
    assert serial_c.cost(x, y, eps, res.f, res.g) == pytest.approx(res.w1, rel=1e-12)
    assert serial_c.marginal_error(x, y, eps, res.f, res.g, v) == pytest.approx(res.err, rel=1e-10)


@pytest.mark.parametrize("maxit", [0, 1, 9])
def test_sinkhorn_lockstep_with_dense(maxit):
    x, y, u, v = _problem(7, 70, 90)
    u[[4, 11]] = 0.0; u /= u.sum()
    eps = 0.01
    C = dense.cost_1d(x, y)
    f, g, it, err = serial_c.sinkhorn(x, y, u, v, eps, 0.0, maxit)
    res = dense.sinkhorn_log(C, u, v, eps, tol=0.0, maxit=maxit)
    assert it == res.iters == maxit
    np.testing.assert_allclose(f, res.f, atol=1e-12)
    np.testing.assert_allclose(g, res.g, atol=1e-12)
    assert err == pytest.approx(res.err, rel=1e-9)


def test_sinkhorn_converged_equals_dense():
    x, y, u, v = _problem(8, 60, 50)
    eps = 0.03
    C = dense.cost_1d(x, y)
    f, g, it, err = serial_c.sinkhorn(x, y, u, v, eps, 1e-10, 100000)
    res = dense.sinkhorn_log(C, u, v, eps, tol=1e-10, maxit=100000)
    assert it == res.iters and err <= 1e-10
    assert serial_c.cost(x, y, eps, f, g) == pytest.approx(res.w1, rel=1e-11)


# ---------------------------------------------------------------- 2D (Sec. 3, Appendix A)

def _grid_problem(seed, N, M, zero=False):
    g = np.random.default_rng(seed)
    x1, x2 = np.sort(g.uniform(0, 1, N)), np.sort(g.uniform(0, 1, N))
    y1, y2 = np.sort(g.uniform(0, 1, M)), np.sort(g.uniform(0, 1, M))
    U = g.uniform(0.1, 1, (N, M))
    V = g.uniform(0.1, 1, (N, M))
    if zero:
        U[1, :] = 0.0           # a whole row of grid 1 without mass
        V[:, 2] = 0.0           # a whole column of grid 2 without mass
    return x1, y1, x2, y2, U / U.sum(), V / V.sum()


@pytest.mark.parametrize("seed,N,M", [(0, 9, 7), (1, 1, 6), (2, 8, 1)])
def test_2d_log_apply_equals_dense(seed, N, M):
    x1, y1, x2, y2, _, _ = _grid_problem(seed, N, M)
    eps = 0.03
    B = np.random.default_rng(seed).normal(0, 0.02, (N, M))
    B[0, 0] = -np.inf
    C = dense.cost_2d(x1, y1, x2, y2)
    want = dense.log_apply_dense(C, np.zeros(N * M), B.ravel(order="F"), eps)
    got = serial_c.log_apply2d(x1, y1, x2, y2, eps, B)
    np.testing.assert_allclose(got.ravel(order="F"), want, atol=1e-12, rtol=0)


def test_2d_cost_and_marginal_error_equal_dense():
    x1, y1, x2, y2, U, V = _grid_problem(3, 7, 6)
    eps = 0.04
    C = dense.cost_2d(x1, y1, x2, y2)
    res = dense.sinkhorn_log(C, U.ravel(order="F"), V.ravel(order="F"), eps, tol=0.0, maxit=7)
    A = res.f.reshape((7, 6), order="F")
    B = res.g.reshape((7, 6), order="F")
    assert serial_c.cost2d(x1, y1, x2, y2, eps, A, B) == pytest.approx(res.w1, rel=1e-12)
    assert serial_c.marginal_error2d(x1, y1, x2, y2, eps, A, B, V) == pytest.approx(res.err, rel=1e-10)


@pytest.mark.parametrize("zero", [False, True])
def test_2d_sinkhorn_lockstep_with_dense(zero):
    x1, y1, x2, y2, U, V = _grid_problem(4, 6, 5, zero)
    eps = 0.05
    C = dense.cost_2d(x1, y1, x2, y2)
    for maxit in (0, 1, 8):
        A, B, it, err = serial_c.sinkhorn2d(x1, y1, x2, y2, U, V, eps, 0.0, maxit)
        res = dense.sinkhorn_log(C, U.ravel(order="F"), V.ravel(order="F"), eps, tol=0.0, maxit=maxit)
        assert it == maxit
        np.testing.assert_allclose(A.ravel(order="F"), res.f, atol=1e-12)
        np.testing.assert_allclose(B.ravel(order="F"), res.g, atol=1e-12)
        assert err == pytest.approx(res.err, rel=1e-9, abs=1e-15)


def test_2d_sinkhorn_single_row_is_the_1d_solve():
    # M = 1: grid points (x_k, y1_0) vs (x_l, y2_0); the y offset is a constant
    # factor of K, so the plan and the potentials' sum match the 1D solve
    x1, y1, x2, y2, U, V = _grid_problem(5, 40, 1)
    eps = 0.02
    A, B, it2, err2 = serial_c.sinkhorn2d(x1, y1, x2, y2, U, V, eps, 1e-11, 100000)
    f, g, it1, err1 = serial_c.sinkhorn(x1, x2, U[:, 0], V[:, 0], eps, 1e-11, 100000)
    assert err2 <= 1e-11 and err1 <= 1e-11
    w2 = serial_c.cost2d(x1, y1, x2, y2, eps, A, B)
    w1 = serial_c.cost(x1, x2, eps, f, g)
    assert w2 == pytest.approx(w1 + abs(y1[0] - y2[0]), rel=1e-9)
