"""GPU parity of d-dimensional plans (finom_plan_nd) against the CPU oracle.

The products K v, K^T u and their stabilised log forms against the dense
definition on small 3D and 4D grids and against the axis-by-axis oracle on
grids whose lines span several tiles; Algorithm 2's loop in lock-step with the
oracle, converged solves (W1, float64 marginal error recomputed by the
oracle, iteration count), the d = 2 case against the 2D plan, and the float64
evaluation of W1 and the marginal error (finom_cost).

Acceptance as for 1D plans: products 1e-5 relative (float32 log-domain) and
1e-12 (float64); W1 1e-4 (float32) and 1e-9 (float64).
"""
import math

import numpy as np
import pytest

from oracle import dense, serial_c
from tests.gpu_util import H, T, relerr

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32_log": 1e-5}
LOCK = {"f64": 1e-10, "f32_log": 2e-5}


def _axes(n, seed, lo=0.0, hi=1.0):
    g = np.random.default_rng(seed)
    return [np.sort(g.uniform(lo, hi, k)) for k in n]


def _masses(G, seed, zeros=False):
    g = np.random.default_rng(seed)
    u, v = g.uniform(0.1, 1, G), g.uniform(0.1, 1, G)
    if zeros:
        u[g.random(G) < 0.05] = 0.0
        v[g.random(G) < 0.05] = 0.0
    return u / u.sum(), v / v.sum()


def _plan(lib, xs, ys, eps, prec):
    return lib.finom_plan_nd([T(x) for x in xs], [T(y) for y in ys], eps, prec)


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("n,eps", [((6, 5, 4), 0.05), ((3, 4, 2, 3), 0.1), ((9, 1, 7), 0.02)])
def test_products_small_dense(lib, prec, n, eps):
    xs, ys = _axes(n, sum(n)), _axes(n, 2 * sum(n))
    G = int(np.prod(n))
    p = _plan(lib, xs, ys, eps, prec)
    assert lib.finom_plan_axes(p) == list(n)
    C = dense.cost_nd(xs, ys)
    g = np.random.default_rng(G)
    v = g.uniform(0, 1, G)
    v[g.random(G) < 0.05] = 0.0
    u = g.uniform(0, 1, G)
    assert relerr(H(lib.finom_kv(p, T(v))), dense.kv_dense(C, v, eps)) <= TOL[prec]
    assert relerr(H(lib.finom_ktu(p, T(u))), dense.ktu_dense(C, u, eps)) <= TOL[prec]
    a = 0.3 * eps * g.normal(0, 1, G)
    b = np.where(v > 0, 0.3 * eps * g.normal(0, 1, G), -np.inf)
    got = H(lib.finom_kv_log(p, T(a), T(b)))
    assert np.max(np.abs(got - dense.log_apply_dense(C, a, b, eps))) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("n", [(1500, 3, 2), (2600, 2, 2)])
def test_products_multi_tile_lines(lib, prec, n):
    """Axis 0 has 1500 + 1500 merged nodes per line (two tiles of 2048: each
    tile forms its carry from the other's weights inside the pass) or
    2600 + 2600 (three tiles: carries from an aggregate launch), so lines carry
    state from tile to tile; checked against the axis-by-axis oracle."""
    xs, ys = _axes(n, 5), _axes(n, 6)
    eps = 0.004
    G = int(np.prod(n))
    p = _plan(lib, xs, ys, eps, prec)
    g = np.random.default_rng(7)
    b = eps * g.normal(0, 0.5, G)
    b[::13] = -np.inf
    a = np.zeros(G)
    got = H(lib.finom_kv_log(p, T(a), T(b)))
    want = serial_c.log_apply_nd(xs, ys, eps, b)
    fin = np.isfinite(want)
    assert np.array_equal(np.isneginf(got), ~fin)
    assert np.max(np.abs(got[fin] - want[fin])) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("maxit", [1, 4, 25])
def test_lockstep_with_oracle(lib, prec, maxit):
    n = (12, 9, 7)
    xs, ys = _axes(n, 11), _axes(n, 12)
    G = int(np.prod(n))
    u, v = _masses(G, 13, zeros=True)
    eps = 0.03
    p = _plan(lib, xs, ys, eps, prec)
    f, g, res = lib.finom_solve(p, T(u), T(v), 0.0, maxit)
    A, B, it, err = serial_c.sinkhorn_nd(xs, ys, u, v, eps, 0.0, maxit)
    assert res["iters"] == it == maxit
    mu, mv = u > 0, v > 0
    assert np.max(np.abs(H(f)[mu] - A[mu])) / eps <= LOCK[prec]
    assert np.max(np.abs(H(g)[mv] - B[mv])) / eps <= LOCK[prec]
    assert np.all(np.isneginf(H(f)[~mu])) and np.all(np.isneginf(H(g)[~mv]))
    if prec == "f64":
        assert res["marginal_err"] == pytest.approx(err, rel=1e-8)
    else:
        assert abs(res["marginal_err"] - err) <= 2e-4 * err + 2e-7


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("n", [(1100, 3), (2300, 2)])
def test_lockstep_two_and_three_tile_lines(lib, prec, n):
    """A 2D grid whose axis-0 lines span two tiles (1100 + 1100 merged nodes)
    or three (2300 + 2300): every pass of four iterations against the oracle."""
    xs, ys = _axes(n, 31), _axes(n, 32)
    G = int(np.prod(n))
    u, v = _masses(G, 33, zeros=True)
    eps = 0.01
    p = _plan(lib, xs, ys, eps, prec)
    f, g, res = lib.finom_solve(p, T(u), T(v), 0.0, 4)
    A, B, it, err = serial_c.sinkhorn_nd(xs, ys, u, v, eps, 0.0, 4)
    assert res["iters"] == it == 4
    mu, mv = u > 0, v > 0
    assert np.max(np.abs(H(f)[mu] - A[mu])) / eps <= LOCK[prec]
    assert np.max(np.abs(H(g)[mv] - B[mv])) / eps <= LOCK[prec]
    if prec == "f64":
        assert res["marginal_err"] == pytest.approx(err, rel=1e-8)
    else:
        assert abs(res["marginal_err"] - err) <= 2e-4 * err + 2e-7


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32_log", 1e-6)])
def test_converged_matches_oracle(lib, prec, tol):
    n = (10, 8, 6)
    xs, ys = _axes(n, 21), _axes(n, 22)
    G = int(np.prod(n))
    u, v = _masses(G, 23)
    eps = 0.05
    p = _plan(lib, xs, ys, eps, prec)
    f, g, res = lib.finom_solve(p, T(u), T(v), tol, 100000)
    A, B, it, err = serial_c.sinkhorn_nd(xs, ys, u, v, eps, tol, 100000)
    w1o = serial_c.cost_nd_potentials(xs, ys, eps, A, B)
    assert res["converged"] == 1
    if prec == "f64":
        assert res["iters"] == it
        assert res["w1"] == pytest.approx(w1o, rel=1e-9)
    else:
        assert abs(res["iters"] - it) <= max(3, 0.02 * it)
        assert res["w1"] == pytest.approx(w1o, rel=1e-4)
    e_or = serial_c.marginal_error_nd(xs, ys, eps, H(f), H(g), v)
    assert e_or <= tol
    assert res["marginal_err"] == pytest.approx(e_or, rel=1e-6, abs=1e-13)
    # finom_cost on the returned potentials: the same float64 evaluation
    w1c, errc = lib.finom_cost(p, T(u), T(v), f, g)
    assert w1c == pytest.approx(w1o, rel=1e-9 if prec == "f64" else 1e-4)
    assert errc == pytest.approx(e_or, rel=1e-6, abs=1e-13)


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_d2_equals_2d_plan(lib, prec):
    """d = 2 through finom_plan_nd against finom_plan_2d and the 2D oracle."""
    N, M, eps = 40, 30, 0.02
    xs, ys = _axes((N, M), 31), _axes((N, M), 32)
    U, V = _masses(N * M, 33)
    pn = _plan(lib, xs, ys, eps, prec)
    p2 = lib.finom_plan_2d(T(xs[0]), T(ys[0]), T(xs[1]), T(ys[1]), eps, prec)
    f1, g1, r1 = lib.finom_solve(pn, T(U), T(V), 0.0, 20)
    f2, g2, r2 = lib.finom_solve(p2, T(U), T(V), 0.0, 20)
    A, B, it, err = serial_c.sinkhorn2d(xs[0], xs[1], ys[0], ys[1], U.reshape(N, M, order="F"),
                                        V.reshape(N, M, order="F"), eps, 0.0, 20)
    assert r1["iters"] == r2["iters"] == it == 20
    assert np.max(np.abs(H(f1) - A.ravel(order="F"))) / eps <= LOCK[prec]
    assert np.max(np.abs(H(f1) - H(f2))) / eps <= 2 * LOCK[prec]
    assert r1["w1"] == pytest.approx(r2["w1"], rel=1e-9 if prec == "f64" else 1e-5)


def test_invalid_nd_arguments(lib):
    xs = _axes((4, 3), 1)
    with pytest.raises(lib.FinomError):
        lib.finom_plan_nd([T(x) for x in xs], [T(x) for x in xs], 0.0, "f32_log")
    bad = [T(np.array([0.3, 0.1, 0.2, 0.5])), T(xs[1])]
    with pytest.raises(lib.FinomError):
        lib.finom_plan_nd(bad, [T(x) for x in xs], 0.1, "f32_log")
    p1 = lib.finom_plan(T(xs[0]), T(xs[0]), 0.1, "f32_log")
    with pytest.raises(lib.FinomError) as e:
        lib.finom_plan_axes(p1)
    assert e.value.status == lib.FINOM_ENOTSUP
