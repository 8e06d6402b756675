"""Pins of the d-dimensional oracle (CPU only).

The dense cost of d-dimensional tensor-product grids and the axis-by-axis
products and Sinkhorn loop of ``oracle.serial_c`` are checked against things
fixed independently of them: the 1D and 2D cost definitions (d = 1, 2), the
Kronecker structure of the kernel (numpy.kron of the axis kernels), the dense
log-sum-exp product and dense Sinkhorn on the full cost matrix, the 2D serial
C oracle, brute-force LP optima as eps -> 0, and the marginal constraints.
"""
import math

import numpy as np
import pytest

from oracle import dense, exact, serial_c


def _axes(n, seed, lo=0.0, hi=1.0):
    g = np.random.default_rng(seed)
    return [np.sort(g.uniform(lo, hi, k)) for k in n]


def _masses(G, seed):
    g = np.random.default_rng(seed)
    u, v = g.uniform(0.1, 1, G), g.uniform(0.1, 1, G)
    return u / u.sum(), v / v.sum()


def test_cost_nd_reduces_to_1d_and_2d():
    xs, ys = _axes((7,), 1), _axes((7,), 2)
    assert np.array_equal(dense.cost_nd(xs, ys), dense.cost_1d(xs[0], ys[0]))
    xs, ys = _axes((5, 4), 3), _axes((5, 4), 4)
    np.testing.assert_array_equal(dense.cost_nd(xs, ys), dense.cost_2d(xs[0], xs[1], ys[0], ys[1]))


def test_cost_nd_entry_by_entry():
    xs, ys = _axes((3, 2, 4), 5), _axes((3, 2, 4), 6)
    C = dense.cost_nd(xs, ys)
    for i in range(24):
        a = (i % 3, (i // 3) % 2, i // 6)
        for j in range(24):
            b = (j % 3, (j // 3) % 2, j // 6)
            want = sum(abs(xs[k][a[k]] - ys[k][b[k]]) for k in range(3))
            assert C[i, j] == pytest.approx(want, abs=1e-15)


def test_kernel_is_kronecker_of_axis_kernels():
    """K = K_3 (x) K_2 (x) K_1 for points numbered with axis 0 fastest."""
    xs, ys = _axes((3, 4, 2), 7), _axes((3, 4, 2), 8)
    eps = 0.3
    K = dense.kernel(dense.cost_nd(xs, ys), eps)
    Ks = [dense.kernel(dense.cost_1d(x, y), eps) for x, y in zip(xs, ys)]
    np.testing.assert_allclose(K, np.kron(Ks[2], np.kron(Ks[1], Ks[0])), rtol=1e-13)


@pytest.mark.parametrize("n", [(4, 3, 5), (6, 1, 3), (2, 2, 2, 3)])
def test_axis_by_axis_product_equals_dense(n):
    xs, ys = _axes(n, 10), _axes(n, 11)
    eps = 0.07
    G = int(np.prod(n))
    B = np.random.default_rng(12).normal(0, 0.05, G)
    B[::7] = -np.inf
    got = serial_c.log_apply_nd(xs, ys, eps, B)
    want = dense.log_apply_dense(dense.cost_nd(xs, ys), np.zeros(G), B, eps)
    assert np.max(np.abs(got - want)) <= 1e-12


def test_sinkhorn_nd_lockstep_with_dense():
    n = (4, 3, 3)
    xs, ys = _axes(n, 20), _axes(n, 21)
    G = int(np.prod(n))
    u, v = _masses(G, 22)
    eps = 0.05
    C = dense.cost_nd(xs, ys)
    for maxit in (1, 5, 30):
        A, B, it, err = serial_c.sinkhorn_nd(xs, ys, u, v, eps, 0.0, maxit)
        r = dense.sinkhorn_log(C, u, v, eps, 0.0, maxit, f0=np.full(G, eps * math.log(1 / G)),
                               g0=np.full(G, eps * math.log(1 / G)))
        assert it == r.iters == maxit
        assert np.max(np.abs(A - r.f)) / eps <= 1e-11 and np.max(np.abs(B - r.g)) / eps <= 1e-11
        assert err == pytest.approx(r.err, rel=1e-9)
        assert serial_c.cost_nd_potentials(xs, ys, eps, A, B) == pytest.approx(
            dense.transport_cost(C, A, B, eps), rel=1e-11)


def test_sinkhorn_nd_d2_equals_2d_oracle():
    n = (5, 4)
    xs, ys = _axes(n, 30), _axes(n, 31)
    U, V = _masses(20, 32)
    eps = 0.04
    A, B, it, err = serial_c.sinkhorn_nd(xs, ys, U, V, eps, 0.0, 12)
    A2, B2, it2, err2 = serial_c.sinkhorn2d(xs[0], xs[1], ys[0], ys[1], U.reshape(5, 4, order="F"),
                                            V.reshape(5, 4, order="F"), eps, 0.0, 12)
    assert it == it2
    assert np.max(np.abs(A - A2.ravel(order="F"))) / eps <= 1e-11
    assert err == pytest.approx(err2, rel=1e-9)


def test_sinkhorn_nd_marginals_and_lp_limit():
    """Converged 3D solves: both marginals within tol, and <C, Gamma_eps>
    approaches the LP optimum from above within eps log(G^2) as eps -> 0."""
    n = (2, 2, 2)
    xs, ys = _axes(n, 40), _axes(n, 41)
    u, v = _masses(8, 42)
    C = dense.cost_nd(xs, ys)
    w_lp = exact.w1_lp(C, u, v)
    prev = None
    for eps in (0.1, 0.03, 0.01):
        A, B, it, err = serial_c.sinkhorn_nd(xs, ys, u, v, eps, 1e-12, 200000)
        assert err <= 1e-12
        P = dense.plan_from_potentials(C, A, B, eps)
        assert np.max(np.abs(P.sum(axis=1) - u)) <= 1e-10
        w = serial_c.cost_nd_potentials(xs, ys, eps, A, B)
        assert -1e-12 <= w - w_lp <= eps * math.log(64) + 1e-12
        if prev is not None:
            assert w <= prev + 1e-12
        prev = w
