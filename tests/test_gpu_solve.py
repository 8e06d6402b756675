"""GPU parity of the Sinkhorn loop (Algorithm 1) against the CPU oracle.

Lock-step: after the same number of iterations the GPU potentials equal the
oracle's (FP64 plans to ~1e-11 eps, FP32 log-domain plans to ~1e-5 eps).
Converged: W1 relative error <= 1e-4 (FP32) / 1e-9 (FP64), marginal error of
the returned potentials <= the tolerance (float64 check), same stopping
iteration (FP64) or nearly (FP32).
"""
import math

import numpy as np
import pytest

from oracle import dense, serial_c
from tests.gpu_util import H, T, meshes, relerr

pytestmark = pytest.mark.gpu


def _masses(N, M, seed, zeros=False):
    g = np.random.default_rng(seed)
    u = g.uniform(0, 1, N)
    v = g.uniform(0, 1, M)
    if zeros:
        u[g.random(N) < 0.05] = 0.0
        v[g.random(M) < 0.05] = 0.0
    return u / u.sum(), v / v.sum()


def _pos(f, m):
    return f[m > 0]


LOCK_TOL = {"f64": 1e-10, "f32_log": 2e-5}   # |f_gpu - f_oracle| / eps on points with mass
# Float32 log-domain iterates: the mantissa sums of the scans take 2^d from
# the float32 ex2 instruction, whose relative error is at most 2^-22.5
# (1.7e-7), and a term's path through the scan (its thread's run, the raking
# warp, the tile carries, the output point) crosses some 30 such factors.  A
# point's weight therefore carries a relative error of ~sqrt(30) x 1.7e-7
# ~ 1e-6 at most in practice.  With one point on a side that one weight sets
# the marginal error (F32_ERR_ONE); over many points the errors average out
# (a few 1e-9 measured at N = 500), and F32_ERR_ABS = 0.2 tol for tol = 1e-6
# bounds them, with 2e-4 of the error itself for the float32 check.
F32_ERR_REL, F32_ERR_ABS, F32_ERR_ONE = 2e-4, 2e-7, 1e-6


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("maxit", [1, 2, 7, 40])
@pytest.mark.parametrize("N,M,kind,eps", [(300, 257, "uniform_random", 0.01), (2500, 3100, "ties", 0.004),
                                          (1, 40, "uniform_random", 0.05), (64, 1, "uniform_random", 0.05)])
def test_lockstep_with_oracle(lib, prec, maxit, N, M, kind, eps):
    x, y = meshes(kind, N, M, N + M)
    u, v = _masses(N, M, N * M, zeros=True)
    p = lib.finom_plan(T(x), T(y), eps, prec)
    f, g, res = lib.finom_solve(p, T(u), T(v), 0.0, maxit)
    fo, go, it, err = serial_c.sinkhorn(x, y, u, v, eps, 0.0, maxit)
    if min(N, M) == 1:
        # one point on a side: the plan is exact after one iteration, and the
        # error may reach exactly 0 (<= tol = 0) at different iterations
        assert res["iters"] >= 1 and it >= 1
    else:
        assert res["iters"] == it == maxit
    assert np.max(np.abs(_pos(H(f), u) - _pos(fo, u))) / eps <= LOCK_TOL[prec]
    assert np.max(np.abs(_pos(H(g), v) - _pos(go, v))) / eps <= LOCK_TOL[prec]
    assert np.all(np.isneginf(H(f)[u == 0])) and np.all(np.isneginf(H(g)[v == 0]))
    # the float64 marginal error of the returned potentials against the
    # oracle's at the same iteration; float32 potentials add the noise above
    if prec == "f64":
        assert res["marginal_err"] == pytest.approx(err, rel=1e-6, abs=1e-12)
    else:
        floor = F32_ERR_ONE if min(N, M) == 1 else F32_ERR_ABS
        assert abs(res["marginal_err"] - err) <= F32_ERR_REL * err + floor


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_first_loop_head_check(lib, prec):
    """maxit = 0: nothing is updated; the check is made on phi = 1/N, psi = 1/M."""
    N, M, eps = 200, 150, 0.02
    x, y = meshes("uniform_random", N, M, 4)
    u, v = _masses(N, M, 4)
    p = lib.finom_plan(T(x), T(y), eps, prec)
    f, g, res = lib.finom_solve(p, T(u), T(v), 1e-6, 0)
    fo, go, it, err = serial_c.sinkhorn(x, y, u, v, eps, 1e-6, 0)
    assert res["iters"] == 0
    np.testing.assert_allclose(H(f), fo, rtol=1e-14)
    assert res["marginal_err_loop"] == pytest.approx(err, rel=1e-5)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32_log", 1e-6)])
@pytest.mark.parametrize("N,M,kind,eps", [(500, 500, "uniform_random", 0.02), (1800, 2300, "graded", 0.005),
                                          (1200, 1200, "chebyshev", 0.01)])
def test_converged_matches_oracle(lib, prec, tol, N, M, kind, eps):
    x, y = meshes(kind, N, M, 11 * N)
    u, v = _masses(N, M, 3 * M)
    p = lib.finom_plan(T(x), T(y), eps, prec)
    f, g, res = lib.finom_solve(p, T(u), T(v), tol, 200000)
    fo, go, it, err = serial_c.sinkhorn(x, y, u, v, eps, tol, 200000)
    w1o = serial_c.cost(x, y, eps, fo, go)
    assert res["converged"] == 1
    if prec == "f64":
        assert res["iters"] == it
        assert res["w1"] == pytest.approx(w1o, rel=1e-9)
    else:
        assert abs(res["iters"] - it) <= max(3, 0.02 * it)
        assert res["w1"] == pytest.approx(w1o, rel=1e-4)
        # the float32 loop's own check at its stop (the loop head of iteration
        # l) against the oracle's error at the same loop head: within 0.2 tol
        _, _, _, err_l = serial_c.sinkhorn(x, y, u, v, eps, 0.0, res["iters"])
        assert abs(res["marginal_err_loop"] - err_l) <= 0.2 * tol
    # float64 marginal error of the returned potentials, recomputed by the oracle
    e_or = serial_c.marginal_error(x, y, eps, H(f), H(g), v)
    assert e_or <= (tol if prec == "f64" else 3 * tol)
    assert res["marginal_err"] == pytest.approx(e_or, rel=1e-6, abs=1e-13)
    assert res["w1"] == pytest.approx(serial_c.cost(x, y, eps, H(f), H(g)), rel=1e-10)


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_config1_fp64_workload(lib, prec):
    """1D FP64 workload: N = M = 1000, eps = 1e-2, tol 1e-9, 2000 iterations."""
    from paper_2605_26659_gb300 import inputs
    pr = inputs.config1()
    p = lib.finom_plan(T(pr.x), T(pr.y), pr.eps, prec)
    f, g, res = lib.finom_solve(p, T(pr.u), T(pr.v), pr.tol, pr.maxit)
    C = dense.cost_1d(pr.x, pr.y)
    phi, psi, it, err = dense.sinkhorn_linear(C, pr.u, pr.v, pr.eps, pr.tol, pr.maxit)
    fo, go = pr.eps * np.log(phi), pr.eps * np.log(psi)
    assert res["iters"] == it
    w1o = dense.transport_cost(C, fo, go, pr.eps)
    if prec == "f64":
        assert res["w1"] == pytest.approx(w1o, rel=1e-10)
        assert res["marginal_err"] == pytest.approx(err, rel=1e-6)
        assert np.max(np.abs(H(f) - fo)) / pr.eps <= 1e-9
    else:
        assert res["w1"] == pytest.approx(w1o, rel=1e-4)
        assert abs(res["marginal_err"] - err) <= F32_ERR_REL * err + F32_ERR_ABS


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_mu_nu_symmetry(lib, prec):
    N, M, eps = 900, 700, 0.01
    x, y = meshes("uniform_random", N, M, 77)
    u, v = _masses(N, M, 78)
    p1 = lib.finom_plan(T(x), T(y), eps, prec)
    p2 = lib.finom_plan(T(y), T(x), eps, prec)
    _, _, r1 = lib.finom_solve(p1, T(u), T(v), 1e-7, 100000)
    _, _, r2 = lib.finom_solve(p2, T(v), T(u), 1e-7, 100000)
    assert r1["converged"] and r2["converged"]
    assert r1["w1"] == pytest.approx(r2["w1"], rel=1e-5)


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_warm_start_and_stepwise(lib, prec):
    N, M, eps = 1500, 1300, 0.005
    x, y = meshes("graded", N, M, 0)
    u, v = _masses(N, M, 1)
    p = lib.finom_plan(T(x), T(y), eps, prec)
    # 30 iterations stepwise == 30 iterations blocking
    lib.finom_solve_begin(p, T(u), T(v), 0.0, 30)
    lib.finom_solve_step(p, 100)
    done, it = lib.finom_solve_poll(p)
    assert done and it == 30
    f1, g1, r1 = lib.finom_solve_end(p)
    f2, g2, r2 = lib.finom_solve(p, T(u), T(v), 0.0, 30)
    assert np.array_equal(H(f1), H(f2)) and np.array_equal(H(g1), H(g2))
    # warm start from iteration 30 for 20 more == 50 from scratch
    f3, g3, r3 = lib.finom_solve(p, T(u), T(v), 0.0, 20, f=f2.clone(), g=g2.clone(), warm=True)
    fo, go, it, err = serial_c.sinkhorn(x, y, u, v, eps, 0.0, 50)
    assert np.max(np.abs(H(f3) - fo)) / eps <= 10 * LOCK_TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_invalid_masses(lib, prec):
    x, y = meshes("uniform_random", 50, 40, 2)
    p = lib.finom_plan(T(x), T(y), 0.05, prec)
    u, v = _masses(50, 40, 3)
    bad = u.copy(); bad[3] = -0.1
    with pytest.raises(lib.FinomError):
        lib.finom_solve(p, T(bad), T(v), 1e-6, 10)
    with pytest.raises(lib.FinomError):
        lib.finom_solve(p, T(np.zeros(50)), T(v), 1e-6, 10)
    # the plan stays usable after a rejected call
    f, g, res = lib.finom_solve(p, T(u), T(v), 1e-6, 10)
    assert res["iters"] == 10
