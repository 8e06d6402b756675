"""Solves warm-started through a decreasing sequence of eps
(finom_solve_eps_scaling) reach the same fixed point as the plain solve,
checked with the oracle's float64 error and cost of the returned
potentials, in fewer iterations."""
import numpy as np
import pytest

from oracle import serial_c
from tests.gpu_util import H, T

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32_log", 1e-6)])
def test_eps_scaling_1d(lib, prec, tol):
    from paper_2605_26659_gb300 import inputs
    pr = inputs.config2(1 << 12)
    p = lib.finom_plan(T(pr.x), T(pr.y), pr.eps, prec)
    f0, g0, r0 = lib.finom_solve(p, T(pr.u), T(pr.v), tol, 200000)
    f1, g1, r1 = lib.finom_solve_eps_scaling(p, T(pr.u), T(pr.v), tol, 200000, eps0=3e-2, factor=0.5, tol_stage=1e-4)
    assert r0["converged"] == r1["converged"] == 1
    assert r1["iters"] < r0["iters"]
    e1 = serial_c.marginal_error(pr.x, pr.y, pr.eps, H(f1), H(g1), pr.v)
    assert e1 <= (tol if prec == "f64" else 3 * tol)
    w0 = serial_c.cost(pr.x, pr.y, pr.eps, H(f0), H(g0))
    w1 = serial_c.cost(pr.x, pr.y, pr.eps, H(f1), H(g1))
    assert w1 == pytest.approx(w0, rel=1e-6 if prec == "f64" else 1e-4)
    assert r1["w1"] == pytest.approx(w1, rel=1e-9)


def test_eps_scaling_2d(lib):
    from paper_2605_26659_gb300 import inputs
    pr = inputs.config3(48, 40)
    U, V = pr.U.ravel(order="F"), pr.V.ravel(order="F")
    p = lib.finom_plan_2d(T(pr.x1), T(pr.x2), T(pr.y1), T(pr.y2), pr.eps, "f64")
    f0, g0, r0 = lib.finom_solve(p, T(U), T(V), 1e-8, 200000)
    f1, g1, r1 = lib.finom_solve_eps_scaling(p, T(U), T(V), 1e-8, 200000, eps0=2e-2, factor=0.5, tol_stage=1e-4)
    assert r0["converged"] == r1["converged"] == 1
    assert r1["w1"] == pytest.approx(r0["w1"], rel=1e-6)
    A = H(f1).reshape((48, 40), order="F")
    B = H(g1).reshape((48, 40), order="F")
    assert serial_c.marginal_error2d(pr.x1, pr.y1, pr.x2, pr.y2, pr.eps, A, B, pr.V) <= 1e-8


def test_eps_scaling_argument_errors(lib):
    from paper_2605_26659_gb300 import inputs
    pr = inputs.config2(256)
    p = lib.finom_plan(T(pr.x), T(pr.y), pr.eps, "f32_log")
    for kw in (dict(eps0=pr.eps / 2), dict(eps0=1e-2, factor=1.5), dict(eps0=1e-2, factor=0.0)):
        args = dict(eps0=1e-2, factor=0.5, tol_stage=1e-4)
        args.update(kw)
        with pytest.raises(lib.FinomError) as e:
            lib.finom_solve_eps_scaling(p, T(pr.u), T(pr.v), 1e-6, 1000, **args)
        assert e.value.status == lib.FINOM_EINVAL


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_time_to_error_trace(lib, prec):
    """The traced loop-head errors are the oracle's at the same iterations (to
    the precision of the loop's own check: its S - 1 uses a truncated series
    near S = 1, ~1e-9 relative in float64), and the GPU times increase."""
    from paper_2605_26659_gb300 import inputs
    pr = inputs.chebyshev(2000)
    p = lib.finom_plan(T(pr.x), T(pr.y), pr.eps, prec)
    its, err, ms = lib.finom_solve_trace(p, T(pr.u), T(pr.v), 200, every=25)
    assert list(its) == [25, 50, 75, 100, 125, 150, 175, 199]
    assert np.all(np.diff(ms) > 0)
    for l, e in zip(its, err):
        _, _, it, eo = serial_c.sinkhorn(pr.x, pr.y, pr.u, pr.v, pr.eps, 0.0, int(l))
        # float32: the loop's own check in float32 (mantissa sums of the scans,
        # ~2e-4 relative) plus the float32 iterate's noise (ex2 relative error
        # 2^-22.5, at most ~1.2e-7 of marginal error)
        assert e == pytest.approx(eo, rel=1e-7 if prec == "f64" else 2e-4, abs=1e-13 if prec == "f64" else 2e-7)
