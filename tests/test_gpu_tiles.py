"""The half-step kernel with every tile kind (points per thread E in
{1, 2, 4, 8} on 256 threads, and E = -1: 64-point tiles on 64 threads) on 1D
plans: products and solves against the CPU oracle, the tile counts,
agreement across kinds, and the autotuner.

Small problems run with small tiles by default (the tuning table), so the
other GPU tests cover E < 8 too; here every E runs on the same inputs, with
problems that span many tiles of the smallest size and end in a ragged tile.
"""
import math

import numpy as np
import pytest

from oracle import dense, serial_c
from tests.gpu_util import H, T, meshes, relerr

pytestmark = pytest.mark.gpu

ELEMS = [-1, 1, 2, 4, 8]
POINTS = {-1: 64, 1: 256, 2: 512, 4: 1024, 8: 2048}   # merged points per tile
TOL = {"f64": 1e-12, "f32_log": 1e-5}


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("E", ELEMS)
@pytest.mark.parametrize("N,M,kind", [(3000, 2500, "uniform_random"), (777, 5003, "graded"),
                                      (2049, 2047, "ties"), (1, 300, "uniform_random")])
def test_products_every_tile_size(lib, prec, E, N, M, kind):
    x, y = meshes(kind, N, M, 11 * N + M)
    eps = 0.01
    p = lib.finom_plan(T(x), T(y), eps, prec)
    lib.finom_plan_set_elems(p, E)
    e, tiles = lib.finom_plan_elems(p)
    assert e == E and tiles == math.ceil((N + M) / POINTS[E])
    g = np.random.default_rng(N + M)
    v = g.uniform(0, 1, M)
    v[g.random(M) < 0.05] = 0.0
    u = g.uniform(0, 1, N)
    C = dense.cost_1d(x, y)
    tol = TOL[prec]
    assert relerr(H(lib.finom_kv(p, T(v))), dense.kv_dense(C, v, eps)) <= tol
    assert relerr(H(lib.finom_ktu(p, T(u))), dense.ktu_dense(C, u, eps)) <= tol
    a = 0.3 * eps * np.sin(7 * x)
    b = np.where(v > 0, 0.3 * eps * np.cos(5 * y), -np.inf)
    got = H(lib.finom_kv_log(p, T(a), T(b)))
    want = dense.log_apply_dense(C, a, b, eps)
    assert np.max(np.abs(got - want)) <= tol


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("E", ELEMS)
def test_solve_every_tile_size(lib, prec, E):
    from paper_2605_26659_gb300 import inputs
    pr = inputs.config1()
    p = lib.finom_plan(T(pr.x), T(pr.y), pr.eps, prec)
    lib.finom_plan_set_elems(p, E)
    f, g, res = lib.finom_solve(p, T(pr.u), T(pr.v), 0.0, 25)
    fo, go, it, err = serial_c.sinkhorn(pr.x, pr.y, pr.u, pr.v, pr.eps, 0.0, 25)
    assert res["iters"] == it == 25
    lock = 1e-10 if prec == "f64" else 2e-5
    assert np.max(np.abs(H(f) - fo)) / pr.eps <= lock and np.max(np.abs(H(g) - go)) / pr.eps <= lock
    # a problem that converges in ~900 iterations (eps = 0.03)
    x, y = meshes("uniform_random", 1500, 1300, 4)
    gg = np.random.default_rng(2)
    u, v = gg.uniform(0.1, 1, 1500), gg.uniform(0.1, 1, 1300)
    u, v = u / u.sum(), v / v.sum()
    p = lib.finom_plan(T(x), T(y), 0.03, prec)
    lib.finom_plan_set_elems(p, E)
    tol = 1e-9 if prec == "f64" else 1e-6
    f, g, res = lib.finom_solve(p, T(u), T(v), tol, 100000)
    fo, go, it, err = serial_c.sinkhorn(x, y, u, v, 0.03, tol, 100000)
    assert res["converged"] == 1
    assert res["w1"] == pytest.approx(serial_c.cost(x, y, 0.03, fo, go), rel=1e-9 if prec == "f64" else 1e-4)
    if prec == "f64":
        assert res["iters"] == it


def test_tile_sizes_agree_fp64(lib):
    x, y = meshes("graded", 6000, 5000, 5)
    g = np.random.default_rng(1)
    u, v = g.uniform(0.1, 1, 6000), g.uniform(0.1, 1, 5000)
    outs = []
    for E in ELEMS:
        p = lib.finom_plan(T(x), T(y), 0.005, "f64")
        lib.finom_plan_set_elems(p, E)
        f, gg, res = lib.finom_solve(p, T(u), T(v), 0.0, 40)
        outs.append((H(f), H(gg), res["w1"]))
    for f, gg, w1 in outs[1:]:
        assert np.max(np.abs(f - outs[0][0])) <= 1e-13 and np.max(np.abs(gg - outs[0][1])) <= 1e-13
        assert w1 == pytest.approx(outs[0][2], rel=1e-13)


def test_set_elems_refuses_other_plans(lib):
    x, y = meshes("uniform_random", 100, 90, 2)
    p = lib.finom_plan(T(x), T(y), 0.01, "f32_log")
    with pytest.raises(lib.FinomError) as e:
        lib.finom_plan_set_elems(p, 3)
    assert e.value.status == lib.FINOM_EINVAL
    p2 = lib.finom_plan_2d(T(x), T(x), T(y), T(y), 0.01, "f32_log")
    with pytest.raises(lib.FinomError) as e:
        lib.finom_plan_set_elems(p2, 2)
    assert e.value.status == lib.FINOM_ENOTSUP


def test_autotune_installs_the_fastest(lib):
    old = lib.finom_tune_get("f32_log", 12)
    best, times = lib.finom_autotune("f32_log", 12, iters=32)
    assert best in ELEMS and set(times) == set(ELEMS)
    assert all(t > 0 for t in times.values()) and times[best] == min(times.values())
    assert lib.finom_tune_get("f32_log", 12) == best
    x, y = meshes("uniform_random", 1500, 1400, 3)   # 2900 merged points: bucket 12
    p = lib.finom_plan(T(x), T(y), 0.01, "f32_log")
    assert lib.finom_plan_elems(p)[0] == best
    lib.finom_tune_set("f32_log", 12, old)


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_launch_tail_paths_agree(lib, prec):
    """The last CTA of a launch scans the tile aggregates into carries in
    chunks of E x (threads) tiles: N + M = 200,000 points give 98 tiles with
    E = 8 (one chunk), 196 with E = 4, 391 with E = 2, 782 with E = 1 and
    3125 64-point tiles (49 chunks), so one and several chunks run on the same
    problem; a 30-iteration solve must agree across them."""
    x, y = meshes("uniform_random", 110000, 90000, 8)
    g = np.random.default_rng(3)
    u, v = g.uniform(0.1, 1, 110000), g.uniform(0.1, 1, 90000)
    outs = {}
    for E in ELEMS:
        p = lib.finom_plan(T(x), T(y), 0.002, prec)
        lib.finom_plan_set_elems(p, E)
        assert lib.finom_plan_elems(p)[1] == math.ceil(200000 / POINTS[E])
        f, gg, res = lib.finom_solve(p, T(u), T(v), 0.0, 30)
        outs[E] = (H(f), H(gg), res)
    ref = outs[8]
    lock = 1e-12 if prec == "f64" else 3e-5
    for E in (-1, 1, 2, 4):
        f, gg, res = outs[E]
        assert np.max(np.abs(f - ref[0])) / 0.002 <= lock and np.max(np.abs(gg - ref[1])) / 0.002 <= lock
        if prec == "f64":
            assert res["marginal_err"] == pytest.approx(ref[2]["marginal_err"], rel=1e-9)
        else:
            assert abs(res["marginal_err"] - ref[2]["marginal_err"]) <= 2e-4 * ref[2]["marginal_err"] + 2e-7
