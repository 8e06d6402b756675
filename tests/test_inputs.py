"""The seeded input recipes (paper_2605_26659_gb300/inputs.py) produce the
workloads they are meant to: meshes sorted in [0, 1] with the stated grading,
masses normalised over the stated densities, sizes and eps in their ranges,
the arrival process at its rate and mix; the same seed gives the same data."""
import math

import numpy as np
import pytest

from paper_2605_26659_gb300 import inputs


def _is_measure(w):
    return np.all(w >= 0) and math.isclose(float(np.sum(w)), 1.0, rel_tol=1e-12)


def test_voronoi_widths_tile_the_unit_interval():
    x = np.sort(np.random.default_rng(0).uniform(0, 1, 50))
    w = inputs.voronoi_widths(x)
    assert np.all(w > 0) and math.isclose(w.sum(), 1.0, rel_tol=1e-12)
    assert w[0] == pytest.approx(0.5 * (x[0] + x[1]))


def test_config1_fp64_workload():
    p = inputs.config1()
    assert len(p.x) == len(p.y) == 1000
    assert np.all(np.diff(p.x) >= 0) and np.all(np.diff(p.y) >= 0)
    assert p.x.min() >= 0 and p.x.max() <= 1
    assert _is_measure(p.u) and _is_measure(p.v)
    assert (p.eps, p.tol, p.maxit) == (1e-2, 1e-9, 2000)
    # the same two-Gaussian density (means 0.3 / 0.7) on both meshes
    assert np.sum(p.u[(p.x > 0.2) & (p.x < 0.4)]) == pytest.approx(0.5, abs=0.05)


def test_config2_graded_meshes():
    n = 4096
    p = inputs.config2(n)
    i = np.arange(n)
    np.testing.assert_array_equal(p.x, ((i + 0.5) / n) ** 2)
    t = (i + 0.5) / n
    np.testing.assert_allclose(p.y, 0.5 * (1 + np.tanh(3 * (2 * t - 1)) / np.tanh(3)), rtol=1e-15)
    assert p.x[1] - p.x[0] < p.x[-1] - p.x[-2]            # clustered at 0
    assert p.y[1] - p.y[0] < p.y[n // 2] - p.y[n // 2 - 1]  # clustered at both ends
    assert _is_measure(p.u) and _is_measure(p.v)
    assert (p.eps, p.tol) == (1e-3, 1e-6)


def test_config3_tensor_grids():
    p = inputs.config3(64, 48)
    for a, n in ((p.x1, 64), (p.x2, 64), (p.y1, 48), (p.y2, 48)):
        assert len(a) == n and np.all(np.diff(a) > 0) and a.min() > 0 and a.max() < 1
        mid = np.searchsorted(a, 0.5)
        assert a[mid] - a[mid - 1] < a[1] - a[0]            # clustered toward the centre
    assert p.U.shape == p.V.shape == (64, 48)
    assert _is_measure(p.U.ravel()) and _is_measure(p.V.ravel())
    assert not np.array_equal(p.x1, p.x2)                   # separately seeded axes
    assert p.eps == 2e-3


def test_config4_batched_instances():
    sizes, eps = inputs.config4_sizes(4096)
    assert sizes.min() >= 256 and sizes.max() <= 65536
    assert eps.min() >= 1e-3 and eps.max() <= 1e-2
    # log-uniform: about a quarter of the sizes in each factor-of-4 band
    assert abs(np.mean(sizes < 1024) - 0.25) < 0.03
    q = inputs.config4_instance(3, 2000, 0.004)
    assert len(q.x) == len(q.y) == 2000 and np.all(np.diff(q.x) >= 0)
    assert _is_measure(q.u) and _is_measure(q.v)
    # 10 % of the points moved to 8 cluster centres: many near-duplicate gaps
    assert np.mean(np.diff(q.x) < 1e-3 / 4) > 0.05


def test_serving_arrivals():
    reqs = inputs.serving_requests(rate=2000.0, duration=1.0)
    assert 1800 < len(reqs) < 2200
    t = np.array([r.t_arrival for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] < 1.0
    assert np.mean(np.diff(t)) == pytest.approx(1 / 2000, rel=0.1)
    one = [r for r in reqs if r.kind == "1d"]
    assert abs(len(one) / len(reqs) - 0.8) < 0.04
    assert all(1000 <= r.size <= 10 ** 6 for r in one)
    assert all(64 <= r.size <= 2048 for r in reqs if r.kind == "2d")
    assert {r.eps for r in reqs} <= {1e-3, 5e-3, 1e-2}
    again = inputs.serving_requests(rate=2000.0, duration=1.0)
    assert [(r.t_arrival, r.size) for r in again] == [(r.t_arrival, r.size) for r in reqs]


def test_request_problems():
    reqs = inputs.serving_requests(rate=2000.0, duration=0.05)
    r1 = next(r for r in reqs if r.kind == "1d")
    p = inputs.request_problem(r1)
    assert len(p.x) == r1.size and _is_measure(p.u) and _is_measure(p.v)
    assert (p.eps, p.tol, p.maxit) == (r1.eps, 1e-6, 10000)
    r2 = next(r for r in reqs if r.kind == "2d" and r.size <= 300)
    q = inputs.request_problem(r2)
    assert q.U.shape == (r2.size, r2.size) and _is_measure(q.U.ravel()) and _is_measure(q.V.ravel())
