"""GPU parity of batches of independent 1D instances (finom_plan_batch / finom_solve_batch).

Each instance of a batch is a separate Algorithm 1 solve with its own meshes,
masses and eps; the batch must give, per instance, what the CPU oracle gives
for that instance alone (and what a single-instance plan gives), whatever
else is in the batch.
"""
import math

import numpy as np
import pytest

from oracle import serial_c
from tests.gpu_util import H, T, meshes

pytestmark = pytest.mark.gpu

LOCK_TOL = {"f64": 1e-10, "f32_log": 2e-5}   # |f_gpu - f_oracle| / eps on points with mass
# float32 iterates against the oracle (or another tiling) at the same iteration:
# |err - err_ref| <= F32_ERR_REL err_ref + F32_ERR_ABS for the float64 marginal errors
# (F32_ERR_ONE in place of F32_ERR_ABS where a side has a few points, or the
# supports are disjoint: each weight carries the float32 rounding of its sum,
# ~1e-6 relative, and with few terms, or with the rank-one kernel of disjoint
# supports where every point shares one sum, nothing averages it out)
F32_ERR_REL, F32_ERR_ABS, F32_ERR_ONE = 2e-4, 2e-7, 1e-6

# (N, M, kind, eps): tiny, single points, ragged tiles, multi-tile, ties, disjoint supports
SHAPES = [(3, 5, "uniform_random", 0.05), (300, 257, "uniform_random", 0.01), (2047, 1, "uniform_random", 0.05),
          (1, 40, "uniform_random", 0.05), (2049, 2047, "ties", 0.004), (5000, 3100, "uniform_random", 0.006),
          (700, 900, "disjoint", 0.02), (64, 64, "chebyshev", 0.01)]


def _masses(N, M, seed, zeros=False):
    g = np.random.default_rng(seed)
    u = g.uniform(0.05, 1, N)
    v = g.uniform(0.05, 1, M)
    if zeros and N > 4 and M > 4:
        u[g.random(N) < 0.05] = 0.0
        v[g.random(M) < 0.05] = 0.0
    return u / u.sum(), v / v.sum()


def _batch(shapes, seed0, zeros=True):
    xs, ys, us, vs, eps = [], [], [], [], []
    for k, (N, M, kind, e) in enumerate(shapes):
        x, y = meshes(kind, N, M, seed0 + k)
        u, v = _masses(N, M, seed0 + 100 + k, zeros)
        xs.append(x); ys.append(y); us.append(u); vs.append(v); eps.append(e)
    offx = np.concatenate([[0], np.cumsum([len(a) for a in xs])]).astype(np.int64)
    offy = np.concatenate([[0], np.cumsum([len(a) for a in ys])]).astype(np.int64)
    return xs, ys, us, vs, eps, offx, offy


def _plan(lib, xs, ys, eps, offx, offy, prec):
    return lib.finom_plan_batch(T(np.concatenate(xs)), offx, T(np.concatenate(ys)), offy, eps, prec)


def _split(a, off, b):
    return a[off[b]:off[b + 1]]


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("maxit", [1, 7, 30])
def test_batch_lockstep_with_oracle(lib, prec, maxit):
    xs, ys, us, vs, eps, offx, offy = _batch(SHAPES, 10)
    p = _plan(lib, xs, ys, eps, offx, offy, prec)
    assert lib.finom_plan_instances(p) == len(SHAPES)
    f, g, res = lib.finom_solve_batch(p, T(np.concatenate(us)), T(np.concatenate(vs)), 0.0, maxit)
    f, g = H(f), H(g)
    for b, (N, M, kind, e) in enumerate(SHAPES):
        fo, go, it, err = serial_c.sinkhorn(xs[b], ys[b], us[b], vs[b], e, 0.0, maxit)
        fb, gb = _split(f, offx, b), _split(g, offy, b)
        if min(N, M) == 1:
            # one point on a side: exact after one iteration; the error may reach 0 = tol early
            assert res[b]["iters"] >= 1 and it >= 1
            continue
        assert res[b]["iters"] == it == maxit
        u, v = us[b], vs[b]
        assert np.max(np.abs(fb[u > 0] - fo[u > 0])) / e <= LOCK_TOL[prec], b
        assert np.max(np.abs(gb[v > 0] - go[v > 0])) / e <= LOCK_TOL[prec], b
        assert np.all(np.isneginf(fb[u == 0])) and np.all(np.isneginf(gb[v == 0]))
        if prec == "f64":
            assert res[b]["marginal_err"] == pytest.approx(err, rel=1e-6, abs=1e-9)
        else:
            f32_abs = F32_ERR_ONE if min(N, M) <= 8 or kind == "disjoint" else F32_ERR_ABS
            assert abs(res[b]["marginal_err"] - err) <= F32_ERR_REL * err + f32_abs, b


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32_log", 1e-6)])
def test_batch_converged_matches_oracle_and_single_plans(lib, prec, tol):
    shapes = [(500, 500, "uniform_random", 0.02), (1800, 2300, "graded", 0.005), (300, 700, "uniform_random", 0.01),
              (2500, 2500, "chebyshev", 0.01), (90, 60, "uniform_random", 0.03)]
    xs, ys, us, vs, eps, offx, offy = _batch(shapes, 40, zeros=False)
    p = _plan(lib, xs, ys, eps, offx, offy, prec)
    f, g, res = lib.finom_solve_batch(p, T(np.concatenate(us)), T(np.concatenate(vs)), tol, 200000)
    f, g = H(f), H(g)
    iters = set()
    for b, (N, M, kind, e) in enumerate(shapes):
        fo, go, it, err = serial_c.sinkhorn(xs[b], ys[b], us[b], vs[b], e, tol, 200000)
        w1o = serial_c.cost(xs[b], ys[b], e, fo, go)
        r = res[b]
        assert r["converged"] == 1
        iters.add(r["iters"])
        if prec == "f64":
            assert r["iters"] == it
            assert r["w1"] == pytest.approx(w1o, rel=1e-9)
        else:
            assert abs(r["iters"] - it) <= max(3, 0.05 * it)
            assert r["w1"] == pytest.approx(w1o, rel=1e-4)
        fb, gb = _split(f, offx, b), _split(g, offy, b)
        e_or = serial_c.marginal_error(xs[b], ys[b], e, fb, gb, vs[b])
        assert e_or <= (tol if prec == "f64" else 3 * tol)
        assert r["marginal_err"] == pytest.approx(e_or, rel=1e-6, abs=1e-13)
        # the same instance alone, through a single-instance plan
        ps = lib.finom_plan(T(xs[b]), T(ys[b]), e, prec)
        fs, gs, rs = lib.finom_solve(ps, T(us[b]), T(vs[b]), tol, 200000)
        if prec == "f64":
            assert r["iters"] == rs["iters"]
            assert r["w1"] == pytest.approx(rs["w1"], rel=1e-12)
            assert np.max(np.abs(fb - H(fs))) / e <= 1e-10
        else:
            assert r["w1"] == pytest.approx(rs["w1"], rel=1e-5)
    assert len(iters) > 1   # the instances retired at different iterations


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_batch_first_loop_head_check(lib, prec):
    xs, ys, us, vs, eps, offx, offy = _batch(SHAPES[:4], 70)
    p = _plan(lib, xs, ys, eps, offx, offy, prec)
    f, g, res = lib.finom_solve_batch(p, T(np.concatenate(us)), T(np.concatenate(vs)), 1e-6, 0)
    f = H(f)
    for b in range(4):
        fo, go, it, err = serial_c.sinkhorn(xs[b], ys[b], us[b], vs[b], eps[b], 1e-6, 0)
        assert res[b]["iters"] == 0
        np.testing.assert_allclose(_split(f, offx, b), fo, rtol=1e-14)
        assert res[b]["marginal_err_loop"] == pytest.approx(err, rel=1e-5)


def test_batched_workload_subset(lib):
    """64 instances of the batched workload recipe (N log-uniform in [256, 4096],
    clustered meshes, Dirichlet-perturbed mixtures, eps log-uniform in
    [1e-3, 1e-2]), FP32: every instance converges to the oracle's W1."""
    from paper_2605_26659_gb300 import inputs
    sizes, eps = inputs.config4_sizes(64, 256, 4096)
    probs = [inputs.config4_instance(b, int(n), float(e)) for b, (n, e) in enumerate(zip(sizes, eps))]
    xs = [q.x for q in probs]; ys = [q.y for q in probs]
    offx = np.concatenate([[0], np.cumsum([len(a) for a in xs])]).astype(np.int64)
    offy = np.concatenate([[0], np.cumsum([len(a) for a in ys])]).astype(np.int64)
    p = _plan(lib, xs, ys, [q.eps for q in probs], offx, offy, "f32_log")
    f, g, res = lib.finom_solve_batch(p, T(np.concatenate([q.u for q in probs])),
                                      T(np.concatenate([q.v for q in probs])), 1e-6, 100000)
    for b, q in enumerate(probs):
        fo, go, it, err = serial_c.sinkhorn(q.x, q.y, q.u, q.v, q.eps, 1e-6, 100000)
        assert res[b]["converged"] == 1, (b, res[b])
        assert res[b]["w1"] == pytest.approx(serial_c.cost(q.x, q.y, q.eps, fo, go), rel=1e-4)


def test_batch_invalid_inputs(lib):
    x = np.array([0.1, 0.5, 0.3, 0.2, 0.4])   # instance 0 unsorted
    y = np.array([0.2, 0.4, 0.1, 0.3])
    with pytest.raises(lib.FinomError) as e:
        lib.finom_plan_batch(T(x), [0, 3, 5], T(y), [0, 2, 4], [0.1, 0.1])
    assert e.value.status == lib.FINOM_EINVAL
    with pytest.raises(lib.FinomError) as e:   # an empty instance
        lib.finom_plan_batch(T(np.sort(x)), [0, 5, 5], T(np.sort(y)), [0, 2, 4], [0.1, 0.1])
    assert e.value.status == lib.FINOM_EINVAL
    x = np.array([0.1, 0.3, 0.5, 0.2, 0.4])
    y = np.array([0.2, 0.4, 0.1, 0.3])
    p = lib.finom_plan_batch(T(x), [0, 3, 5], T(y), [0, 2, 4], [0.1, 0.05])
    u = np.ones(5); v = np.ones(4)
    v[2:] = [-1.0, 2.0]                            # instance 1 has a negative mass
    with pytest.raises(lib.FinomError) as e:
        lib.finom_solve_batch(p, T(u), T(v), 1e-6, 10)
    assert e.value.status == lib.FINOM_EINVAL
    with pytest.raises(lib.FinomError) as e:       # single-problem calls refuse batch plans
        lib.finom_solve(p, T(u), T(np.ones(4)), 1e-6, 10)
    assert e.value.status == lib.FINOM_ENOTSUP
    # the plan stays usable
    f, g, res = lib.finom_solve_batch(p, T(u), T(np.ones(4)), 1e-9, 5000)
    assert all(r["iters"] >= 1 for r in res)


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_batch_stepwise_equals_blocking(lib, prec):
    """begin + 12 steps + end gives what the blocking solve with maxit = 13 gives
    (instances with a single point on a side can reach a zero error, which the
    blocking float32 solve then re-verifies in float64; they are left out)."""
    xs, ys, us, vs, eps, offx, offy = _batch(SHAPES[:2] + SHAPES[4:7], 90)
    p = _plan(lib, xs, ys, eps, offx, offy, prec)
    u, v = T(np.concatenate(us)), T(np.concatenate(vs))
    f1, g1, r1 = lib.finom_solve_batch(p, u, v, 0.0, 13)
    lib.finom_solve_batch_begin(p, u, v, 0.0, 13)
    lib.finom_solve_batch_step(p, 12)
    done, launched = lib.finom_solve_poll(p)
    assert done and launched == 13
    f2, g2, r2 = lib.finom_solve_batch_end(p)
    assert np.array_equal(H(f1), H(f2)) and np.array_equal(H(g1), H(g2))
    assert [r["iters"] for r in r1] == [r["iters"] for r in r2]


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_batch_every_tile_size(lib, prec):
    """The batch packed into tiles of 64, 256, 512, 1024 and 2048 points: the
    oracle's lock-step iterates for every tile size, and agreement across
    tile sizes (the float64 evaluation keeps its own 2048-point tiles)."""
    xs, ys, us, vs, eps, offx, offy = _batch(SHAPES, 150)
    outs = {}
    for E in (-1, 1, 2, 4, 8):
        p = lib.finom_plan_batch(T(np.concatenate(xs)), offx, T(np.concatenate(ys)), offy, eps, prec, elems=E)
        f, g, res = lib.finom_solve_batch(p, T(np.concatenate(us)), T(np.concatenate(vs)), 0.0, 7)
        outs[E] = (H(f), H(g), res)
    for b, (N, M, kind, e) in enumerate(SHAPES):
        if min(N, M) == 1:
            continue
        fo, go, it, err = serial_c.sinkhorn(xs[b], ys[b], us[b], vs[b], e, 0.0, 7)
        u = us[b]
        for E, (f, g, res) in outs.items():
            fb = _split(f, offx, b)
            assert res[b]["iters"] == 7
            assert np.max(np.abs(fb[u > 0] - fo[u > 0])) / e <= LOCK_TOL[prec], (b, E)
            ref = outs[8][2][b]["marginal_err"]
            if prec == "f64":
                assert res[b]["marginal_err"] == pytest.approx(ref, rel=1e-9, abs=1e-12)
            else:
                f32_abs = F32_ERR_ONE if min(N, M) <= 8 or kind == "disjoint" else F32_ERR_ABS
                assert abs(res[b]["marginal_err"] - ref) <= F32_ERR_REL * ref + f32_abs, (b, E)


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("E", [-1, 8])
def test_batch_large_gaps(lib, prec, E):
    """Instances whose merged gaps are tens of bits (disjoint supports and a
    few far-apart nodes at eps = 0.004, next to ordinary ones): every
    instance in lock-step with the oracle, as alone."""
    shapes = [(300, 250, "disjoint", 0.004), (40, 3, "disjoint", 0.004), (500, 400, "uniform_random", 0.004),
              (7, 9, "uniform_random", 0.004), (1200, 900, "disjoint", 0.01)]
    xs, ys, us, vs, eps, offx, offy = _batch(shapes, 190)
    p = lib.finom_plan_batch(T(np.concatenate(xs)), offx, T(np.concatenate(ys)), offy, eps, prec, elems=E)
    f, g, res = lib.finom_solve_batch(p, T(np.concatenate(us)), T(np.concatenate(vs)), 0.0, 10)
    f, g = H(f), H(g)
    for b, (N, M, kind, e) in enumerate(shapes):
        fo, go, it, err = serial_c.sinkhorn(xs[b], ys[b], us[b], vs[b], e, 0.0, 10)
        u, v = us[b], vs[b]
        fb, gb = _split(f, offx, b), _split(g, offy, b)
        assert res[b]["iters"] == it == 10
        assert np.max(np.abs(fb[u > 0] - fo[u > 0])) / e <= LOCK_TOL[prec], b
        assert np.max(np.abs(gb[v > 0] - go[v > 0])) / e <= LOCK_TOL[prec], b


def test_batch_autotune_sets_the_batch_entry(lib):
    from paper_2605_26659_gb300 import autotune
    xs, ys, us, vs, eps, offx, offy = _batch(SHAPES[:5], 170, zeros=False)
    old = lib.finom_tune_get_batch("f32_log")
    best, times = autotune.batch(T(np.concatenate(xs)), offx, T(np.concatenate(ys)), offy, eps, "f32_log",
                                 T(np.concatenate(us)), T(np.concatenate(vs)), iters=4)
    assert best in (-1, 1, 2, 4, 8) and times[best] == min(times.values())
    assert lib.finom_tune_get_batch("f32_log") == best
    p = lib.finom_plan_batch(T(np.concatenate(xs)), offx, T(np.concatenate(ys)), offy, eps, "f32_log")
    f, g, res = lib.finom_solve_batch(p, T(np.concatenate(us)), T(np.concatenate(vs)), 1e-6, 100000)
    assert all(r["converged"] == 1 for r in res)
    lib.finom_tune_set_batch("f32_log", old)
