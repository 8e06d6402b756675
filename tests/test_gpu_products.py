"""GPU parity of the kernel products (plan, K v, K^T u, stabilised log products).

The CUDA path (through the C ABI) against the CPU oracle on the same seeded
inputs.  Acceptance: relative error <= 1e-12 (FP64 plans) and <= 1e-5
(FP32 log-domain plans) on entries >= 1e-30 of the largest, plus the same
bound normwise; dividing indices bit-exact.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import dense, finom_serial as fs, serial_c
from tests.gpu_util import H, T, meshes, relerr

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32_log": 1e-5}


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SHAPES = [(1, 1), (1, 9), (9, 1), (7, 3), (1000, 1048), (2047, 1), (2049, 2047), (3000, 2500),
          (5000, 7000)]


def test_worked_example_dividing_index(lib):
    ex = json.load(open(os.path.join(GOLDEN, "worked_example.json")))
    p = lib.finom_plan(T(ex["x"]), T(ex["y"]), 1.0, "f64")
    z, zt = lib.finom_dividing_index(p)
    assert H(z).tolist() == ex["zeta"]
    assert H(zt).tolist() == fs.dividing_index(ex["y"], ex["x"]).tolist()


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_worked_example_kernel_powers(lib, prec):
    ex = json.load(open(os.path.join(GOLDEN, "worked_example.json")))
    eps = 1.7
    lam = math.exp(-1.0 / eps)
    K = np.array([[lam ** e for e in row] for row in ex["K_exponents"]])
    p = lib.finom_plan(T(ex["x"]), T(ex["y"]), eps, prec)
    v = np.array([0.3, 1.7, 0.2, 0.9, 1.1])
    assert relerr(H(lib.finom_kv(p, T(v))), K @ v) <= TOL[prec]
    assert relerr(H(lib.finom_ktu(p, T(v))), K.T @ v) <= TOL[prec]


@pytest.mark.parametrize("kind", ["uniform_random", "ties", "chebyshev", "disjoint"])
@pytest.mark.parametrize("N,M", SHAPES)
def test_dividing_index_exact(lib, kind, N, M):
    if kind == "chebyshev" and N != M:
        pytest.skip("x = y needs N = M")
    x, y = meshes(kind, N, M, 17 + N + M)
    p = lib.finom_plan(T(x), T(y), 0.01, "f32_log")
    z, zt = lib.finom_dividing_index(p)
    assert np.array_equal(H(z), serial_c.dividing_index(x, y))
    assert np.array_equal(H(zt), serial_c.dividing_index(y, x))


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("kind", ["uniform_random", "ties", "chebyshev", "graded", "disjoint"])
@pytest.mark.parametrize("N,M", SHAPES)
@pytest.mark.parametrize("eps", [0.05, 0.004])
def test_kv_ktu_linear(lib, prec, kind, N, M, eps):
    if kind == "chebyshev" and N != M:
        pytest.skip("x = y needs N = M")
    x, y = meshes(kind, N, M, 3 * N + M)
    g = np.random.default_rng(N * 7 + M)
    v = g.uniform(0, 1, M)
    v[g.random(M) < 0.05] = 0.0
    u = g.uniform(0, 1, N)
    p = lib.finom_plan(T(x), T(y), eps, prec)
    C = dense.cost_1d(x, y)
    tol = TOL[prec]
    assert relerr(H(lib.finom_kv(p, T(v))), dense.kv_dense(C, v, eps)) <= tol
    assert relerr(H(lib.finom_ktu(p, T(u))), dense.ktu_dense(C, u, eps)) <= tol


def _smooth_potentials(x, y, eps, seed):
    """Potentials shaped like Sinkhorn's: 1-Lipschitz plus an eps-scale wiggle."""
    g = np.random.default_rng(seed)
    c1, c2 = g.uniform(-0.8, 0.8, 2)
    a = c1 * x + 0.05 * np.sin(7 * x) + eps * g.normal(0, 0.5, len(x))
    b = -c1 * y - 0.05 * np.sin(7 * y) + c2 + eps * g.normal(0, 0.5, len(y))
    return a, b


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("N,M", [(1, 5), (700, 600), (2049, 3001), (5000, 4000)])
@pytest.mark.parametrize("eps", [0.02, 0.002])
def test_kv_log_stabilised(lib, prec, N, M, eps):
    x, y = meshes("uniform_random", N, M, N + 5 * M)
    a, b = _smooth_potentials(x, y, eps, N)
    b[::17] = -np.inf
    p = lib.finom_plan(T(x), T(y), eps, prec)
    C = dense.cost_1d(x, y)
    got = H(lib.finom_kv_log(p, T(a), T(b)))
    want = dense.log_apply_dense(C, a, b, eps)
    tol = TOL[prec]
    # relative error of exp(out) = absolute error of out
    assert np.max(np.abs(got - want)) <= tol
    got_t = H(lib.finom_ktu_log(p, T(a), T(b)))
    want_t = dense.log_apply_dense(C.T, b, a, eps)
    fin = np.isfinite(want_t)
    assert np.array_equal(np.isneginf(got_t), np.isneginf(want_t))
    assert np.max(np.abs(got_t[fin] - want_t[fin])) <= tol


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_kv_log_rough_potentials(lib, prec):
    """Absorption vectors with large point-to-point jumps (no smoothness)."""
    N, M, eps = 3000, 2600, 0.01
    x, y = meshes("uniform_random", N, M, 99)
    g = np.random.default_rng(5)
    a, b = g.normal(0, 0.05, N), g.normal(0, 0.05, M)
    p = lib.finom_plan(T(x), T(y), eps, prec)
    got = H(lib.finom_kv_log(p, T(a), T(b)))
    want = dense.log_apply_dense(dense.cost_1d(x, y), a, b, eps)
    assert np.max(np.abs(got - want)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_full_size_graded_sampled_rows(lib, prec):
    """N = M = 2^20 graded meshes (the 1D large-mesh workload): sampled rows
    of K v against exact dense row sums, and the same through K^T u."""
    from paper_2605_26659_gb300 import inputs
    prob = inputs.config2()
    p = lib.finom_plan(T(prob.x), T(prob.y), prob.eps, prec)
    kv = H(lib.finom_kv(p, T(prob.v)))
    ktu = H(lib.finom_ktu(p, T(prob.u)))
    g = np.random.default_rng(2026)
    rows = np.concatenate([[0, 1, len(prob.x) - 1], g.integers(0, len(prob.x), 125)])
    want = np.array([np.dot(np.exp(-np.abs(prob.x[i] - prob.y) / prob.eps), prob.v) for i in rows])
    want_t = np.array([np.dot(np.exp(-np.abs(prob.y[j] - prob.x) / prob.eps), prob.u) for j in rows])
    assert relerr(kv[rows], want, floor=1e-30) <= TOL[prec]
    assert relerr(ktu[rows], want_t, floor=1e-30) <= TOL[prec]


def test_invalid_inputs_are_rejected(lib):
    x = T([0.1, 0.5, 0.3])   # unsorted
    y = T([0.2, 0.4])
    with pytest.raises(lib.FinomError) as e:
        lib.finom_plan(x, y, 0.1, "f32_log")
    assert e.value.status == lib.FINOM_EINVAL
    with pytest.raises(lib.FinomError):
        lib.finom_plan(T([0.1, float("nan")]), y, 0.1, "f64")
    with pytest.raises(lib.FinomError):
        lib.finom_plan(T([0.1, 0.2]), y, 0.0, "f64")


def test_large_graded_mesh_sampled_rows(lib):
    """N = M = 2^27 graded meshes (268 M merged points, 131,072 tiles: the
    block-wide launch tail with many chunks, 64-bit offsets): sampled rows of
    K v and K^T u (float32 log-domain plan) against exact dense row sums."""
    import torch
    from paper_2605_26659_gb300 import inputs
    if torch.cuda.get_device_properties(0).total_memory < (120 << 30):
        pytest.skip("needs a GPU with > 120 GB")
    prob = inputs.config2(1 << 27)
    p = lib.finom_plan(T(prob.x), T(prob.y), prob.eps, "f32_log")
    assert lib.finom_plan_elems(p) == (8, (1 << 28) // 2048)
    kv = H(lib.finom_kv(p, T(prob.v)))
    ktu = H(lib.finom_ktu(p, T(prob.u)))
    del p
    g = np.random.default_rng(27)
    rows = np.concatenate([[0, len(prob.x) - 1], g.integers(0, len(prob.x), 6)])
    want = np.array([np.dot(np.exp(-np.abs(prob.x[i] - prob.y) / prob.eps), prob.v) for i in rows])
    want_t = np.array([np.dot(np.exp(-np.abs(prob.y[j] - prob.x) / prob.eps), prob.u) for j in rows])
    assert relerr(kv[rows], want, floor=1e-30) <= TOL["f32_log"]
    assert relerr(ktu[rows], want_t, floor=1e-30) <= TOL["f32_log"]
