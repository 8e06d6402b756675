"""The allocation-free product finom_kv_log_noalloc against finom_kv_log and
against the CPU oracle.

Some callers cannot allocate device memory while they run (memory owned by a
fixed pool or another allocator, a hard budget, no tolerance for allocator
locks).  finom_kv_log_noalloc serves them from a static device array; this
file checks, through the C ABI, that two calls in a row give the product that
finom_kv_log gives and the dense definition of the oracle, for smooth and for
rough absorption vectors, and that plans beyond the array's limit are refused.
Collected last on purpose (test_zz_*), so a failure here does not hide others.
"""
import numpy as np
import pytest

from oracle import dense
from tests.gpu_util import H, T, meshes

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32_log": 1e-5}


def _potentials(x, y, eps, seed):
    g = np.random.default_rng(seed)
    c1 = g.uniform(-0.8, 0.8)
    a = c1 * x + 0.05 * np.sin(7 * x) + eps * g.normal(0, 0.5, len(x))
    b = -c1 * y - 0.05 * np.sin(7 * y) + 0.1 + eps * g.normal(0, 0.5, len(y))
    b[::23] = -np.inf
    return a, b


@pytest.mark.parametrize("prec", ["f32_log", "f64"])
@pytest.mark.parametrize("N,M,eps", [(3000, 2500, 0.01), (700, 5200, 0.003), (1, 7, 0.05)])
def test_noalloc_matches_kv_log_twice(lib, prec, N, M, eps):
    x, y = meshes("uniform_random", N, M, N + 11 * M)
    a, b = _potentials(x, y, eps, N + M)
    p = lib.finom_plan(T(x), T(y), eps, prec)
    ta, tb = T(a), T(b)
    want = H(lib.finom_kv_log(p, ta, tb))
    for _ in range(2):   # the static scratch keeps the previous call's contents
        got = H(lib.finom_kv_log_noalloc(p, ta, tb))
        assert np.max(np.abs(got - want)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f32_log", "f64"])
@pytest.mark.parametrize("rough", [False, True])
@pytest.mark.parametrize("N,M,eps", [(3000, 2500, 0.01), (700, 2200, 0.003), (1, 7, 0.05)])
def test_noalloc_matches_oracle(lib, prec, rough, N, M, eps):
    """Against the dense definition (oracle), smooth absorption vectors and
    rough ones whose neighbouring entries jump by several eps."""
    x, y = meshes("uniform_random", N, M, 3 * N + M)
    a, b = _potentials(x, y, eps, N + 7 * M)
    if rough:
        g = np.random.default_rng(N * M)
        a = a + eps * g.uniform(-6, 6, N)
        b = b + eps * g.uniform(-6, 6, M)
    p = lib.finom_plan(T(x), T(y), eps, prec)
    want = dense.log_apply_dense(dense.cost_1d(x, y), a, b, eps)
    for _ in range(2):
        got = H(lib.finom_kv_log_noalloc(p, T(a), T(b)))
        # relative error of exp(out) = absolute error of out
        assert np.max(np.abs(got - want)) <= TOL[prec]


def test_noalloc_refuses_plans_beyond_its_scratch(lib):
    n = 4 * 1024 * 1024 + 8   # N + M just above 4096 tiles of 2048 points
    x = np.linspace(0.0, 1.0, n)
    p = lib.finom_plan(T(x), T(x), 0.01, "f32_log")
    with pytest.raises(lib.FinomError) as e:
        lib.finom_kv_log_noalloc(p, T(np.zeros(n)), T(np.zeros(n)))
    assert e.value.status == lib.FINOM_EINVAL
