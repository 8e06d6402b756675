"""Transport-plan queries (rows, columns, barycentric projections) against the
dense oracle evaluated on the same potentials."""
import numpy as np
import pytest

from oracle import dense
from tests.gpu_util import H, T, meshes

pytestmark = pytest.mark.gpu


def _solved(lib, prec, N=2500, M=1900, eps=0.01, zeros=False):
    x, y = meshes("graded", N, M, 5)
    g = np.random.default_rng(9)
    u, v = g.uniform(0.1, 1, N), g.uniform(0.1, 1, M)
    if zeros:
        u[::37] = 0.0
        v[::41] = 0.0
    u, v = u / u.sum(), v / v.sum()
    p = lib.finom_plan(T(x), T(y), eps, prec)
    f, gg, res = lib.finom_solve(p, T(u), T(v), 1e-6, 20000)
    return p, x, y, f, gg, eps


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("zeros", [False, True])
def test_rows_and_columns(lib, prec, zeros):
    p, x, y, f, g, eps = _solved(lib, prec, zeros=zeros)
    G = dense.plan_from_potentials(dense.cost_1d(x, y), H(f), H(g), eps)
    for i in (0, 1, 777, len(x) - 1):
        np.testing.assert_allclose(H(lib.finom_transport_row(p, f, g, i)), G[i], rtol=1e-13, atol=0)
    for j in (0, 500, len(y) - 1):
        np.testing.assert_allclose(H(lib.finom_transport_col(p, f, g, j)), G[:, j], rtol=1e-13, atol=0)


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
@pytest.mark.parametrize("zeros", [False, True])
def test_barycentric_projections(lib, prec, zeros):
    p, x, y, f, g, eps = _solved(lib, prec, zeros=zeros)
    tx, ty = lib.finom_barycentric(p, f, g)
    C = dense.cost_1d(x, y)
    # the oracle on the same potentials, with -inf rows and columns kept at
    # their weights (a point without mass maps to the mean under its kernel row)
    fo, go = H(f), H(g)
    fz, gz = np.where(np.isfinite(fo), fo, 0.0), np.where(np.isfinite(go), go, -np.inf)
    with np.errstate(invalid="ignore"):   # the unused side has 0/0 at points without mass
        wx, _ = dense.barycentric(C, fz, gz, eps, x, y)
        fz2, gz2 = np.where(np.isfinite(fo), fo, -np.inf), np.where(np.isfinite(go), go, 0.0)
        _, wy = dense.barycentric(C, fz2, gz2, eps, x, y)
    tol = 1e-10 if prec == "f64" else 5e-5
    assert np.max(np.abs(H(tx) - wx)) <= tol
    assert np.max(np.abs(H(ty) - wy)) <= tol
    # the projections stay inside the other mesh's range
    assert H(tx).min() >= y.min() - tol and H(tx).max() <= y.max() + tol


def test_query_argument_errors(lib):
    p, x, y, f, g, eps = _solved(lib, "f32_log", N=300, M=200)
    with pytest.raises(lib.FinomError) as e:
        lib.finom_transport_row(p, f, g, 300)
    assert e.value.status == lib.FINOM_EINVAL
    with pytest.raises(lib.FinomError) as e:
        lib.finom_transport_col(p, f, g, -1)
    assert e.value.status == lib.FINOM_EINVAL
    p2 = lib.finom_plan_2d(T(x[:10]), T(x[:10]), T(y[:8]), T(y[:8]), 0.01, "f32_log")
    with pytest.raises(lib.FinomError) as e:
        lib.finom_barycentric(p2, T(np.zeros(80)), T(np.zeros(80)))
    assert e.value.status in (lib.FINOM_ENOTSUP, lib.FINOM_EINVAL)
