"""Pins of the CPU oracle against values that do not come from the oracle.

Sources: the paper's worked example (Sec. 2.2, typed into
tests/golden/worked_example.json), LP optima (HiGHS), the 1D closed form
W1 = int |F_mu - F_nu|, the 2 x 2 entropic closed form, the Kronecker identity
K = K_y (x) K_x of Sec. 3.1 (numpy.kron), and invariants of the entropic
problem (marginals, mu <-> nu symmetry, the entropic-bias bound).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import dense, exact, finom_serial as fs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def _exp_matrix(expo, lam):
    return np.array([[0.0 if e is None else lam ** e for e in row] for row in expo])


# ---------------------------------------------------------------- worked example

@pytest.fixture(scope="module")
def ex():
    return _load("worked_example.json")


def test_example_cost_matches_kernel_exponents(ex):
    C = dense.cost_1d(ex["x"], ex["y"])
    assert np.array_equal(C, np.array(ex["K_exponents"], dtype=float))


def test_example_dividing_index(ex):
    assert fs.dividing_index(ex["x"], ex["y"]).tolist() == ex["zeta"]


@pytest.mark.parametrize("eps", [1.0, 0.7, 2.5])
def test_example_kernel_and_blocks(ex, eps):
    lam = math.exp(-1.0 / eps)
    K = dense.kernel(dense.cost_1d(ex["x"], ex["y"]), eps)
    KL = _exp_matrix(ex["K_L_exponents"], lam)
    KU = _exp_matrix(ex["K_U_exponents"], lam)
    np.testing.assert_allclose(K, _exp_matrix(ex["K_exponents"], lam), rtol=1e-14)
    np.testing.assert_allclose(KL + KU, K, rtol=1e-14)


@pytest.mark.parametrize("eps", [1.0, 0.7])
def test_example_vector_representation(ex, eps):
    lam = math.exp(-1.0 / eps)
    r, eta = fs.lower_representation(ex["x"], ex["y"], eps)
    rp, etap = fs.upper_representation(ex["x"], ex["y"], eps)
    np.testing.assert_allclose(r, [lam ** e for e in ex["r_exponents"]], rtol=1e-14)
    np.testing.assert_allclose(rp, [lam ** e for e in ex["rprime_exponents"]], rtol=1e-14)
    assert [len(e) for e in eta] == [len(e) for e in ex["eta_exponents"]]
    assert [len(e) for e in etap] == [len(e) for e in ex["etaprime_exponents"]]
    for got, want in zip(eta + etap, ex["eta_exponents"] + ex["etaprime_exponents"]):
        np.testing.assert_allclose(got, [lam ** e for e in want], rtol=1e-14)


@pytest.mark.parametrize("eps", [1.0, 3.0])
def test_example_recurrences_equal_blocks(ex, eps):
    lam = math.exp(-1.0 / eps)
    KL = _exp_matrix(ex["K_L_exponents"], lam)
    KU = _exp_matrix(ex["K_U_exponents"], lam)
    psi = np.array([0.3, 1.7, 0.2, 0.9, 1.1])
    tot, p, q = fs.matvec_linear(ex["x"], ex["y"], eps, psi)
    np.testing.assert_allclose(p, KL @ psi, rtol=1e-14)
    np.testing.assert_allclose(q, KU @ psi, rtol=1e-14)
    np.testing.assert_allclose(tot, dense.kv_dense(dense.cost_1d(ex["x"], ex["y"]), psi, eps), rtol=1e-14)


def test_example_op_count_bound(ex):
    """eq. (number of multiplications): 3N + zeta(N) - zeta(1) - 2 < 4N."""
    z = ex["zeta"]
    N = len(z)
    mults = 3 * N + z[-1] - z[0] - 2
    adds = 2 * N + z[-1] - z[0] - 2
    assert mults < 4 * N and adds < 3 * N
    # count the multiplications the recurrences perform: each eta entry times psi,
    # plus one r multiply per step, for both p and q
    r, eta = fs.lower_representation(ex["x"], ex["y"], 1.0)
    rp, etap = fs.upper_representation(ex["x"], ex["y"], 1.0)
    assert sum(len(e) for e in eta) + (N - 1) + sum(len(e) for e in etap) + (N - 1) <= mults


# ---------------------------------------------------------------- LP / closed form

@pytest.mark.parametrize("seed", range(6))
def test_lp_equals_1d_closed_form(seed):
    g = np.random.default_rng(seed)
    N, M = g.integers(1, 7, 2)
    x = np.sort(g.uniform(0, 1, N))
    y = np.sort(g.uniform(0, 1, M))
    u = g.uniform(0.1, 1, N); u /= u.sum()
    v = g.uniform(0.1, 1, M); v /= v.sum()
    lp = exact.w1_lp(dense.cost_1d(x, y), u, v)
    cf = exact.w1_closed_form_1d(x, u, y, v)
    assert abs(lp - cf) < 1e-12


def test_closed_form_two_diracs():
    # W1(delta_a, delta_b) = |a - b|
    assert exact.w1_closed_form_1d([0.2], [1.0], [0.75], [1.0]) == pytest.approx(0.55, abs=1e-15)


@pytest.mark.parametrize("eps", [0.2, 0.5, 1.0])
def test_sinkhorn_fixed_point_2x2_closed_form(eps):
    x, y = np.array([0.1, 0.6]), np.array([0.3, 0.9])
    u, v = np.array([0.35, 0.65]), np.array([0.55, 0.45])
    C = dense.cost_1d(x, y)
    G_cf, cost_cf = exact.entropic_2x2(C, u, v, eps)
    res = dense.sinkhorn_log(C, u, v, eps, tol=1e-15, maxit=5000)
    G = dense.plan_from_potentials(C, res.f, res.g, eps)
    np.testing.assert_allclose(G, G_cf, atol=1e-13)
    assert res.w1 == pytest.approx(cost_cf, rel=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_entropic_cost_converges_to_lp(seed):
    """0 <= <C,Gamma_eps> - W1_LP <= eps log(NM) (entropic bias bound)."""
    g = np.random.default_rng(100 + seed)
    N, M = 5, 6
    x = np.sort(g.uniform(0, 1, N)); y = np.sort(g.uniform(0, 1, M))
    u = g.uniform(0.1, 1, N); u /= u.sum()
    v = g.uniform(0.1, 1, M); v /= v.sum()
    C = dense.cost_1d(x, y)
    w_lp = exact.w1_lp(C, u, v)
    prev = None
    for eps in [0.1, 0.03, 0.01, 0.003]:
        res = dense.sinkhorn_log(C, u, v, eps, tol=1e-13, maxit=200000)
        assert res.converged
        gap = res.w1 - w_lp
        assert -1e-11 <= gap <= eps * math.log(N * M) + 1e-11
        if prev is not None:
            assert gap <= prev + 1e-12
        prev = gap


def test_single_source_point_is_exact():
    """N = 1: the only coupling is u_1 v^T, so W1 = sum_j v_j |x_1 - y_j|."""
    x = np.array([0.4]); y = np.array([0.1, 0.35, 0.8])
    u = np.array([1.0]); v = np.array([0.2, 0.5, 0.3])
    C = dense.cost_1d(x, y)
    res = dense.sinkhorn_log(C, u, v, 0.05, tol=1e-14, maxit=10)
    assert res.iters == 1 and res.converged
    assert res.w1 == pytest.approx(float((v * np.abs(0.4 - y)).sum()), rel=1e-13)


# ---------------------------------------------------------------- invariants

def _problem(seed, N=40, M=33):
    g = np.random.default_rng(seed)
    x = np.sort(g.uniform(0, 1, N)); y = np.sort(g.uniform(0, 1, M))
    u = g.uniform(0, 1, N); u /= u.sum()
    v = g.uniform(0, 1, M); v /= v.sum()
    return x, y, u, v


def test_marginals_after_updates():
    x, y, u, v = _problem(1)
    C = dense.cost_1d(x, y)
    eps = 0.05
    res = dense.sinkhorn_log(C, u, v, eps, tol=0.0, maxit=7)
    G = dense.plan_from_potentials(C, res.f, res.g, eps)
    # the last half step was the phi update: row sums equal u to rounding
    np.testing.assert_allclose(G.sum(1), u, rtol=1e-12)
    assert res.err == pytest.approx(np.abs(G.sum(0) - v).sum(), rel=1e-10)


def test_mu_nu_symmetry():
    x, y, u, v = _problem(2)
    C = dense.cost_1d(x, y)
    eps = 0.02
    a = dense.sinkhorn_log(C, u, v, eps, tol=1e-12, maxit=100000)
    b = dense.sinkhorn_log(C.T, v, u, eps, tol=1e-12, maxit=100000)
    assert a.converged and b.converged
    assert a.w1 == pytest.approx(b.w1, rel=1e-9)
    Ga = dense.plan_from_potentials(C, a.f, a.g, eps)
    Gb = dense.plan_from_potentials(C.T, b.f, b.g, eps)
    np.testing.assert_allclose(Ga, Gb.T, atol=1e-10)


def test_log_and_linear_iterates_agree():
    x, y, u, v = _problem(3)
    C = dense.cost_1d(x, y)
    eps = 0.05
    res = dense.sinkhorn_log(C, u, v, eps, tol=0.0, maxit=25)
    phi, psi, it, err = dense.sinkhorn_linear(C, u, v, eps, tol=0.0, maxit=25)
    np.testing.assert_allclose(np.exp(res.f / eps), phi, rtol=1e-11)
    np.testing.assert_allclose(np.exp(res.g / eps), psi, rtol=1e-11)
    assert err == pytest.approx(res.err, rel=1e-9)


def test_zero_masses_are_ignored():
    x, y, u, v = _problem(4, 12, 10)
    u[[0, 5]] = 0.0; u /= u.sum()
    v[[9]] = 0.0; v /= v.sum()
    C = dense.cost_1d(x, y)
    res = dense.sinkhorn_log(C, u, v, 0.05, tol=1e-12, maxit=100000)
    assert res.converged and np.isneginf(res.f[[0, 5]]).all() and np.isneginf(res.g[9])
    G = dense.plan_from_potentials(C, res.f, res.g, 0.05)
    np.testing.assert_allclose(G.sum(1), u, atol=1e-12)


# ---------------------------------------------------------------- serial recurrences vs dense

@pytest.mark.parametrize("seed", range(4))
def test_serial_linear_matvec_equals_dense(seed):
    x, y, u, v = _problem(10 + seed, 57, 43)
    eps = 0.03
    psi = np.random.default_rng(seed).uniform(0, 2, len(y))
    tot, p, q = fs.matvec_linear(x, y, eps, psi)
    np.testing.assert_allclose(tot, dense.kv_dense(dense.cost_1d(x, y), psi, eps), rtol=1e-13)


def test_serial_handles_ties_and_duplicates():
    x = np.array([0.1, 0.3, 0.3, 0.5, 0.9])
    y = np.array([0.0, 0.3, 0.5, 0.5, 0.95, 1.0])
    assert fs.dividing_index(x, y).tolist() == [1, 2, 2, 4, 4]
    psi = np.linspace(0.5, 1.5, len(y))
    tot, _, _ = fs.matvec_linear(x, y, 0.2, psi)
    np.testing.assert_allclose(tot, dense.kv_dense(dense.cost_1d(x, y), psi, 0.2), rtol=1e-14)
    tot_t, _, _ = fs.matvec_linear(y, x, 0.2, np.ones(len(x)))
    np.testing.assert_allclose(tot_t, dense.ktu_dense(dense.cost_1d(x, y), np.ones(len(x)), 0.2), rtol=1e-14)


def test_chebyshev_ties_dividing_index():
    """x = y (Sec. 4.1 meshes): every x_i ties with y_i, so zeta(i) = i (1-based)."""
    n = 17
    k = np.arange(1, n + 1)
    x = np.sort(0.5 + 0.5 * np.cos((2 * k - 1) * np.pi / (2 * n)))
    assert fs.dividing_index(x, x).tolist() == list(range(1, n + 1))


def test_uniform_mesh_constant_ratio():
    """Uniform mesh (prior-work case): the ratio vector is constant e^{-h/eps}."""
    n, eps = 20, 0.1
    x = (np.arange(n) + 0.5) / n
    y = np.arange(n) / n
    r, _ = fs.lower_representation(x, y, eps)
    np.testing.assert_allclose(r, np.full(n - 1, math.exp(-1.0 / n / eps)), rtol=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_serial_log_matvec_equals_dense(seed):
    x, y, u, v = _problem(20 + seed, 45, 60)
    eps = 0.004
    g = np.random.default_rng(seed)
    a = g.normal(0, 0.05, len(x))
    b = g.normal(0, 0.05, len(y))
    tot, _, _ = fs.matvec_log(x, y, eps, a, b)
    want = dense.log_apply_dense(dense.cost_1d(x, y), a, b, eps)
    np.testing.assert_allclose(tot, want, rtol=0, atol=1e-11)


def test_serial_sinkhorn_lockstep_with_dense():
    x, y, u, v = _problem(30, 50, 41)
    eps = 0.01
    C = dense.cost_1d(x, y)
    a, b, it, err = fs.sinkhorn_log(x, y, u, v, eps, tol=0.0, maxit=15)
    res = dense.sinkhorn_log(C, u, v, eps, tol=0.0, maxit=15)
    np.testing.assert_allclose(a, res.f, atol=1e-12)
    np.testing.assert_allclose(b, res.g, atol=1e-12)
    assert err == pytest.approx(res.err, rel=1e-9)


# ---------------------------------------------------------------- 2D

def _grids(seed, N=4, M=3):
    g = np.random.default_rng(seed)
    x1, x2 = np.sort(g.uniform(0, 1, N)), np.sort(g.uniform(0, 1, N))
    y1, y2 = np.sort(g.uniform(0, 1, M)), np.sort(g.uniform(0, 1, M))
    return x1, y1, x2, y2


def test_2d_cost_is_kronecker_of_axis_kernels():
    x1, y1, x2, y2 = _grids(0, 5, 4)
    eps = 0.3
    K = dense.kernel(dense.cost_2d(x1, y1, x2, y2), eps)
    Kx = dense.kernel(dense.cost_1d(x1, x2), eps)
    Ky = dense.kernel(dense.cost_1d(y1, y2), eps)
    np.testing.assert_allclose(K, np.kron(Ky, Kx), rtol=1e-14)


def test_2d_cost_explicit_entry():
    x1, y1, x2, y2 = _grids(1, 3, 2)
    C = dense.cost_2d(x1, y1, x2, y2)
    k, i, l, j = 2, 1, 0, 1
    N = 3
    assert C[k + N * i, l + N * j] == abs(x1[k] - x2[l]) + abs(y1[i] - y2[j])


def test_2d_stabilised_apply_equals_dense():
    x1, y1, x2, y2 = _grids(2, 6, 5)
    eps = 0.05
    g = np.random.default_rng(0)
    A = g.normal(0, 0.03, (6, 5)); B = g.normal(0, 0.03, (6, 5))
    C = dense.cost_2d(x1, y1, x2, y2)
    want = dense.log_apply_dense(C, A.ravel(order="F"), B.ravel(order="F"), eps)
    got = fs.apply2d_log(x1, y1, x2, y2, eps, A, B)
    np.testing.assert_allclose(got.ravel(order="F"), want, atol=1e-11)


def test_2d_sinkhorn_lockstep_and_lp():
    x1, y1, x2, y2 = _grids(3, 3, 2)
    g = np.random.default_rng(3)
    U = g.uniform(0.1, 1, (3, 2)); U /= U.sum()
    V = g.uniform(0.1, 1, (3, 2)); V /= V.sum()
    C = dense.cost_2d(x1, y1, x2, y2)
    u, v = U.ravel(order="F"), V.ravel(order="F")
    eps = 0.02
    A, B, it, err = fs.sinkhorn2d_log(x1, y1, x2, y2, U, V, eps, tol=0.0, maxit=10)
    res = dense.sinkhorn_log(C, u, v, eps, tol=0.0, maxit=10)
    np.testing.assert_allclose(A.ravel(order="F"), res.f, atol=1e-12)
    np.testing.assert_allclose(B.ravel(order="F"), res.g, atol=1e-12)
    w_lp = exact.w1_lp(C, u, v)
    res = dense.sinkhorn_log(C, u, v, 0.003, tol=1e-12, maxit=500000)
    assert res.converged
    assert -1e-10 <= res.w1 - w_lp <= 0.003 * math.log(36) + 1e-10


def test_2d_with_one_row_reduces_to_1d():
    x1, y1, x2, y2 = _grids(4, 7, 1)
    g = np.random.default_rng(4)
    U = g.uniform(0.1, 1, (7, 1)); U /= U.sum()
    V = g.uniform(0.1, 1, (7, 1)); V /= V.sum()
    eps = 0.05
    C2 = dense.cost_2d(x1, y1, x2, y2)
    C1 = dense.cost_1d(x1, x2) + abs(y1[0] - y2[0])
    np.testing.assert_allclose(C2, C1, rtol=1e-15)
    r2 = dense.sinkhorn_log(C2, U.ravel(), V.ravel(), eps, 1e-12, 100000)
    r1 = dense.sinkhorn_log(dense.cost_1d(x1, x2), U.ravel(), V.ravel(), eps, 1e-12, 100000)
    assert r2.w1 == pytest.approx(r1.w1 + abs(y1[0] - y2[0]), rel=1e-9)


def test_barycentric_single_source_point_is_the_mean():
    """With one source point every column of the converged plan holds v_j,
    so x_0 maps to the mean of nu and every y_j maps back to x_0."""
    x, y = np.array([0.37]), np.array([0.1, 0.25, 0.6, 0.8])
    u, v = np.array([1.0]), np.array([0.1, 0.2, 0.3, 0.4])
    C = dense.cost_1d(x, y)
    res = dense.sinkhorn_log(C, u, v, 0.05, tol=1e-14, maxit=100)
    tx, ty = dense.barycentric(C, res.f, res.g, 0.05, x, y)
    assert tx[0] == pytest.approx(float(v @ y), abs=1e-13)
    np.testing.assert_allclose(ty, 0.37, atol=1e-14)


def test_barycentric_small_eps_is_the_monotone_matching():
    """Equal masses on sorted, separated points: as eps -> 0 the entropic plan
    tends to the sorted matching (the 1D optimal plan for W1 with equal masses
    is monotone), so x_i maps to y_i and y_i to x_i; and swapping the roles of
    the measures transposes the maps."""
    x = np.array([0.05, 0.3, 0.55, 0.8])
    y = np.array([0.12, 0.41, 0.6, 0.95])
    w = np.full(4, 0.25)
    C = dense.cost_1d(x, y)
    res = dense.sinkhorn_log(C, w, w, 0.002, tol=1e-13, maxit=50000)
    tx, ty = dense.barycentric(C, res.f, res.g, 0.002, x, y)
    np.testing.assert_allclose(tx, y, atol=1e-6)
    np.testing.assert_allclose(ty, x, atol=1e-6)
    rs = dense.sinkhorn_log(C.T, w, w, 0.002, tol=1e-13, maxit=50000)
    sx, sy = dense.barycentric(C.T, rs.f, rs.g, 0.002, y, x)
    np.testing.assert_allclose(sx, ty, atol=1e-6)
    np.testing.assert_allclose(sy, tx, atol=1e-6)
