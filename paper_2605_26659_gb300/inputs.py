"""Seeded synthetic inputs for the FINOM workloads (no method arithmetic).

This module only draws meshes and mass vectors; it computes nothing of the
Sinkhorn method.  It is the one module that both the CUDA path (through the
tests and the benchmark) and the CPU oracle are fed from.  It imports neither
the CUDA library nor the oracle.

Seeds: ``numpy.random.Generator(PCG64(SEED0 + 100 * config + stream))``.

Workloads
---------
``config1``   1D, N = M = 1000, sorted U[0,1] meshes, two-Gaussian mixture
              (means 0.3 / 0.7, sigma 0.05) times cell widths; eps = 1e-2,
              tol = 1e-9, maxit = 2000.
``config2``   1D graded meshes, N = M = 2^20 by default: x_i = ((i+1/2)/N)^2,
              y_j = (1 + tanh(3 (2 t_j - 1)) / tanh 3) / 2 with t_j = (j+1/2)/M;
              three-component mixtures (means U[0.1,0.9], sigma U[0.02,0.1]);
              eps = 1e-3, tol = 1e-6.
``config3``   2D tensor-product meshes n x n (n = 1024 by default), axis nodes
              1/2 + artanh((2t-1) tanh 2.5) / 5 with stratified jitter
              t = (k + U_k)/n, four anisotropic Gaussians times cell areas;
              eps = 2e-3, tol = 1e-6.
``config4``   batch of uneven 1D instances: N log-uniform in [256, 65536],
              M = N, sorted U[0,1] meshes with 10 % of the points moved into
              8 clusters, Dirichlet(2)-perturbed two-Gaussian mixtures, eps
              log-uniform in [1e-3, 1e-2].
``serving_requests``  Poisson arrivals (2000 / s), 80 % 1D (graded meshes as
              config2, N log-uniform [1e3, 1e6]) and 20 % 2D (tanh meshes as
              config3, side log-uniform [64, 2048]), eps in {1e-3, 5e-3, 1e-2}.
``chebyshev``, ``random_nodes``, ``random_2d``  the paper's Sec. 4 workloads.

Cell widths are the Voronoi cells of the points clipped to [0, 1]: the cell
of x_i runs from the midpoint with its left neighbour (0 for the first point)
to the midpoint with its right neighbour (1 for the last point).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED0 = 2605266590

__all__ = [
    "SEED0", "rng", "voronoi_widths", "Problem1D", "Problem2D", "config1",
    "config2", "config3", "config4", "serving_requests", "chebyshev",
    "random_nodes", "random_2d", "uniform_mesh", "worked_example",
]


def rng(config: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED0 + 100 * config + stream))


def voronoi_widths(x):
    """Widths of the Voronoi cells of sorted points x, clipped to [0, 1]."""
    x = np.asarray(x, dtype=np.float64)
    mids = 0.5 * (x[1:] + x[:-1])
    left = np.concatenate([[0.0], mids])
    right = np.concatenate([mids, [1.0]])
    return np.maximum(right - left, 0.0)


def _normal_pdf(t, mu, sigma):
    return np.exp(-0.5 * ((t - mu) / sigma) ** 2) / (sigma * math.sqrt(2 * math.pi))


def _mixture(t, means, sigmas, weights):
    out = np.zeros_like(t, dtype=np.float64)
    for m, s, w in zip(means, sigmas, weights):
        out += w * _normal_pdf(t, m, s)
    return out


def _normalise(w):
    w = np.asarray(w, dtype=np.float64)
    return w / w.sum()


@dataclass
class Problem1D:
    x: np.ndarray
    y: np.ndarray
    u: np.ndarray
    v: np.ndarray
    eps: float
    tol: float
    maxit: int
    name: str = ""


@dataclass
class Problem2D:
    x1: np.ndarray      # first-axis nodes of mu's grid  (N)
    y1: np.ndarray      # second-axis nodes of mu's grid (M)
    x2: np.ndarray      # first-axis nodes of nu's grid  (N)
    y2: np.ndarray      # second-axis nodes of nu's grid (M)
    U: np.ndarray       # N x M masses of mu (column-major grid: U[k, i] at (x1_k, y1_i))
    V: np.ndarray       # N x M masses of nu
    eps: float
    tol: float
    maxit: int
    name: str = ""


def config1(n: int = 1000) -> Problem1D:
    x = np.sort(rng(1, 0).uniform(0.0, 1.0, n))
    y = np.sort(rng(1, 1).uniform(0.0, 1.0, n))
    means, sig, w = [0.3, 0.7], [0.05, 0.05], [0.5, 0.5]
    u = _normalise(_mixture(x, means, sig, w) * voronoi_widths(x))
    v = _normalise(_mixture(y, means, sig, w) * voronoi_widths(y))
    return Problem1D(x, y, u, v, eps=1e-2, tol=1e-9, maxit=2000,
                     name=f"1D FP64 N=M={n}, sorted U[0,1], 2-Gaussian mixture, eps=1e-2")


def graded_x(n):
    i = np.arange(n, dtype=np.float64)
    return ((i + 0.5) / n) ** 2


def tanh_stretched(n, stretch=3.0):
    t = (np.arange(n, dtype=np.float64) + 0.5) / n
    return 0.5 * (1.0 + np.tanh(stretch * (2.0 * t - 1.0)) / math.tanh(stretch))


def _three_mixture(g: np.random.Generator):
    means = g.uniform(0.1, 0.9, 3)
    sig = g.uniform(0.02, 0.1, 3)
    return means, sig, [1.0 / 3] * 3


def config2(n: int = 1 << 20, m: int | None = None) -> Problem1D:
    m = n if m is None else m
    x = graded_x(n)
    y = tanh_stretched(m, 3.0)
    mu_par = _three_mixture(rng(2, 2))
    nu_par = _three_mixture(rng(2, 3))
    u = _normalise(_mixture(x, *mu_par) * voronoi_widths(x))
    v = _normalise(_mixture(y, *nu_par) * voronoi_widths(y))
    return Problem1D(x, y, u, v, eps=1e-3, tol=1e-6, maxit=100000,
                     name=f"1D graded N={n} M={m}, 3-Gaussian mixtures, eps=1e-3")


def tanh_center_nodes(n, g: np.random.Generator, stretch=2.5):
    t = (np.arange(n, dtype=np.float64) + g.uniform(0.0, 1.0, n)) / n
    return np.sort(0.5 + 0.5 * np.arctanh((2.0 * t - 1.0) * math.tanh(stretch)) / stretch)


def _aniso_mixture_2d(g: np.random.Generator, ncomp=4):
    means = g.uniform(0.15, 0.85, (ncomp, 2))
    sig = g.uniform(0.03, 0.15, (ncomp, 2))
    return means, sig


def _density_2d(xa, ya, means, sig):
    out = np.zeros((len(xa), len(ya)))
    for (mx, my), (sx, sy) in zip(means, sig):
        out += np.outer(_normal_pdf(xa, mx, sx), _normal_pdf(ya, my, sy)) / len(means)
    return out


def config3(n: int = 1024, m: int | None = None) -> Problem2D:
    m = n if m is None else m
    x1 = tanh_center_nodes(n, rng(3, 0))
    y1 = tanh_center_nodes(m, rng(3, 1))
    x2 = tanh_center_nodes(n, rng(3, 2))
    y2 = tanh_center_nodes(m, rng(3, 3))
    mu = _aniso_mixture_2d(rng(3, 4))
    nu = _aniso_mixture_2d(rng(3, 5))
    U = _density_2d(x1, y1, *mu) * np.outer(voronoi_widths(x1), voronoi_widths(y1))
    V = _density_2d(x2, y2, *nu) * np.outer(voronoi_widths(x2), voronoi_widths(y2))
    return Problem2D(x1, y1, x2, y2, U / U.sum(), V / V.sum(), eps=2e-3, tol=1e-6,
                     maxit=100000, name=f"2D tanh-stretched {n}x{m}, 4 anisotropic Gaussians, eps=2e-3")


def _clustered_mesh(n, g: np.random.Generator, centers):
    pts = g.uniform(0.0, 1.0, n)
    k = max(1, n // 10)
    idx = g.choice(n, size=k, replace=False)
    c = centers[g.integers(0, len(centers), size=k)]
    pts[idx] = np.clip(c + g.normal(0.0, 1e-3, size=k), 0.0, 1.0)
    return np.sort(pts)


def config4_sizes(count: int = 4096, lo: int = 256, hi: int = 65536):
    g = rng(4, 0)
    sizes = np.exp(g.uniform(math.log(lo), math.log(hi), count)).astype(np.int64)
    eps = np.exp(g.uniform(math.log(1e-3), math.log(1e-2), count))
    return sizes, eps


def config4_instance(b: int, n: int, eps: float) -> Problem1D:
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED0 + 400, b])))
    centers = g.uniform(0.0, 1.0, 8)
    x = _clustered_mesh(n, g, centers)
    y = _clustered_mesh(n, g, centers)

    def masses(pts):
        means = g.uniform(0.2, 0.8, 2)
        sig = g.uniform(0.03, 0.15, 2)
        base = _mixture(pts, means, sig, [0.5, 0.5]) * voronoi_widths(pts)
        return _normalise(base * g.gamma(2.0, 1.0, len(pts)))

    return Problem1D(x, y, masses(x), masses(y), eps=float(eps), tol=1e-6, maxit=100000,
                     name=f"batched instance {b} N=M={n} eps={eps:.3g}")


def config4(count: int = 4096, lo: int = 256, hi: int = 65536):
    sizes, eps = config4_sizes(count, lo, hi)
    return [config4_instance(b, int(n), float(e)) for b, (n, e) in enumerate(zip(sizes, eps))]


@dataclass
class Request:
    t_arrival: float
    kind: str           # "1d" or "2d"
    size: int           # N (1D) or side (2D)
    eps: float
    seed: int
    meta: dict = field(default_factory=dict)


def serving_requests(rate: float = 2000.0, duration: float = 30.0, p1d: float = 0.8,
                     lo1=1e3, hi1=1e6, lo2=64, hi2=2048):
    g = rng(5, 0)
    t = 0.0
    out = []
    k = 0
    while True:
        t += g.exponential(1.0 / rate)
        if t >= duration:
            break
        if g.uniform() < p1d:
            size = int(math.exp(g.uniform(math.log(lo1), math.log(hi1))))
            kind = "1d"
        else:
            size = int(math.exp(g.uniform(math.log(lo2), math.log(hi2))))
            kind = "2d"
        eps = float(g.choice([1e-3, 5e-3, 1e-2]))
        out.append(Request(t, kind, size, eps, seed=SEED0 + 500 + k))
        k += 1
    return out


def request_problem(req: Request):
    g = np.random.Generator(np.random.PCG64(req.seed))
    if req.kind == "1d":
        n = req.size
        x = graded_x(n)
        y = tanh_stretched(n, 3.0)
        u = _normalise(_mixture(x, *_three_mixture(g)) * voronoi_widths(x))
        v = _normalise(_mixture(y, *_three_mixture(g)) * voronoi_widths(y))
        return Problem1D(x, y, u, v, eps=req.eps, tol=1e-6, maxit=10000, name="request-1d")
    n = req.size
    x1, y1, x2, y2 = (tanh_center_nodes(n, g) for _ in range(4))
    U = _density_2d(x1, y1, *_aniso_mixture_2d(g)) * np.outer(voronoi_widths(x1), voronoi_widths(y1))
    V = _density_2d(x2, y2, *_aniso_mixture_2d(g)) * np.outer(voronoi_widths(x2), voronoi_widths(y2))
    return Problem2D(x1, y1, x2, y2, U / U.sum(), V / V.sum(), eps=req.eps, tol=1e-6,
                     maxit=10000, name="request-2d")


def chebyshev(n: int, eps: float = 1e-2, seed_stream: int = 0) -> Problem1D:
    """Sec. 4.1: x_k = y_k = 1/2 + cos((2k-1) pi / (2N)) / 2, u, v iid U[0,1]."""
    k = np.arange(1, n + 1, dtype=np.float64)
    x = np.sort(0.5 + 0.5 * np.cos((2 * k - 1) * math.pi / (2 * n)))
    g = rng(6, seed_stream)
    return Problem1D(x, x.copy(), _normalise(g.uniform(0, 1, n)), _normalise(g.uniform(0, 1, n)),
                     eps=eps, tol=1e-9, maxit=1000, name=f"Chebyshev N={n}")


def random_nodes(n: int, m: int | None = None, eps: float = 1e-2, seed_stream: int = 0) -> Problem1D:
    """Sec. 4.2: sorted U[0,1] nodes, u, v iid U[0,1] normalised."""
    m = n if m is None else m
    g = rng(7, seed_stream)
    x = np.sort(g.uniform(0, 1, n))
    y = np.sort(g.uniform(0, 1, m))
    return Problem1D(x, y, _normalise(g.uniform(0, 1, n)), _normalise(g.uniform(0, 1, m)),
                     eps=eps, tol=1e-9, maxit=1000, name=f"random nodes N={n} M={m}")


def random_2d(n: int, m: int | None = None, eps: float = 1e-2, seed_stream: int = 0) -> Problem2D:
    """Sec. 4.3: four independent sorted U[0,1] axes, U[0,1] masses."""
    m = n if m is None else m
    g = rng(8, seed_stream)
    x1, x2 = np.sort(g.uniform(0, 1, n)), np.sort(g.uniform(0, 1, n))
    y1, y2 = np.sort(g.uniform(0, 1, m)), np.sort(g.uniform(0, 1, m))
    U = g.uniform(0, 1, (n, m))
    V = g.uniform(0, 1, (n, m))
    return Problem2D(x1, y1, x2, y2, U / U.sum(), V / V.sum(), eps=eps, tol=1e-9, maxit=1000,
                     name=f"random 2D {n}x{m}")


def uniform_mesh(n: int, eps: float = 5e-2, seed_stream: int = 0) -> Problem1D:
    """Uniform mesh (the prior-work special case): x = y = (i + 1/2)/n."""
    x = (np.arange(n, dtype=np.float64) + 0.5) / n
    g = rng(9, seed_stream)
    return Problem1D(x, x.copy(), _normalise(g.uniform(0, 1, n)), _normalise(g.uniform(0, 1, n)),
                     eps=eps, tol=1e-9, maxit=1000, name=f"uniform N={n}")


def worked_example():
    """The meshes of the paper's Example in Sec. 2.2."""
    return (np.array([1.0, 3.0, 7.0, 9.0, 12.0]), np.array([2.0, 5.0, 6.0, 9.0, 10.0]))
