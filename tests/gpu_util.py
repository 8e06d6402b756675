"""Helpers shared by the GPU tests (tensor conversion, error metrics)."""
import numpy as np


def T(a, dtype=None):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float64), dtype=dtype or torch.float64, device="cuda")


def H(t):
    return t.detach().cpu().numpy()


def relerr(got, want, floor=1e-30):
    """Max elementwise relative error over entries >= floor * max|want|, and the L1 normwise one."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    m = np.max(np.abs(want))
    mask = np.abs(want) >= floor * m
    elem = float(np.max(np.abs(got[mask] - want[mask]) / np.abs(want[mask]))) if mask.any() else 0.0
    norm = float(np.sum(np.abs(got - want)) / np.sum(np.abs(want)))
    return max(elem, norm)


def meshes(kind, N, M, seed):
    g = np.random.default_rng(seed)
    if kind == "uniform_random":
        return np.sort(g.uniform(0, 1, N)), np.sort(g.uniform(0, 1, M))
    if kind == "ties":
        return (np.sort(np.round(g.uniform(0, 1, N) * 53) / 53),
                np.sort(np.round(g.uniform(0, 1, M) * 53) / 53))
    if kind == "chebyshev":
        k = np.arange(1, N + 1)
        x = np.sort(0.5 + 0.5 * np.cos((2 * k - 1) * np.pi / (2 * N)))
        return x, x.copy()[:M] if M <= N else x
    if kind == "graded":
        i = np.arange(N)
        j = np.arange(M)
        t = (j + 0.5) / M
        return ((i + 0.5) / N) ** 2, 0.5 * (1 + np.tanh(3 * (2 * t - 1)) / np.tanh(3))
    if kind == "disjoint":   # all x left of all y
        return np.sort(g.uniform(0, 0.4, N)), np.sort(g.uniform(0.6, 1, M))
    raise ValueError(kind)
