"""Write the full-size oracle results that the GPU parity tests compare with.

Stored values come from the CPU oracle only (``oracle.serial_c``: the float64
FINOM recurrences of Sec. 2.3 inside Algorithm 1 / Algorithm 2, pinned to the
dense definition by ``tests/test_oracle_serial_c.py``).  Inputs are the seeded
workload recipes of ``paper_2605_26659_gb300.inputs`` (draws only, no method
arithmetic).  Nothing here touches the CUDA library.

Usage (from the repository root; each config is independent):

    python tests/golden/make_full_size.py config1
    python tests/golden/make_full_size.py config2      # ~1 h on one core
    python tests/golden/make_full_size.py config3      # ~30 min on one core
    python tests/golden/make_full_size.py config4 -j 8 # a subset of the batch

Each run writes ``tests/golden/full_<config>.json`` with the solve's
iteration count, float64 marginal error at the stop, W1 = <C, Gamma>, the dual
value, and the potentials at a strided sample of points (for the batch: one
record per instance), plus the command and seeds that made it.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import serial_c  # noqa: E402
from paper_2605_26659_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SAMPLE = 512   # potentials stored at this many evenly spaced points (per axis in 2D)


def _finite(a):
    a = np.asarray(a, dtype=np.float64)
    return [float(v) if np.isfinite(v) else None for v in a]


def _dual(u, f, v, g):
    su = float(np.sum(u[u > 0] * f[u > 0]))
    sv = float(np.sum(v[v > 0] * g[v > 0]))
    return su + sv


def solve_1d(pr, maxit=None, sample=SAMPLE):
    t0 = time.time()
    maxit = pr.maxit if maxit is None else maxit
    f, g, it, err = serial_c.sinkhorn(pr.x, pr.y, pr.u, pr.v, pr.eps, pr.tol, maxit)
    w1 = serial_c.cost(pr.x, pr.y, pr.eps, f, g)
    ix = np.unique(np.linspace(0, len(pr.x) - 1, min(sample, len(pr.x))).astype(np.int64))
    iy = np.unique(np.linspace(0, len(pr.y) - 1, min(sample, len(pr.y))).astype(np.int64))
    return {
        "N": len(pr.x), "M": len(pr.y), "eps": pr.eps, "tol": pr.tol, "maxit": int(maxit),
        "iters": it, "marginal_err": err, "w1": w1, "dual": _dual(pr.u, f, pr.v, g),
        "converged": bool(err <= pr.tol),
        "f_index": ix.tolist(), "f": _finite(f[ix]), "g_index": iy.tolist(), "g": _finite(g[iy]),
        "oracle_seconds": round(time.time() - t0, 1),
    }


def config1():
    pr = inputs.config1()
    return {"workload": pr.name, "recipe": "inputs.config1()", **solve_1d(pr)}


def config2(n):
    pr = inputs.config2(n)
    return {"workload": pr.name, "recipe": f"inputs.config2({n})", **solve_1d(pr)}


def config3(n):
    pr = inputs.config3(n)
    t0 = time.time()
    A, B, it, err = serial_c.sinkhorn2d(pr.x1, pr.y1, pr.x2, pr.y2, pr.U, pr.V, pr.eps, pr.tol,
                                        pr.maxit)
    w1 = serial_c.cost2d(pr.x1, pr.y1, pr.x2, pr.y2, pr.eps, A, B)
    k = np.unique(np.linspace(0, n - 1, min(32, n)).astype(np.int64))
    dual = float(np.sum(pr.U[pr.U > 0] * A[pr.U > 0]) + np.sum(pr.V[pr.V > 0] * B[pr.V > 0]))
    return {
        "workload": pr.name, "recipe": f"inputs.config3({n})", "N": n, "M": n, "eps": pr.eps,
        "tol": pr.tol, "maxit": pr.maxit, "iters": it, "marginal_err": err, "w1": w1,
        "dual": dual, "converged": bool(err <= pr.tol), "index": k.tolist(),
        "A": [_finite(A[i, k]) for i in k], "B": [_finite(B[i, k]) for i in k],
        "oracle_seconds": round(time.time() - t0, 1),
    }


def config4_subset(count=4096):
    """Instances of the 4096-instance batch spanning its size range: the 6
    largest (N up to 65,536), the 6 smallest, and 12 evenly spaced by rank."""
    sizes, eps = inputs.config4_sizes(count)
    order = np.argsort(sizes, kind="stable")
    pick = list(order[-6:]) + list(order[:6]) + list(order[np.linspace(6, count - 7, 12).astype(int)])
    return sorted({int(b) for b in pick}), sizes, eps


def _one4(args):
    b, n, e = args
    pr = inputs.config4_instance(b, n, e)
    r = solve_1d(pr, sample=48)
    r["instance"] = b
    return r


def config4(jobs):
    bs, sizes, eps = config4_subset()
    work = [(b, int(sizes[b]), float(eps[b])) for b in bs]
    work.sort(key=lambda w: -w[1])
    with mp.get_context("spawn").Pool(jobs) as pool:
        recs = pool.map(_one4, work, chunksize=1)
    recs.sort(key=lambda r: r["instance"])
    return {"workload": "batched uneven 1D instances (subset of the 4096-instance batch)",
            "recipe": "inputs.config4_instance(b, sizes[b], eps[b]) for b in instances",
            "instances": recs}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("config", choices=["config1", "config2", "config3", "config4"])
    ap.add_argument("-n", type=int, default=None, help="size (config2: N = M; config3: side)")
    ap.add_argument("-j", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("-o", default=None)
    a = ap.parse_args()
    t0 = time.time()
    if a.config == "config1":
        rec = config1()
    elif a.config == "config2":
        rec = config2(a.n or (1 << 20))
    elif a.config == "config3":
        rec = config3(a.n or 1024)
    else:
        rec = config4(a.j)
    rec["command"] = "python tests/golden/make_full_size.py " + " ".join(sys.argv[1:])
    rec["seed0"] = inputs.SEED0
    rec["generator_seconds"] = round(time.time() - t0, 1)
    out = a.o or os.path.join(HERE, f"full_{a.config}.json")
    with open(out, "w") as fh:
        json.dump(rec, fh, indent=1)
        fh.write("\n")
    print(out, rec.get("iters"), rec.get("w1"), rec.get("marginal_err"), rec["generator_seconds"])


if __name__ == "__main__":
    main()
