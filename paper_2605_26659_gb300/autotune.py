"""Autotuner of the kernel's tile size (points per thread) for 1D plans.

`run()` calls the library's native autotuner (finom_autotune) for every size
bucket 2^lo .. 2^hi of both precisions, which times a few Sinkhorn
iterations of a synthetic problem per candidate and installs the fastest in
the library's table; the table is written to a JSON cache.  `batch()` times
the candidates on a given batch of instances and sets the batch entry.  `apply()` loads
a cache into the library (api.load() does this when FINOM_TUNE_CACHE names
a file).  Usage on the GPU: python -m paper_2605_26659_gb300.autotune out.json
"""
from __future__ import annotations

import json
import sys

from . import api

PRECISIONS = ("f64", "f32_log")


def run(lo: int = 10, hi: int = 22, iters: int = 64, path: str | None = None):
    table = {"buckets": {}, "times_us": {}}
    for prec in PRECISIONS:
        table["buckets"][prec] = {}
        table["times_us"][prec] = {}
        for b in range(lo, hi + 1):
            best, times = api.finom_autotune(prec, b, iters)
            table["buckets"][prec][str(b)] = best
            table["times_us"][prec][str(b)] = {str(k): round(v, 3) for k, v in times.items()}
    if path:
        with open(path, "w") as f:
            json.dump(table, f, indent=1)
    return table


def batch(x, offx, y, offy, eps, precision="f32_log", u=None, v=None, iters=8, warmup=3):
    """The batch entry of the table: plans the batch with every candidate
    number of points per thread, times `iters` iterations of every instance
    (CUDA events, after `warmup`), installs the fastest as the batch default
    (finom_tune_set_batch); returns (best, {E: ms per iteration})."""
    import numpy as np
    import torch
    dev = x.device
    if u is None:
        u = torch.ones(int(offx[-1]), dtype=torch.float64, device=dev)
    if v is None:
        v = torch.ones(int(offy[-1]), dtype=torch.float64, device=dev)
    times = {}
    for e in (-1, 1, 2, 4, 8):
        p = api.finom_plan_batch(x, offx, y, offy, eps, precision, elems=e)
        api.finom_solve_batch_begin(p, u, v, 0.0, 1 << 30)
        api.finom_solve_batch_step(p, warmup)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        api.finom_solve_batch_step(p, iters)
        t1.record()
        torch.cuda.synchronize()
        times[e] = t0.elapsed_time(t1) / iters
        api.finom_plan_destroy(p)
    best = min(times, key=times.get)
    api.finom_tune_set_batch(precision, best)
    return best, times


def apply(path: str):
    with open(path) as f:
        table = json.load(f)
    for prec, buckets in table["buckets"].items():
        for b, e in buckets.items():
            api.finom_tune_set(prec, int(b), int(e))
    return table


if __name__ == "__main__":
    out = run(path=sys.argv[1] if len(sys.argv) > 1 else None)
    print(json.dumps(out["buckets"]))
    print(json.dumps(out["times_us"]))
