"""Autotuner of the kernel's tile size (points per thread) for 1D plans.

`run()` calls the library's native autotuner (finom_autotune) for every size
bucket 2^lo .. 2^hi of both precisions, which times a few Sinkhorn
iterations of a synthetic problem per candidate and installs the fastest in
the library's table; the table is written to a JSON cache.  `apply()` loads
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
