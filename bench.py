#!/usr/bin/env python3
"""Benchmark of the FINOM hot path: Sinkhorn iterations on the 1D large graded mesh.

Workload: N = M = 2^20 graded meshes (x_i = ((i+1/2)/N)^2, tanh-stretched y,
stretch 3), three-component Gaussian mixtures, eps = 1e-3, FP32 log-domain
scans.  One step = one Sinkhorn iteration (K^T phi half step with the fused
divide and marginal-error check, then the K psi half step): 2^21
point-iterations.  L2 is flushed (256 MB write) before every timed step, and
each step is timed with CUDA events on the launching stream.

Unless `--no-sub`, the default line also carries bounded sub-results: `serve`
(the first 100 arrivals of the serving workload), `batch` (the batch workload),
`small_fp64` (the 1000-point float64 workload: time per iteration and its
2000-iteration solve beside the stored oracle solve) and `grid_2d` (the 2D
workload on 1024 x 1024 grids: 10 timed steps and one end-to-end solve).

`--workload batch` times batches of independent 1D instances (4096 instances,
N = M log-uniform in [256, 65536], clustered meshes, eps log-uniform in
[1e-3, 1e-2]); one step = one iteration of every instance (four launches).

`--workload serve` runs the serving loop: Poisson arrivals at 2000 req/s
(the first `--requests` of them), 80 % 1D requests (N log-uniform in
[1e3, 1e6], graded meshes) and 20 % 2D (side log-uniform in [64, 2048],
tanh-clustered axes), eps in {1e-3, 5e-3, 1e-2}, tol 1e-6, FP32 log-domain
with float64 verification; value = solves/s from the first arrival to the
last completion, with p50/p99 latency, beside the plain form (the same kind
of requests one at a time in FP64).

`--workload 2d` times the 2D path instead (Algorithm 2 with the Appendix A
stabilisation): 1024 x 1024 grids, tanh-clustered axes, four anisotropic
Gaussians, eps = 2e-3; one step = one iteration = four axis passes of the
half-step kernel and two tiled transposes, 2 * 1024^2 point-iterations.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
(serial float64 FINOM recurrences in plain C) on the same workload instead.
Under torchrun every rank runs its own replica of the workload (weak
scaling); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "point-iters/s (K·v) vs HBM roofline; served solves/s, p99 at W1 relerr≤1e-4"
UNIT = "point-iters/s"
FALLBACK_HBM_GBS = 6800.0
PROFILE_MD = os.path.join(ROOT, "profiles", "k_half_graded_1d_2e20.md")
KERNEL_SOURCES = ["paper_2605_26659_gb300/csrc/half.cuh", "paper_2605_26659_gb300/csrc/dev_common.cuh"]
# algorithmic bytes of one kernel application per merged point (N = M): x 8,
# y 8, input potentials 8, reference potentials 8, masses 4, new potentials 8
# per output point, i.e. 44 N bytes = 22 B per merged point
ALG_BYTES_PER_POINT = 22.0
GOLDEN_C2 = os.path.join(ROOT, "tests", "golden", "full_config2.json")
GOLDEN_C1 = os.path.join(ROOT, "tests", "golden", "full_config1.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["finom", "reference"], default="finom")
    ap.add_argument("--n", "--mesh-points", dest="n", type=int, default=1 << 20, help="points per mesh (default 2^20)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--workload", choices=["1d", "2d", "batch", "serve", "small"], default="1d")
    ap.add_argument("--requests", type=int, default=200, help="serve: requests of the arrival process")
    ap.add_argument("--slots", type=int, default=64, help="serve: concurrent solves (streams)")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="serve: device memory for active solves")
    ap.add_argument("--policy", choices=["fifo", "smallest"], default="smallest",
                    help="serve: admission order of queued requests")
    ap.add_argument("--rates", type=str, default="",
                    help="serve: extra arrival rates (req/s, comma-separated) for a latency-vs-load sweep")
    ap.add_argument("--batch-points", type=int, default=1 << 16,
                    help="serve: 1D requests with N + M up to this are batched (0: every request alone)")
    ap.add_argument("--eps-stages", type=int, default=0,
                    help="serve: eps-scaling stages of the second run (0: no second run)")
    ap.add_argument("--count", type=int, default=4096, help="batch: instances (default 4096)")
    ap.add_argument("--e2e-count", type=int, default=512, help="batch: instances of the end-to-end solve")
    ap.add_argument("--plain-count", type=int, default=16,
                    help="batch: instances solved one at a time in FP64 for the plain-form comparison")
    ap.add_argument("--side", type=int, default=1024, help="2D grid side (default 1024)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="1d: skip the served and batched sub-results of the default line")
    return ap.parse_args()


def kernel_sha():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    try:
        txt = open(PROFILE_MD).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s*;\s*kernel_sha:\s*([0-9a-f]+)", txt)
    if not m or m.group(2) != kernel_sha():
        return None
    return float(m.group(1))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    """One process per GPU under torchrun: NCCL on GPUs; gloo where no GPU is
    visible (the host-side logic of the multi-rank path, tested on CPU)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def max_over_ranks(v, ws):
    """The maximum of v over the ranks (every rank gets it)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_baseline(pr, budget_s=12.0):
    """The CPU oracle (serial C FINOM, float64) on a bounded sample: whole
    Sinkhorn iterations on the full-size meshes, one core."""
    from oracle import serial_c
    serial_c.lib()
    t0 = time.perf_counter()
    serial_c.sinkhorn(pr.x, pr.y, pr.u, pr.v, pr.eps, 0.0, 1)
    t1 = time.perf_counter() - t0
    iters = max(1, min(200, int(budget_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    serial_c.sinkhorn(pr.x, pr.y, pr.u, pr.v, pr.eps, 0.0, iters)
    dt = time.perf_counter() - t0
    # the oracle computes the loop-head check once per completed iteration + once at exit
    return {"value": (len(pr.x) + len(pr.y)) * iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{iters} Sinkhorn iterations of the serial C float64 FINOM oracle on the full "
                      f"N=M={len(pr.x)} graded meshes ({dt:.1f} s)"}


def cpu_baseline_2d(pr, budget_s=12.0):
    """The CPU oracle on the 2D workload: whole Sinkhorn iterations (line-by-line
    float64 FINOM in plain C), one core."""
    from oracle import serial_c
    serial_c.lib()
    t0 = time.perf_counter()
    serial_c.sinkhorn2d(pr.x1, pr.y1, pr.x2, pr.y2, pr.U, pr.V, pr.eps, 0.0, 1)
    t1 = time.perf_counter() - t0
    iters = max(1, min(50, int(budget_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    serial_c.sinkhorn2d(pr.x1, pr.y1, pr.x2, pr.y2, pr.U, pr.V, pr.eps, 0.0, iters)
    dt = time.perf_counter() - t0
    n = pr.U.size + pr.V.size
    return {"value": n * iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{iters} Sinkhorn iterations of the serial C float64 2D oracle on the full "
                      f"{pr.U.shape[0]}x{pr.U.shape[1]} grids ({dt:.1f} s)"}


def config_1d(N, M, eps, ws):
    return {"workload": f"1D graded meshes N=M={N} (x=((i+1/2)/N)^2, tanh-stretched y, stretch 3), "
                        f"3-Gaussian mixtures, eps=1e-3, FP32 log-domain; 1 Sinkhorn iteration per step",
            "N": N, "M": M, "eps": eps, "point_iters_per_step": N + M,
            "l2": "flushed before every timed step (256 MB write)", "parallelism": f"replicas x{ws}"}


def config_2d(N, M, eps, ws):
    return {"workload": f"2D grids {N}x{M} (tanh-clustered axes, stretch 2.5), 4 anisotropic "
                        f"Gaussians, eps=2e-3, FP32 log-domain; 1 Sinkhorn iteration per step",
            "N": N, "M": M, "eps": eps, "point_iters_per_step": 2 * N * M,
            "l2": "flushed before every timed step (256 MB write)", "parallelism": f"replicas x{ws}"}


def _sample_stride(t_full, steps, warmup, budget_s=150.0, power=1):
    """Smallest power-of-two stride s with (steps + warmup) iterations of the
    strided sample (t_full / s^power each) inside the time budget."""
    s = 1
    while (steps + warmup) * t_full / s ** power > budget_s and s < 1 << 12:
        s *= 2
    return s


def run_reference(args, ws, rank):
    """The oracle on the host cores, on this arm's workload and config: each
    step is one Sinkhorn iteration of the serial C float64 oracle on a strided
    sample of the meshes (every s-th point, masses renormalised; s the
    smallest power of two that keeps the whole run within a few minutes),
    reported per point-iteration."""
    if rank != 0:
        return
    import numpy as np
    if args.workload == "2d":
        return run_reference_2d(args)
    from paper_2605_26659_gb300 import inputs
    pr = inputs.config2(args.n)
    from oracle import serial_c
    serial_c.lib()
    t0 = time.perf_counter()
    f, g, _, _ = serial_c.sinkhorn(pr.x, pr.y, pr.u, pr.v, pr.eps, 0.0, 1)
    t_full = time.perf_counter() - t0
    st = _sample_stride(t_full, args.steps, args.warmup)
    x, y = pr.x[::st], pr.y[::st]
    u, v = pr.u[::st] / pr.u[::st].sum(), pr.v[::st] / pr.v[::st].sum()
    f, g, _, _ = serial_c.sinkhorn(x, y, u, v, pr.eps, 0.0, 0)
    for _ in range(args.warmup):
        f, g, _, _ = serial_c.sinkhorn(x, y, u, v, pr.eps, 0.0, 1, f0=f, g0=g)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, g, _, _ = serial_c.sinkhorn(x, y, u, v, pr.eps, 0.0, 1, f0=f, g0=g)
    dt = time.perf_counter() - t0
    val = (len(x) + len(y)) * args.steps / dt
    sample = (f"{args.steps} Sinkhorn iterations of the serial C float64 oracle on every {st}-th point of the "
              f"N=M={args.n} graded meshes ({len(x)}+{len(y)} points, {dt:.1f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "gpu_launches": 0, "config": config_1d(args.n, args.n, pr.eps, 1),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_2d(args):
    from paper_2605_26659_gb300 import inputs
    from oracle import serial_c
    pr = inputs.config3(args.side)
    serial_c.lib()
    t0 = time.perf_counter()
    serial_c.sinkhorn2d(pr.x1, pr.y1, pr.x2, pr.y2, pr.U, pr.V, pr.eps, 0.0, 1)
    t_full = time.perf_counter() - t0
    st = _sample_stride(t_full, args.steps, args.warmup, power=2)
    x1, y1, x2, y2 = pr.x1[::st], pr.y1[::st], pr.x2[::st], pr.y2[::st]
    U, V = pr.U[::st, ::st], pr.V[::st, ::st]
    U, V = U / U.sum(), V / V.sum()
    A, B, _, _ = serial_c.sinkhorn2d(x1, y1, x2, y2, U, V, pr.eps, 0.0, 0)
    for _ in range(args.warmup):
        A, B, _, _ = serial_c.sinkhorn2d(x1, y1, x2, y2, U, V, pr.eps, 0.0, 1, A, B)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        A, B, _, _ = serial_c.sinkhorn2d(x1, y1, x2, y2, U, V, pr.eps, 0.0, 1, A, B)
    dt = time.perf_counter() - t0
    n = U.size + V.size
    val = n * args.steps / dt
    sample = (f"{args.steps} Sinkhorn iterations of the serial C float64 2D oracle on every {st}-th grid line "
              f"of the {args.side}x{args.side} grids ({U.shape[0]}x{U.shape[1]}, {dt:.1f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "gpu_launches": 0, "config": config_2d(args.side, args.side, pr.eps, 1),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(api, plan, args, stream, dev, ws):
    """W untimed steps, then K steps each after a 256 MB L2 flush, each timed
    with CUDA events on the launching stream; clocks sampled meanwhile."""
    import torch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        flush.zero_()
        api.finom_solve_step(plan, 1, stream=stream)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    for s_ev, e_ev in evs:
        flush.zero_()
        s_ev.record(stream)
        api.finom_solve_step(plan, 1, stream=stream)
        e_ev.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    times = [s.elapsed_time(e) for s, e in evs]
    return float(sum(times)), clocks


def run_finom_2d(args, ws, rank, local, emit=True):
    import torch

    from paper_2605_26659_gb300 import api, inputs
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    api.load()
    pr = inputs.config3(args.side)
    N, M = pr.U.shape
    NM = N * M
    flat = lambda G: G.ravel(order="F")
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = api.finom_plan_2d(T(pr.x1), T(pr.x2), T(pr.y1), T(pr.y2), pr.eps, "f32_log", stream=stream)
    api.finom_solve_begin(plan, T(flat(pr.U)), T(flat(pr.V)), 0.0, 1 << 40, stream=stream)
    total_ms, clocks = timed_steps(api, plan, args, stream, dev, ws)
    done, iters = api.finom_solve_poll(plan, stream=stream)
    assert not done and iters == args.warmup + args.steps + 1, (done, iters)
    total_ms = max_over_ranks(total_ms, ws)
    step_s = total_ms / 1e3 / args.steps
    pts = 2 * NM
    value = ws * pts * args.steps / (total_ms / 1e3)
    # algorithmic bytes per application: 36 B per grid point (potentials in,
    # reference and out 8 + 8 + 8, mass 4, a 4-byte intermediate written and
    # read 8); two applications per step.  The path itself moves more: level
    # pairs of 8 B, 16 B + 16 B of transpose and 32 B of division pass.
    bytes_per_step = 2 * 36.0 * NM
    peak, peak_kind = peaks()
    achieved = bytes_per_step / step_s / 1e9

    e2e = None
    if args.e2e_steps > 0:
        hs = [torch.tensor(a, dtype=torch.float64).pin_memory()
              for a in (pr.x1, pr.x2, pr.y1, pr.y2, flat(pr.U), flat(pr.V))]
        hf = torch.empty(NM, dtype=torch.float64).pin_memory()
        hg = torch.empty(NM, dtype=torch.float64).pin_memory()
        done_pts, secs = 0, 0.0
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dx1, dx2, dy1, dy2, du, dv = (t.to(dev, non_blocking=True) for t in hs)
            p2 = api.finom_plan_2d(dx1, dx2, dy1, dy2, pr.eps, "f32_log", stream=stream)
            f, g, res = api.finom_solve(p2, du, dv, pr.tol, 200000, stream=stream)
            hf.copy_(f, non_blocking=True)
            hg.copy_(g, non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            api.finom_plan_destroy(p2)
            if k > 0:
                done_pts += pts * res["iters"]
                secs += dt
        e2e = {"value": ws * done_pts / secs, "unit": UNIT,
               "h2d_bytes_per_step": 8 * (2 * N + 2 * M + 2 * NM), "d2h_bytes_per_step": 8 * 2 * NM,
               "solve_iters": res["iters"], "converged": res["converged"],
               "marginal_err": res["marginal_err"], "w1": res["w1"], "seconds_per_solve": secs / args.e2e_steps}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_2d(pr)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_2d(N, M, pr.eps, ws),
            "gpu_launches": 6 * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "the whole 2D step: finom::k_half axis passes (4) + k_rot transposes (2)",
                         "algorithmic_bytes_per_step": bytes_per_step},
            "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
        }
        if emit:
            print(json.dumps(line), flush=True)
        api.finom_plan_destroy(plan)
        return line
    api.finom_plan_destroy(plan)
    return None


def run_small(dev, stream):
    """The 1000-point float64 workload (N = M = 1000, eps = 1e-2, tol 1e-9,
    2000 iterations): time per iteration of the stepwise loop (CUDA events
    over 512 iterations after 64), and the blocking solve beside the stored
    float64 oracle solve of the same problem."""
    import torch
    from paper_2605_26659_gb300 import api, inputs
    pr = inputs.config1()
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    p = api.finom_plan(T(pr.x), T(pr.y), pr.eps, "f64", stream=stream)
    elems = api.finom_plan_elems(p)[0]
    api.finom_solve_begin(p, T(pr.u), T(pr.v), 0.0, 1 << 40, stream=stream)
    api.finom_solve_step(p, 64, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    api.finom_solve_step(p, 512, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    us_iter = e0.elapsed_time(e1) * 1e3 / 512
    u, v = T(pr.u), T(pr.v)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f, g, res = api.finom_solve(p, u, v, pr.tol, pr.maxit, stream=stream)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    api.finom_plan_destroy(p)
    out = {"value": us_iter, "unit": "us/iteration", "dtype": "f64", "tile_kind": elems,
           "solve": {"seconds": secs, "iters": res["iters"], "w1": res["w1"], "marginal_err": res["marginal_err"]},
           "config": {"workload": pr.name + f", tol {pr.tol:g}, maxit {pr.maxit}"}}
    try:
        gold = json.load(open(GOLDEN_C1))
        out["solve"]["oracle"] = {"w1": gold["w1"], "iters": gold["iters"], "marginal_err": gold["marginal_err"],
                                  "w1_relerr": abs(res["w1"] - gold["w1"]) / abs(gold["w1"]),
                                  "source": "tests/golden/full_config1.json (serial C float64 FINOM oracle)"}
    except (OSError, KeyError, ValueError):
        pass
    return out


def run_finom_small(args, ws, rank, local):
    """The 1000-point float64 workload alone, as its own line: point-iters/s
    of the stepwise loop (its us per iteration from run_small)."""
    import torch
    from paper_2605_26659_gb300 import api
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    api.load()
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 1)):
        run_small(dev, stream)
    small = run_small(dev, stream)
    if rank == 0:
        us = small["value"]
        line = {"metric": METRIC, "value": ws * 2000 / (us * 1e-6), "unit": UNIT, "n_gpus": ws, "steps": 512,
                "warmup": max(args.warmup, 1), "ms_per_step": us * 1e-3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": small["config"]["workload"], "parallelism": f"replicas x{ws}",
                           "l2": "resident (88 KB of inputs; latency-bound)", "tile_kind": small["tile_kind"]},
                "gpu_launches": 2 * 512, "roofline": None, "small_fp64": small}
        print(json.dumps(line), flush=True)


def _concat_batch(probs):
    import numpy as np
    offx = np.concatenate([[0], np.cumsum([len(q.x) for q in probs])]).astype(np.int64)
    offy = np.concatenate([[0], np.cumsum([len(q.y) for q in probs])]).astype(np.int64)
    cat = lambda k: np.concatenate([getattr(q, k) for q in probs])
    return cat("x"), cat("y"), cat("u"), cat("v"), offx, offy, [q.eps for q in probs]


def run_finom_batch(args, ws, rank, local, emit=True):
    import torch

    from paper_2605_26659_gb300 import api, inputs
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    api.load()
    probs = inputs.config4(args.count)
    x, y, u, v, offx, offy, eps = _concat_batch(probs)
    L = len(x) + len(y)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = api.finom_plan_batch(T(x), offx, T(y), offy, eps, "f32_log", stream=stream)
    api.finom_solve_batch_begin(plan, T(u), T(v), 0.0, 1 << 30, stream=stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        flush.zero_()
        api.finom_solve_batch_step(plan, 1, stream=stream)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    for s_ev, e_ev in evs:
        flush.zero_()
        s_ev.record(stream)
        api.finom_solve_batch_step(plan, 1, stream=stream)
        e_ev.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    total_ms = max_over_ranks(float(sum(s.elapsed_time(e) for s, e in evs)), ws)
    step_s = total_ms / 1e3 / args.steps
    value = ws * L * args.steps / (total_ms / 1e3)
    bytes_per_step = 2 * ALG_BYTES_PER_POINT * L   # two half steps
    peak, peak_kind = peaks()
    achieved = bytes_per_step / step_s / 1e9
    api.finom_plan_destroy(plan)

    # end to end: a sub-batch solved to tol 1e-6 from host buffers (FP32, float64
    # verified) against the plain form: the same instances one at a time in FP64
    e2e = None
    if args.e2e_steps > 0:
        sub = probs[:args.e2e_count]
        sx, sy, su, sv, soffx, soffy, seps = _concat_batch(sub)
        hs = [torch.tensor(a, dtype=torch.float64).pin_memory() for a in (sx, sy, su, sv)]
        hf = torch.empty(len(sx), dtype=torch.float64).pin_memory()
        hg = torch.empty(len(sy), dtype=torch.float64).pin_memory()
        times = []
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dx, dy, du, dv = (t.to(dev, non_blocking=True) for t in hs)
            pb = api.finom_plan_batch(dx, soffx, dy, soffy, seps, "f32_log", stream=stream)
            f, g, res = api.finom_solve_batch(pb, du, dv, 1e-6, 100000, stream=stream)
            hf.copy_(f, non_blocking=True)
            hg.copy_(g, non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            api.finom_plan_destroy(pb)
            if k > 0:
                times.append(dt)
        secs = sum(times) / len(times)
        pts = sum((len(q.x) + len(q.y)) * r["iters"] for q, r in zip(sub, res))
        nconv = sum(r["converged"] for r in res)
        # the plain form, a sample of the same instances
        plain = []
        for q in sub[:args.plain_count]:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p1 = api.finom_plan(T(q.x), T(q.y), q.eps, "f64", stream=stream)
            _, _, r1 = api.finom_solve(p1, T(q.u), T(q.v), 1e-6, 100000, stream=stream)
            torch.cuda.synchronize()
            plain.append(time.perf_counter() - t0)
            api.finom_plan_destroy(p1)
        plain_per_solve = sum(plain) / len(plain)
        e2e = {"value": ws * pts / secs, "unit": UNIT,
               "h2d_bytes_per_step": 8 * (2 * len(sx) + 2 * len(sy)), "d2h_bytes_per_step": 8 * (len(sx) + len(sy)),
               "instances": len(sub), "converged": int(nconv), "seconds_per_batch": secs,
               "solves_per_s": len(sub) / secs,
               "plain_fp64_one_at_a_time": {"solves_per_s": 1.0 / plain_per_solve, "sample": len(plain),
                                            "seconds_per_solve": plain_per_solve}}
    cpu = None
    if emit and rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_batch(probs)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched 1D instances: {len(probs)} problems, N = M log-uniform in "
                                   f"[256, 65536], clustered meshes, Dirichlet-perturbed mixtures, eps "
                                   f"log-uniform in [1e-3, 1e-2], FP32 log-domain; 1 iteration of every "
                                   f"instance per step", "instances": len(probs), "merged_points": L,
                       "l2": "flushed before every timed step (256 MB write)", "parallelism": f"replicas x{ws}"},
            "gpu_launches": 6 * args.steps,   # per iteration: 2 half steps, 2 instance ends, 2 compactions
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "finom::k_half<float, kBatchY|kBatchX> + k_batch_end + k_batch_compact",
                         "algorithmic_bytes_per_step": bytes_per_step},
            "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
        }
        if emit:
            print(json.dumps(line), flush=True)
        return line
    return None


def _submit_request(srv, pr):
    if hasattr(pr, "x"):
        return srv.submit_1d(pr.x, pr.y, pr.u, pr.v, pr.eps, pr.tol, pr.maxit)
    return srv.submit_2d(pr.x1, pr.x2, pr.y1, pr.y2, pr.U, pr.V, pr.eps, pr.tol, pr.maxit)


def _request_points(pr):
    return len(pr.x) + len(pr.y) if hasattr(pr, "x") else 2 * pr.U.size


def _serve_once(api, args, reqs, probs, stages):
    """Submit the requests at their arrival times to a fresh server, step it
    until every request has finished; returns (wall seconds, results in
    request order, peak active solves)."""
    srv = api.Server(int(args.budget_gb * 2**30), max_active=args.slots, precision="f32_log")
    srv.set_policy(args.policy)
    srv.set_batching(args.batch_points)
    if stages:
        srv.set_eps_scaling(stages, 0.5, 1e-4)
    t0 = time.perf_counter()
    nxt, ids, done, peak_active = 0, {}, {}, 0
    while len(done) < len(probs):
        now = time.perf_counter() - t0
        while nxt < len(probs) and reqs[nxt].t_arrival <= now:
            ids[_submit_request(srv, probs[nxt])] = nxt
            nxt += 1
        pend, act, fin = srv.step()
        peak_active = max(peak_active, act)
        if fin:
            for rid in [r for r in ids if ids[r] not in done]:
                got = srv.result(rid)
                if got is not None:
                    done[ids[rid]] = got[0]
    wall = time.perf_counter() - t0
    srv.close()
    return wall, [done[k] for k in range(len(probs))], peak_active


def run_finom_serve(args, ws, rank, local, emit=True):
    """Served solves/s and latency of the serving loop on the arrival process."""
    import numpy as np
    import torch

    from paper_2605_26659_gb300 import api, inputs
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    api.load()
    reqs = inputs.serving_requests()[:args.requests]
    probs = [inputs.request_problem(r) for r in reqs]
    n1d = sum(1 for r in reqs if r.kind == "1d")
    # warm-up: a few small solves (plans, graphs, kernels loaded)
    srv = api.Server(int(args.budget_gb * 2**30), max_active=args.slots, precision="f32_log")
    warm = [q for q in probs if _request_points(q) < 200000][:max(args.warmup, 1)]
    srv.run([_submit_request(srv, q) for q in warm])
    srv.close()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    wall, res, peak_active = _serve_once(api, args, reqs, probs, 0)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    wall = max_over_ranks(wall, ws)
    lat = np.array([r["latency_s"] for r in res])
    que = np.array([r["queue_s"] for r in res])
    nconv = sum(r["converged"] for r in res)
    pts = sum(_request_points(q) * r["iters"] for q, r in zip(probs, res))
    # latency against load: the same kinds of requests at other arrival rates
    sweep = None
    if args.rates:
        sweep = {}
        for rate in [float(r) for r in args.rates.split(",") if r]:
            rq = inputs.serving_requests(rate=rate, duration=2.0 * args.requests / rate + 1.0)[:args.requests]
            pb = [inputs.request_problem(r) for r in rq]
            w, rs, pk = _serve_once(api, args, rq, pb, 0)
            lt = np.array([r["latency_s"] for r in rs])
            sweep[str(rate)] = {"solves_per_s": len(pb) / w, "p50_s": float(np.percentile(lt, 50)),
                                "p99_s": float(np.percentile(lt, 99)), "arrival_span_s": rq[-1].t_arrival,
                                "peak_active": pk, "converged": int(sum(r["converged"] for r in rs))}
    # the same arrivals with eps scaling in the server (same fixed points)
    scaled = None
    if args.eps_stages > 0:
        wall2, res2, _ = _serve_once(api, args, reqs, probs, args.eps_stages)
        lat2 = np.array([r["latency_s"] for r in res2])
        w1d = [abs(a["w1"] - b["w1"]) / abs(a["w1"]) for a, b in zip(res, res2) if a["converged"] and b["converged"]]
        scaled = {"solves_per_s": ws * len(probs) / wall2, "stages": args.eps_stages, "factor": 0.5,
                  "tol_stage": 1e-4, "converged": int(sum(r["converged"] for r in res2)),
                  "latency_s": {"p50": float(np.percentile(lat2, 50)), "p99": float(np.percentile(lat2, 99))},
                  "iterations": int(sum(r["iters"] for r in res2)),
                  "iterations_plain": int(sum(r["iters"] for r in res)),
                  "w1_max_relerr_vs_plain_served": max(w1d) if w1d else None}
    solves_per_s = ws * len(probs) / wall
    h2d = sum(8 * (2 * (len(q.x) + len(q.y)) if hasattr(q, "x") else 2 * (q.U.size + len(q.x1) + len(q.y1)))
              for q in probs)
    launches = sum(r["iters"] * (2 if hasattr(q, "x") else 4) for q, r in zip(probs, res))
    d2h = sum(8 * _request_points(q) for q in probs)
    # the plain form: requests of the same process, one at a time, FP64, from host arrays
    T = lambda a: torch.tensor(np.asarray(a).ravel(order="F"), dtype=torch.float64, device=dev)
    plain, w1_dev = [], []
    stream = torch.cuda.current_stream(dev)
    for k, q in enumerate(probs[:args.plain_count]):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if hasattr(q, "x"):
            p1 = api.finom_plan(T(q.x), T(q.y), q.eps, "f64", stream=stream)
            f1, g1, r1 = api.finom_solve(p1, T(q.u), T(q.v), q.tol, q.maxit, stream=stream)
        else:
            p1 = api.finom_plan_2d(T(q.x1), T(q.x2), T(q.y1), T(q.y2), q.eps, "f64", stream=stream)
            f1, g1, r1 = api.finom_solve(p1, T(q.U), T(q.V), q.tol, q.maxit, stream=stream)
        f1.cpu(), g1.cpu()
        torch.cuda.synchronize()
        plain.append(time.perf_counter() - t1)
        api.finom_plan_destroy(p1)
        if r1["converged"] and res[k]["converged"]:
            w1_dev.append(abs(res[k]["w1"] - r1["w1"]) / abs(r1["w1"]))
    plain_per_solve = sum(plain) / len(plain)
    peak, peak_kind = peaks()
    # algorithmic bytes of every application served: 22 B per merged point
    # (1D), 36 B per grid point (2D), two applications per iteration
    alg = sum(r["iters"] * (2 * ALG_BYTES_PER_POINT * (len(q.x) + len(q.y)) if hasattr(q, "x") else 72.0 * q.U.size)
              for q, r in zip(probs, res))
    achieved = alg / wall / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": solves_per_s, "unit": "solves/s", "n_gpus": ws,
            "steps": len(probs), "warmup": len(warm), "ms_per_step": 1e3 * wall / len(probs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"serving loop: the first {len(probs)} requests of Poisson arrivals at "
                                   f"2000 req/s, {n1d} 1D (N log-uniform in [1e3, 1e6], graded meshes) and "
                                   f"{len(probs) - n1d} 2D (side log-uniform in [64, 2048], tanh-clustered "
                                   f"axes), eps in {{1e-3, 5e-3, 1e-2}}, tol 1e-6, maxit 10000, FP32 "
                                   f"log-domain with float64 verification; one step = one request",
                       "slots": args.slots, "budget_gb": args.budget_gb, "peak_active": peak_active,
                       "batch_points": args.batch_points,
                       "policy": args.policy,
                       "l2": "inputs and potentials of the active solves exceed L2",
                       "parallelism": f"replicas x{ws}"},
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max()), "queue_p50": float(np.percentile(que, 50)),
                          "queue_p99": float(np.percentile(que, 99))},
            "converged": int(nconv), "point_iters_per_s": pts / wall,
            "gpu_launches": launches,
            "gpu_launches_note": "half-step launches if every request ran alone (2 per 1D iteration, 4 per 2D); "
                                 "batched 1D requests share theirs, so this is an upper bound",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "every k_half launch of the served solves, over the wall time",
                         "algorithmic_bytes": alg},
            "clocks": clocks,
            "e2e": {"value": solves_per_s, "unit": "solves/s", "h2d_bytes_per_step": h2d / len(probs),
                    "d2h_bytes_per_step": d2h / len(probs)},
            "plain_fp64_one_at_a_time": {"solves_per_s": 1.0 / plain_per_solve, "sample": len(plain),
                                         "seconds_per_solve": plain_per_solve,
                                         "w1_max_relerr_served_vs_plain": max(w1_dev) if w1_dev else None},
            "eps_scaling": scaled,
            "rate_sweep": sweep,
            "cpu_baseline": None,
        }
        if emit:
            print(json.dumps(line), flush=True)
        return line
    return None


def cpu_baseline_batch(probs, budget_s=12.0):
    """The CPU oracle on instances of the batch, one instance per host thread
    (the serial C oracle runs outside the GIL), until the time budget is spent."""
    import concurrent.futures as cf

    from oracle import serial_c
    serial_c.lib()
    cores = max(1, os.cpu_count() or 1)
    t0 = time.perf_counter()

    def one(q):
        if time.perf_counter() - t0 > budget_s:
            return 0
        _, _, it, _ = serial_c.sinkhorn(q.x, q.y, q.u, q.v, q.eps, 0.0, 20)
        return (len(q.x) + len(q.y)) * it

    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        done = [p for p in ex.map(one, probs) if p > 0]
    dt = time.perf_counter() - t0
    return {"value": sum(done) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"20 Sinkhorn iterations of each of the first {len(done)} instances, serial C float64 "
                      f"oracle, one instance per thread on {cores} threads ({dt:.1f} s)"}


def run_finom(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_2605_26659_gb300 import api, inputs
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    api.load()
    pr = inputs.config2(args.n)
    N, M = len(pr.x), len(pr.y)
    L = N + M
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    x, y, u, v = T(pr.x), T(pr.y), T(pr.u), T(pr.v)
    stream = torch.cuda.current_stream(dev)
    plan = api.finom_plan(x, y, pr.eps, "f32_log", stream=stream)
    api.finom_solve_begin(plan, u, v, 0.0, 1 << 40, stream=stream)
    total_ms, clocks = timed_steps(api, plan, args, stream, dev, ws)
    done, iters = api.finom_solve_poll(plan, stream=stream)
    assert not done and iters == args.warmup + args.steps + 1, (done, iters)
    total_ms = max_over_ranks(total_ms, ws)
    step_s = total_ms / 1e3 / args.steps
    value = ws * L * args.steps / (total_ms / 1e3)

    # roofline of the dominant kernel (the half step; two launches per step)
    bytes_per_launch = ALG_BYTES_PER_POINT * L
    peak, peak_kind = peaks()
    achieved = bytes_per_launch / (step_s / 2) / 1e9
    traffic = profiled_traffic()

    # end to end through the public API with host buffers: copy the inputs in,
    # plan, solve to the workload's tolerance, read the potentials back
    e2e = None
    if args.e2e_steps > 0:
        hx, hy, hu, hv = (torch.tensor(a, dtype=torch.float64).pin_memory() for a in (pr.x, pr.y, pr.u, pr.v))
        hf = torch.empty(N, dtype=torch.float64).pin_memory()
        hg = torch.empty(M, dtype=torch.float64).pin_memory()
        pts, secs = 0, 0.0
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dx, dy, du, dv = (t.to(dev, non_blocking=True) for t in (hx, hy, hu, hv))
            p2 = api.finom_plan(dx, dy, pr.eps, "f32_log", stream=stream)
            f, g, res = api.finom_solve(p2, du, dv, pr.tol, 60000, stream=stream)
            hf.copy_(f, non_blocking=True)
            hg.copy_(g, non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            api.finom_plan_destroy(p2)
            if k > 0:   # the first call is a warm-up
                pts += L * res["iters"]
                secs += dt
        e2e = {"value": ws * pts / secs, "unit": UNIT, "h2d_bytes_per_step": 8 * (2 * N + 2 * M),
               "d2h_bytes_per_step": 8 * (N + M), "solve_iters": res["iters"], "converged": res["converged"],
               "marginal_err": res["marginal_err"], "w1": res["w1"], "seconds_per_solve": secs / args.e2e_steps}
        # the CPU float64 oracle's full solve of the same workload (stored by
        # tests/golden/make_full_size.py, which calls only the oracle)
        try:
            gold = json.load(open(GOLDEN_C2))
            if gold["N"] == N and gold["M"] == M:
                e2e["oracle"] = {"w1": gold["w1"], "iters": gold["iters"], "marginal_err": gold["marginal_err"],
                                 "w1_relerr": abs(res["w1"] - gold["w1"]) / abs(gold["w1"]),
                                 "source": "tests/golden/full_config2.json (serial C float64 FINOM oracle)"}
        except (OSError, KeyError, ValueError):
            pass

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(pr)

    # the second half of the metric, bounded so that the default run stays
    # short: served solves/s with p50 / p99 on the first arrivals of the
    # serving process, and the batched form, each beside the plain
    # one-at-a-time FP64 form
    serve = batch = small = grid = None
    if not args.no_sub:
        small = run_small(dev, stream)
        sub = argparse.Namespace(**vars(args))
        sub.side, sub.steps, sub.warmup, sub.e2e_steps, sub.no_cpu_baseline = 1024, 10, 3, 1, True
        grid = run_finom_2d(sub, ws, rank, local, emit=False)
        sub = argparse.Namespace(**vars(args))
        sub.requests, sub.plain_count, sub.slots, sub.budget_gb, sub.policy = 100, 4, 64, 64.0, "smallest"
        sub.rates, sub.eps_stages, sub.warmup = "", 0, 3
        serve = run_finom_serve(sub, ws, rank, local, emit=False)
        sub = argparse.Namespace(**vars(args))
        sub.count, sub.e2e_count, sub.plain_count, sub.steps, sub.warmup, sub.e2e_steps = 4096, 512, 8, 10, 3, 1
        batch = run_finom_batch(sub, ws, rank, local, emit=False)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_1d(N, M, pr.eps, ws),
            "gpu_launches": 2 * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "finom::k_half<float, kHalfY|kHalfX, 8> (half steps on absolute levels)",
                         "algorithmic_bytes_per_launch": bytes_per_launch,
                         "algorithmic_bytes_per_merged_point": ALG_BYTES_PER_POINT},
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        if serve is not None:
            line["serve"] = {k: serve[k] for k in ("value", "unit", "steps", "latency_s", "converged",
                                                   "point_iters_per_s", "roofline", "clocks", "e2e",
                                                   "plain_fp64_one_at_a_time", "config")}
            line["serve"]["requests"] = serve["steps"]
        if batch is not None:
            line["batch"] = {k: batch[k] for k in ("value", "unit", "ms_per_step", "roofline", "clocks", "e2e",
                                                   "config")}
        if small is not None:
            line["small_fp64"] = small
        if grid is not None:
            line["grid_2d"] = {k: grid[k] for k in ("value", "unit", "ms_per_step", "roofline", "clocks", "e2e",
                                                    "config")}
        print(json.dumps(line), flush=True)
    api.finom_plan_destroy(plan)


def main():
    args = parse()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "2d":
        run_finom_2d(args, ws, rank, local)
    elif args.workload == "batch":
        run_finom_batch(args, ws, rank, local)
    elif args.workload == "serve":
        run_finom_serve(args, ws, rank, local)
    elif args.workload == "small":
        run_finom_small(args, ws, rank, local)
    else:
        run_finom(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
