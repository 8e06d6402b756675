"""GPU tests of the serving loop (finom_server_*): continuous batching of 1D
and 2D solves of mixed sizes.

Each served solve runs the arithmetic of finom_solve on its own plan, so a
request's result must be the same (bit for bit) alone and in a mix of
concurrent requests, and must match the CPU oracle's solve of that problem
(W1 relative error <= 1e-4, float64 marginal error <= tol).
"""
import numpy as np
import pytest

from oracle import serial_c
from tests.gpu_util import meshes

pytestmark = pytest.mark.gpu


def _masses(N, M, seed):
    g = np.random.default_rng(seed)
    u = g.uniform(0.05, 1, N)
    v = g.uniform(0.05, 1, M)
    return u / u.sum(), v / v.sum()


def _requests():
    """1D and 2D problems of mixed sizes: (kind, arrays, eps, tol, maxit)."""
    from paper_2605_26659_gb300 import inputs
    out = []
    for k, (N, M, kind, eps) in enumerate([(300, 257, "uniform_random", 0.02), (5000, 3100, "graded", 0.01),
                                           (40, 1, "uniform_random", 0.05), (2049, 2047, "ties", 0.01),
                                           (12000, 12000, "graded", 0.01)]):
        x, y = meshes(kind, N, M, 300 + k)
        u, v = _masses(N, M, 400 + k)
        out.append(("1d", (x, y, u, v), eps, 1e-7, 20000))
    for (N, M) in [(64, 48), (96, 80)]:
        pr = inputs.config3(N, M)
        out.append(("2d", (pr.x1, pr.x2, pr.y1, pr.y2, pr.U, pr.V), pr.eps, 1e-6, 20000))
    return out


def _submit(srv, req):
    kind, a, eps, tol, maxit = req
    if kind == "1d":
        return srv.submit_1d(*a, eps, tol, maxit)
    return srv.submit_2d(*a, eps, tol, maxit)


def _oracle(req):
    kind, a, eps, tol, maxit = req
    if kind == "1d":
        x, y, u, v = a
        fo, go, it, err = serial_c.sinkhorn(x, y, u, v, eps, tol, maxit)
        return serial_c.cost(x, y, eps, fo, go), it
    x1, x2, y1, y2, U, V = a
    Ao, Bo, it, err = serial_c.sinkhorn2d(x1, y1, x2, y2, U, V, eps, tol, maxit)
    return serial_c.cost2d(x1, y1, x2, y2, eps, Ao, Bo), it


def _oracle_err(req, f, g):
    kind, a, eps, tol, maxit = req
    if kind == "1d":
        x, y, u, v = a
        return serial_c.marginal_error(x, y, eps, f, g, v)
    x1, x2, y1, y2, U, V = a
    return serial_c.marginal_error2d(x1, y1, x2, y2, eps, f, g, V)


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_served_alone_equals_in_the_mix_and_matches_oracle(lib, prec):
    reqs = _requests()
    alone = []
    for r in reqs:   # each request on its own server, one slot
        srv = lib.Server(1 << 34, max_active=1, precision=prec)
        rid = _submit(srv, r)
        alone.append(srv.run([rid])[rid])
        srv.close()
    # the mix: every request queued at once, three slots, a 12 MB budget that
    # makes some requests wait for memory (float32: the small 1D requests are
    # batched, float64: each is solved alone)
    srv = lib.Server(12 << 20, max_active=3, precision=prec)
    ids = [_submit(srv, r) for r in reqs]
    peak_active = 0
    out = {}
    while len(out) < len(ids):
        pend, act, fin = srv.step()
        peak_active = max(peak_active, act)
        assert act <= 3
        for rid in ids:
            if rid not in out:
                got = srv.result(rid)
                if got is not None:
                    out[rid] = got
    srv.close()
    assert peak_active >= 2   # requests overlapped on the GPU
    for r, a, rid in zip(reqs, alone, ids):
        da, fa, ga = a
        dm, fm, gm = out[rid]
        assert da["status"] == dm["status"] == 0
        assert da["converged"] == dm["converged"] == 1, (r[0], da, dm)
        # the same result alone and in the mix, bit for bit
        assert np.array_equal(fa, fm) and np.array_equal(ga, gm)
        assert da["iters"] == dm["iters"] and da["w1"] == dm["w1"]
        assert da["marginal_err"] == dm["marginal_err"]
        # and the oracle's
        w1o, ito = _oracle(r)
        assert dm["w1"] == pytest.approx(w1o, rel=1e-4 if prec == "f32_log" else 1e-9)
        if prec == "f64" and min(np.size(r[1][0]), np.size(r[1][1])) > 1:
            assert dm["iters"] == ito
        e_or = _oracle_err(r, fm, gm)
        assert e_or <= r[3] * (1 + 1e-6) + 1e-15
        assert dm["marginal_err"] == pytest.approx(e_or, rel=1e-6, abs=1e-13)
        assert dm["latency_s"] >= dm["queue_s"] >= 0.0


def test_served_solve_equals_blocking_solve(lib):
    """A served FP64 solve gives what finom_solve gives on the same inputs."""
    from tests.gpu_util import T, H
    x, y = meshes("graded", 3000, 2500, 7)
    u, v = _masses(3000, 2500, 8)
    srv = lib.Server(1 << 30, max_active=2, precision="f64")
    rid = srv.submit_1d(x, y, u, v, 0.01, 1e-9, 5000)
    d, f, g = srv.run([rid])[rid]
    srv.close()
    p = lib.finom_plan(T(x), T(y), 0.01, "f64")
    fb, gb, rb = lib.finom_solve(p, T(u), T(v), 1e-9, 5000)
    assert d["iters"] == rb["iters"] and d["converged"] == rb["converged"] == 1
    assert np.max(np.abs(f - H(fb))) <= 1e-12 * 0.01 and d["w1"] == pytest.approx(rb["w1"], rel=1e-13)


def test_admission_by_footprint_and_slots(lib):
    reqs = _requests()[:4]
    # a budget below every footprint: one solve at a time (an idle server
    # still admits the queue head)
    srv = lib.Server(1, max_active=4, precision="f32_log")
    ids = [_submit(srv, r) for r in reqs]
    done = {}
    while len(done) < len(ids):
        pend, act, fin = srv.step()
        assert act <= 1
        for rid in ids:
            if rid not in done:
                got = srv.result(rid)
                if got is not None:
                    done[rid] = got
    srv.close()
    # one at a time, first come first served: each request is admitted after
    # its predecessor has finished
    d = [done[rid][0] for rid in ids]
    assert all(x["converged"] == 1 for x in d)
    for a, b in zip(d, d[1:]):
        assert b["queue_s"] >= a["latency_s"] - 0.05


def test_bad_request_fails_alone(lib):
    srv = lib.Server(1 << 30, max_active=4, precision="f32_log")
    x, y = meshes("uniform_random", 500, 400, 1)
    u, v = _masses(500, 400, 2)
    good = srv.submit_1d(x, y, u, v, 0.02, 1e-6, 5000)
    bad = srv.submit_1d(x[::-1].copy(), y, u, v, 0.02, 1e-6, 5000)   # unsorted mesh
    neg = srv.submit_1d(x, y, -u, v, 0.02, 1e-6, 5000)               # negative masses
    assert srv.result(good) is None                                    # not finished yet
    out = srv.run([good, bad, neg])
    srv.close()
    assert out[good][0]["status"] == 0 and out[good][0]["converged"] == 1
    assert out[bad][0]["status"] == lib.FINOM_EINVAL
    assert out[neg][0]["status"] == lib.FINOM_EINVAL


def test_cancel_queued_and_active(lib):
    srv = lib.Server(1 << 30, max_active=1, precision="f32_log")
    x, y = meshes("graded", 20000, 20000, 3)
    u, v = _masses(20000, 20000, 4)
    a = srv.submit_1d(x, y, u, v, 0.001, 1e-9, 100000)   # long: still active when cancelled
    b = srv.submit_1d(x, y, u, v, 0.02, 1e-6, 5000)      # queued behind it
    c = srv.submit_1d(x, y, u, v, 0.02, 1e-6, 5000)
    srv.step()
    srv.step()
    srv.cancel(b)
    srv.cancel(a)
    with pytest.raises(lib.FinomError):
        srv.cancel(12345)
    out = srv.run([a, b, c])
    srv.close()
    assert out[a][0]["status"] == lib.FINOM_ECANCELED
    assert out[b][0]["status"] == lib.FINOM_ECANCELED
    assert out[c][0]["status"] == 0 and out[c][0]["converged"] == 1


@pytest.mark.parametrize("prec", ["f64", "f32_log"])
def test_eps_scaling_in_the_server(lib, prec):
    """With eps scaling on, served solves reach the same fixed point (the
    oracle's float64 error of the returned potentials within tol, W1 equal to
    the plain served W1) and results stay the same alone and in the mix."""
    from paper_2605_26659_gb300 import inputs
    pr = inputs.config2(1 << 12)
    reqs = [("1d", (pr.x, pr.y, pr.u, pr.v), pr.eps, 1e-6, 50000)] + _requests()[:2] + _requests()[5:6]
    plain = lib.Server(1 << 32, max_active=4, precision=prec)
    ids = [_submit(plain, r) for r in reqs]
    base = plain.run(ids)
    plain.close()
    mixed = lib.Server(1 << 32, max_active=4, precision=prec)
    mixed.set_eps_scaling(3, 0.5, 1e-4)
    ids2 = [_submit(mixed, r) for r in reqs]
    got = mixed.run(ids2)
    mixed.close()
    for r, i0, i1 in zip(reqs, ids, ids2):
        d0, d1 = base[i0][0], got[i1][0]
        assert d1["status"] == 0 and d1["converged"] == 1, (r[0], d1)
        assert d1["w1"] == pytest.approx(d0["w1"], rel=1e-6 if prec == "f64" else 1e-4)
        assert _oracle_err(r, got[i1][1], got[i1][2]) <= r[3] * (1 + 1e-6) + 1e-15
    # graded mesh at eps = 1e-3: fewer iterations in total with the stages
    assert got[ids2[0]][0]["iters"] < base[ids[0]][0]["iters"]
    alone = lib.Server(1 << 32, max_active=1, precision=prec)
    alone.set_eps_scaling(3, 0.5, 1e-4)
    rid = _submit(alone, reqs[0])
    a = alone.run([rid])[rid]
    alone.close()
    assert np.array_equal(a[1], got[ids2[0]][1]) and a[0]["iters"] == got[ids2[0]][0]["iters"]


def test_smallest_first_admission(lib):
    """One solve at a time: smallest first admits the queued requests by size,
    first come first served by arrival; results are the same either way."""
    reqs = [_requests()[k] for k in (1, 0, 3)]      # 8100, 557, 4096 merged points
    out = {}
    for policy in ("fifo", "smallest"):
        srv = lib.Server(1, max_active=1, precision="f32_log")
        srv.set_policy(policy)
        ids = [_submit(srv, r) for r in reqs]
        res = srv.run(ids)
        out[policy] = [res[i] for i in ids]
        srv.close()
    q = {p: [d[0]["queue_s"] for d in out[p]] for p in out}
    assert q["fifo"][0] < q["fifo"][1] < q["fifo"][2]
    assert q["smallest"][1] < q["smallest"][2] < q["smallest"][0]
    for a, b in zip(out["fifo"], out["smallest"]):
        assert np.array_equal(a[1], b[1]) and a[0]["iters"] == b[0]["iters"]
    srv = lib.Server(1, max_active=1)
    rc = lib._lib.finom_server_set_policy(srv.handle, 7)
    assert rc == lib.FINOM_EINVAL
    srv.close()


def _small_1d(n, seed, eps, kind="uniform_random"):
    x, y = meshes(kind, n, n + 17, seed)
    u, v = _masses(n, n + 17, seed + 1)
    return ("1d", (x, y, u, v), eps, 1e-6, 20000)


@pytest.mark.parametrize("prec", ["f32_log", "f64"])
def test_batched_requests_run_together_and_match_the_oracle(lib, prec):
    """Compatible small 1D requests queued on a one-slot server are admitted
    as one batch (one active solve, admitted at once); each result is the one
    the request gets alone, and the oracle's."""
    reqs = [_small_1d(n, 50 + n, eps) for n, eps in [(900, 0.02), (3000, 0.01), (64, 0.015), (1500, 0.02)]]
    srv = lib.Server(1 << 32, max_active=1, precision=prec)
    srv.set_batching(1 << 16)
    ids = [_submit(srv, r) for r in reqs]
    out, peak = {}, 0
    while len(out) < len(ids):
        pend, act, fin = srv.step()
        peak = max(peak, act)
        for rid in ids:
            if rid not in out:
                got = srv.result(rid)
                if got is not None:
                    out[rid] = got
    srv.close()
    assert peak == 1
    d = [out[rid][0] for rid in ids]
    # one admission for all four: none waited for another to finish
    assert max(x["queue_s"] for x in d) < min(x["latency_s"] for x in d)
    for r, rid in zip(reqs, ids):
        dm, fm, gm = out[rid]
        assert dm["status"] == 0 and dm["converged"] == 1
        srv1 = lib.Server(1 << 32, max_active=1, precision=prec)
        srv1.set_batching(1 << 16)
        k = _submit(srv1, r)
        da, fa, ga = srv1.run([k])[k]
        srv1.close()
        assert np.array_equal(fa, fm) and np.array_equal(ga, gm) and da["iters"] == dm["iters"]
        w1o, ito = _oracle(r)
        assert dm["w1"] == pytest.approx(w1o, rel=1e-4 if prec == "f32_log" else 1e-9)
        if prec == "f64":
            assert dm["iters"] == ito
        e_or = _oracle_err(r, fm, gm)
        assert e_or <= r[3] * (1 + 1e-6) + 1e-15
        assert dm["marginal_err"] == pytest.approx(e_or, rel=1e-6, abs=1e-13)


def test_batching_limit_and_compatibility(lib):
    """Requests above the limit, with another tol, or with eps more than a
    factor 2 apart are not batched together; batching off serves every
    request alone; both give the oracle's fixed point."""
    reqs = [_small_1d(800, 7, 0.01), _small_1d(700, 9, 0.05), _small_1d(5000, 11, 0.01),
            ("1d",) + _small_1d(600, 13, 0.01)[1:3] + (1e-7, 20000)]
    res = {}
    for limit in (4096, 0):
        srv = lib.Server(1 << 32, max_active=1, precision="f32_log")
        srv.set_batching(limit)
        ids = [_submit(srv, r) for r in reqs]
        res[limit] = srv.run(ids)
        res[limit] = [res[limit][i] for i in ids]
        srv.close()
    # with one slot and nothing compatible, each request waits for the one before
    d = [x[0] for x in res[4096]]
    for a, b in zip(d, d[1:]):
        assert b["queue_s"] >= a["latency_s"] - 0.05
    for r, a, b in zip(reqs, res[4096], res[0]):
        assert a[0]["converged"] == b[0]["converged"] == 1
        w1o, _ = _oracle(r)
        assert a[0]["w1"] == pytest.approx(w1o, rel=1e-4) and b[0]["w1"] == pytest.approx(w1o, rel=1e-4)
        assert _oracle_err(r, a[1], a[2]) <= r[3] * (1 + 1e-6) + 1e-15
    srv = lib.Server(1, max_active=1)
    assert lib._lib.finom_server_set_batching(srv.handle, -1) == lib.FINOM_EINVAL
    assert lib._lib.finom_server_set_batching(srv.handle, (1 << 22) + 1) == lib.FINOM_EINVAL
    srv.close()


def test_cancel_batched_requests(lib):
    """Cancelling every request of a running batch stops it early; cancelling
    one of two leaves the other to converge."""
    x, y = meshes("graded", 20000, 20000, 3)
    u, v = _masses(20000, 20000, 4)
    srv = lib.Server(1 << 32, max_active=1, precision="f32_log")
    long_ = [srv.submit_1d(x, y, u, v, 0.001, 1e-9, 100000) for _ in range(3)]   # one batch
    srv.step()
    for rid in long_:
        srv.cancel(rid)
    x2, y2 = meshes("uniform_random", 900, 700, 5)
    u2, v2 = _masses(900, 700, 6)
    a = srv.submit_1d(x2, y2, u2, v2, 0.02, 1e-6, 5000)
    b = srv.submit_1d(x2, y2, u2, v2, 0.02, 1e-6, 5000)
    out = srv.run(long_ + [a, b])
    assert all(out[r][0]["status"] == lib.FINOM_ECANCELED for r in long_)
    assert all(out[r][0]["iters"] < 100000 for r in long_)
    assert out[a][0]["status"] == 0 and out[a][0]["converged"] == 1
    c = srv.submit_1d(x2, y2, u2, v2, 0.02, 1e-6, 5000)
    d = srv.submit_1d(x2, y2, u2, v2, 0.02, 1e-6, 5000)
    srv.step()
    srv.cancel(c)
    out = srv.run([c, d])
    srv.close()
    assert out[c][0]["status"] == lib.FINOM_ECANCELED
    assert out[d][0]["status"] == 0 and out[d][0]["converged"] == 1


def test_close_with_running_batches_and_reapers(lib):
    """Closing a server while batches run on their threads, solves run on their
    streams and retired plans wait for their reaper stops the batches, joins
    every thread and frees everything (the process goes on to use the GPU)."""
    srv = lib.Server(1 << 32, max_active=4, precision="f32_log")
    x, y = meshes("graded", 20000, 20000, 3)
    u, v = _masses(20000, 20000, 4)
    for _ in range(6):   # one long batch
        srv.submit_1d(x, y, u, v, 0.001, 1e-9, 100000)
    x2, y2 = meshes("uniform_random", 90000, 80000, 5)   # above the batching limit: alone
    u2, v2 = _masses(90000, 80000, 6)
    srv.submit_1d(x2, y2, u2, v2, 0.001, 1e-9, 100000)
    small = [_small_1d(n, 70 + n, 0.02) for n in (300, 500, 700)]
    ids = [_submit(srv, r) for r in small]
    for _ in range(3):
        srv.step()
    srv.close()
    # the GPU is usable afterwards, and a new server serves the small requests
    srv = lib.Server(1 << 32, max_active=2, precision="f32_log")
    ids = [_submit(srv, r) for r in small]
    out = srv.run(ids)
    srv.close()
    assert all(out[i][0]["status"] == 0 and out[i][0]["converged"] == 1 for i in ids)
