"""The 2^(k/64) table of the float64 kernels' table-driven 2^x (Tang's
method, base 2) and the steps of that 2^x, checked on the CPU.

The table (paper_2605_26659_gb300/csrc/exp2_table.h) is pinned against the C
library's exp2 and against the identities 2^(a/64) 2^(b/64) = 2^((a+b)/64);
the reduction x = n + k/64 + r (integer operations on the bits of x) and the
degree-6 series are replayed in Python, step for step as the kernel takes
them, against exp2 over the range the scans use.
"""
import math
import os
import re
import struct

import numpy as np

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2605_26659_gb300", "csrc", "exp2_table.h")


def _table():
    txt = open(HDR).read()
    vals = [float.fromhex(h) for h in re.findall(r"0x[0-9a-f]\.[0-9a-f]+p[+-]\d+", txt)]
    assert len(vals) == 64
    return vals


def _ulp(v):
    return math.ulp(v)


def test_table_is_two_to_the_k_over_64():
    t = _table()
    for k, v in enumerate(t):
        assert abs(v - math.exp2(k / 64)) <= _ulp(v), k
    # products of entries (each within half an ulp of its exact value)
    for a in range(64):
        for b in range(64 - a):
            assert abs(t[a] * t[b] - t[a + b]) <= 2 * _ulp(t[a + b]), (a, b)
    for a in range(1, 64):
        assert abs(t[a] * t[64 - a] - 2.0) <= 4 * _ulp(2.0), a


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _double(b):
    return struct.unpack("<d", struct.pack("<Q", b & 0xFFFFFFFFFFFFFFFF))[0]


def _exp2_tab(x, t):
    """The kernel's steps (integer parts as Python ints, float64 parts as
    float64 with fused multiply-adds emulated exactly)."""
    u = _bits(x)
    ex = (u >> 52) & 0x7FF
    neg = (u >> 63) != 0
    if ex >= 1023 + 11:
        nan = ex == 0x7FF and (u & ((1 << 52) - 1)) != 0
        return 0.0 if (neg or nan) else math.inf
    if ex < 1023 - 53:
        return 1.0
    m = (u & ((1 << 52) - 1)) | (1 << 52)
    sh = ex - 1023
    X = (m << sh) if sh >= 0 else (m >> (-sh))
    Xs = -X if neg else X
    n = Xs >> 52
    if n < -1021:
        return 0.0
    if n > 1023:
        return math.inf
    F = Xs & ((1 << 52) - 1)
    k = F >> 46
    r = float(F & ((1 << 46) - 1))
    c = 0.69314718055994530942 * 2.0 ** -52
    tt = r * c

    def fma(a, b, d):   # one rounding
        from fractions import Fraction
        return float(Fraction(a) * Fraction(b) + Fraction(d))

    p = 1.3888888888888888889e-03
    for coef in (8.3333333333333333333e-03, 4.1666666666666666667e-02, 1.6666666666666666667e-01, 0.5, 1.0, 1.0):
        p = fma(p, tt, coef)
    v = t[k] * p
    return _double(_bits(v) + (n << 52))


def test_table_driven_exp2_steps_against_exp2():
    t = _table()
    g = np.random.default_rng(20)
    xs = list(g.uniform(-1021, 1023, 3000)) + list(g.uniform(-2, 2, 3000)) + list(g.normal(0, 1e-3, 500))
    xs += [0.0, -0.0, 1.0, -1.0, 0.5, -0.5, 1 / 64, -1 / 64, 63 / 64, -1e-17, 1e-17, 1023.0, -1021.0,
           1023.5, 2.0 ** -52, -(2.0 ** -52), 1000.015625, -1000.015625]
    worst = 0.0
    for x in xs:
        got = _exp2_tab(float(x), t)
        want = math.exp2(float(x))
        worst = max(worst, abs(got - want) / _ulp(want))
    assert worst <= 3.0, worst
    # the ends
    assert _exp2_tab(-1022.0, t) == 0.0 and _exp2_tab(-1e300, t) == 0.0 and _exp2_tab(-math.inf, t) == 0.0
    assert _exp2_tab(1024.5, t) == math.inf and _exp2_tab(math.inf, t) == math.inf
    assert _exp2_tab(math.nan, t) == 0.0


def _exp2_split(x, t):
    """2^x = v 2^n, n = floor(x), v = 2^(x - n): the kernel's steps for the
    terms of the float64 scans (levels of any size; none gives v = 0)."""
    ux = _bits(x)
    if (ux >> 63) and ((ux >> 52) & 0x7FF) >= 1023 + 900:
        return 0.0, 0.0
    n = math.floor(x)
    f = x - n
    u = _bits(f)
    ex = (u >> 52) & 0x7FF
    if ex < 1023 - 53:
        return 1.0, float(n)
    if ex >= 1023:
        return 1.0, float(n + 1)
    F = ((u & ((1 << 52) - 1)) | (1 << 52)) >> (1023 - ex)
    k = F >> 46
    r = float(F & ((1 << 46) - 1))
    tt = r * (0.69314718055994530942 * 2.0 ** -52)
    from fractions import Fraction
    p = 1.3888888888888888889e-03
    for coef in (8.3333333333333333333e-03, 4.1666666666666666667e-02, 1.6666666666666666667e-01, 0.5, 1.0, 1.0):
        p = float(Fraction(p) * Fraction(tt) + Fraction(coef))
    return t[k] * p, float(n)


def _pow2_neg(d):
    u = _bits(d)
    ex = (u >> 52) & 0x7FF
    if ex < 1023:
        return 1.0
    if ex >= 1023 + 10:
        return 0.0
    k = (((u & ((1 << 52) - 1)) | (1 << 52)) >> (52 - (ex - 1023)))
    return 0.0 if k > 1022 else _double((1023 - k) << 52)


def test_split_terms_and_whole_number_scales():
    t = _table()
    g = np.random.default_rng(21)
    xs = list(g.uniform(-3e4, 3e4, 3000)) + list(g.uniform(-3, 3, 3000)) + [0.0, -1e-20, 5e-17, 2047.999, -0.5,
                                                                                   -3.0 - 1e-17, 7.0 - 2.0 ** -50]
    for x in xs:
        v, n = _exp2_split(float(x), t)
        assert n in (math.floor(x), math.floor(x) + 1) and 1.0 <= v < 2.0
        # 2^x = 2^(x - n) 2^n, x - n in [0, 1) rounded at most once
        want = math.exp2(x - n)
        assert abs(v - want) <= 3 * _ulp(want), x
    assert _exp2_split(-1e300, t) == (0.0, 0.0)
    for d in range(-1100, 1100):
        want = 0.0 if abs(d) > 1022 else 2.0 ** -abs(d)
        assert _pow2_neg(float(d)) == want
    assert _pow2_neg(1e300) == 0.0 and _pow2_neg(-1e300) == 0.0 and _pow2_neg(0.0) == 1.0


def test_table_header_is_what_its_generator_writes():
    import contextlib
    import importlib.util
    import io
    gen = os.path.join(os.path.dirname(HDR), "gen_exp2_table.py")
    spec = importlib.util.spec_from_file_location("gen_exp2_table", gen)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        mod.main()
    assert buf.getvalue() == open(HDR).read()
