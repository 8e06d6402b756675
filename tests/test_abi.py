"""The C ABI library builds, loads and exports every entry point of include/finom.h (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "finom.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(finom_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2605_26659_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for n in ["finom_plan", "finom_plan_destroy", "finom_kv", "finom_ktu", "finom_solve",
              "finom_dividing_index", "finom_kv_log", "finom_ktu_log", "finom_cost"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (finom_[a-z0-9_]+)\b", out))
    assert set(declared()) <= exported


def test_version_and_error_string_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.finom_version.restype = ctypes.c_int
    lib.finom_last_error.restype = ctypes.c_char_p
    assert lib.finom_version() >= 100
    assert isinstance(lib.finom_last_error(), bytes)


def test_null_plan_is_rejected_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.finom_kv.argtypes = [ctypes.c_void_p] * 4
    lib.finom_kv.restype = ctypes.c_int
    assert lib.finom_kv(None, None, None, None) == 1   # FINOM_EINVAL
    lib.finom_plan.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                               ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.finom_plan.restype = ctypes.c_int
    h = ctypes.c_void_p()
    # bad sizes / eps are rejected before any CUDA call
    assert lib.finom_plan(None, 0, None, 5, 0.1, 1, None, ctypes.byref(h)) == 1
    assert lib.finom_plan(None, 5, None, 5, -1.0, 1, None, ctypes.byref(h)) == 1


def test_tuning_table_round_trip_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.finom_tune_set.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_int32]
    lib.finom_tune_set.restype = ctypes.c_int
    lib.finom_tune_get.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    lib.finom_tune_get.restype = ctypes.c_int
    e = ctypes.c_int32()
    for prec in (0, 1):
        for b in (0, 10, 20, 39):
            assert lib.finom_tune_get(prec, b, ctypes.byref(e)) == 0
            assert e.value in (-1, 1, 2, 4, 8)
    old = ctypes.c_int32()
    lib.finom_tune_get(1, 12, ctypes.byref(old))
    assert lib.finom_tune_set(1, 12, 4) == 0
    assert lib.finom_tune_get(1, 12, ctypes.byref(e)) == 0 and e.value == 4
    assert lib.finom_tune_set(1, 12, old.value) == 0
    # invalid entries are refused and change nothing
    assert lib.finom_tune_set(1, 12, 3) == 1
    assert lib.finom_tune_set(1, 40, 2) == 1
    assert lib.finom_tune_set(7, 12, 2) == 1
    assert lib.finom_tune_get(1, -1, ctypes.byref(e)) == 1
    lib.finom_tune_get(1, 12, ctypes.byref(e))
    assert e.value == old.value


def test_tuning_cache_applies_without_gpu(libpath, tmp_path):
    """The autotuner's JSON cache round trip: apply() installs its entries in
    the library's table (host-side; no GPU needed)."""
    import json
    from paper_2605_26659_gb300 import api, autotune
    api.load()
    before = {(p, b): api.finom_tune_get(p, b) for p in ("f64", "f32_log") for b in (11, 17)}
    cache = {"buckets": {"f64": {"11": 2, "17": 8}, "f32_log": {"11": 4, "17": 1}}}
    path = tmp_path / "tune.json"
    path.write_text(json.dumps(cache))
    autotune.apply(str(path))
    try:
        assert api.finom_tune_get("f64", 11) == 2 and api.finom_tune_get("f64", 17) == 8
        assert api.finom_tune_get("f32_log", 11) == 4 and api.finom_tune_get("f32_log", 17) == 1
    finally:
        for (p, b), e in before.items():
            api.finom_tune_set(p, b, e)
    old = api.finom_tune_get_batch("f32_log")
    api.finom_tune_set_batch("f32_log", 2)
    assert api.finom_tune_get_batch("f32_log") == 2
    api.finom_tune_set_batch("f32_log", old)
