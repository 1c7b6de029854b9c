"""The C-ABI library builds, loads and exports every entry point include/swept.h declares.

No GPU needed: only calls that validate arguments before touching CUDA are made.
"""
from __future__ import annotations

import ctypes
import os
import re

import pytest

import paper_1504_01380_gb300 as sw
from paper_1504_01380_gb300 import build as swbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(swept_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    swbuild.build()
    return sw.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert names, "no declarations found"
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} not exported"
    assert names == set(sw.EXPORTS)


def test_strerror_and_version(lib):
    assert sw.strerror(0) == "ok"
    assert "invalid" in sw.strerror(-1)
    assert sw.swept_version().endswith("sm_103a")


def _plan_rc(lib, N, radius, stencil, params, dtype, B):
    h = ctypes.c_void_p()
    prm = (ctypes.c_double * len(params))(*params)
    return lib.swept_plan(ctypes.byref(h), N, radius, stencil, prm, len(params), dtype, B)


@pytest.mark.parametrize("N,radius,stencil,params,dtype,B,code", [
    (20, 1, 0, [0.25], 0, 32, -1),          # shorter than one tile of the given width
    (1280, 1, 0, [0.25], 0, 512, -1),       # uneven tiles would need 8 wide windows out of 2
    (100, 2, 1, [0.002, 0.5], 0, 128, -1),  # KS: shorter than one 128-point tile
    (1000, 1, 0, [0.25], 0, 512, -1),       # 1 tile of 512 with 488 left: needs 16 wide windows
    (2000, 1, 0, [0.25], 0, 1024, -1),      # 1 tile of 1024 with 976 left: needs 31 wide windows
    (1024, 2, 0, [0.25], 0, 32, -1),        # radius does not match heat
    (1024, 1, 1, [0.002, 0.5], 0, 64, -1),  # radius does not match KS
    (1024, 2, 1, [0.002, 0.5], 0, 32, -1),  # KS needs K % 2 == 0
    (1024, 1, 0, [0.25], 0, 96, -5),        # K = 3 not built
    (1024, 1, 0, [0.25], 0, 48, -1),        # B not a multiple of 32
    (1024, 1, 0, [0.25], 7, 32, -1),        # unknown dtype
    (1024, 1, 5, [0.25], 0, 32, -1),        # unknown stencil
    (0, 1, 0, [0.25], 0, 32, -1),           # empty grid
    (1024, 2, 1, [0.002, 0.0], 0, 64, -1),  # dx must be positive
    (1024, 2, 1, [0.002], 0, 64, -1),       # KS needs two parameters
    (1024, 1, 4, [1e-4, 1e-3, 1.4], 1, 512, -5),  # compensated Euler: B <= 256
    (1024, 1, 4, [1e-4, 1e-3, 1.4], 2, 64, -5),   # plain FP32: forward-Euler heat and KS only
    (1024, 1, 2, [0.25], 2, 64, -5),              # plain FP32: no Runge-Kutta
    (1024, 1, 4, [1e-4, 1e-3, 1.4], 0, 256, -5),  # FP64 Euler: B <= 128
    (1024, 2, 4, [1e-4, 1e-3, 1.4], 0, 32, -1),   # Euler radius is 1
    (1024, 1, 4, [1e-4, 1e-3], 0, 32, -1),        # Euler needs {dt, dx, gamma}
    (1024, 1, 4, [1e-4, 1e-3, 1.0], 0, 32, -1),   # gamma must exceed 1
    (1024, 1, 4, [1e-4, 0.0, 1.4], 0, 32, -1),    # dx must be positive
])
def test_plan_validation(lib, N, radius, stencil, params, dtype, B, code):
    assert _plan_rc(lib, N, radius, stencil, params, dtype, B) == code


def test_null_arguments(lib):
    assert lib.swept_advance(None, None, 10, None) == -1
    assert lib.swept_naive_advance(None, None, 10, None) == -1
    assert lib.swept_reduce(None, None, 0, None, None, None) == -1
    assert lib.swept_f32c_split(0, None, None, None) == -1
    info = (ctypes.c_int64 * 6)()
    assert lib.swept_plan_info(None, info, 6) == -1
    n, nr, ms = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    assert lib.swept_plan_last_advance(None, ctypes.byref(n), ctypes.byref(nr), ctypes.byref(ms)) == -1
    assert lib.swept_plan_set(None, 7, 1) == -1
    lib.swept_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError, match="not built"):
        sw._lib = None
        try:
            sw.load(str(tmp_path / "missing.so"))
        finally:
            sw._lib = None


def test_binding_constants_match_the_header():
    """Every SWEPT_* integer constant of the binding has the value include/swept.h defines."""
    text = open(os.path.join(ROOT, "include", "swept.h")).read()
    defined = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(SWEPT_\w+)\s+(-?\d+)\b", text)}
    assert {"SWEPT_OPT_RESIDENT", "SWEPT_OPT_NAIVE_RESIDENT", "SWEPT_OPT_STREAM"} <= set(defined)
    checked = 0
    for name, value in defined.items():
        if hasattr(sw, name):
            assert getattr(sw, name) == value, name
            checked += 1
    assert checked >= 20
