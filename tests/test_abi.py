"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every function include/gpsoc.h declares; the
binding's structures match the header's layout."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_17950_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def _declared():
    src = open(os.path.join(ROOT, "include", "gpsoc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gpsoc_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2602_17950_gb300 import gpsoc
    assert set(_declared()) <= set(gpsoc._PROTOS)


def test_struct_sizes_match_c_layout():
    from paper_2602_17950_gb300 import gpsoc as g
    assert ctypes.sizeof(g.Grid) == 4 + 12 + 24              # int, int[3], double[3]
    assert ctypes.sizeof(g.Params) == 32
    assert ctypes.sizeof(g.Result) == 8 * 4 + 8 * 7 + 4 * 8 + 4 * 8


def test_version_and_error_without_gpu(lib):
    from paper_2602_17950_gb300 import gpsoc as g
    L = g.library()
    assert L.gpsoc_version().startswith(b"gpsoc")
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    grid = g.Grid(2, (ctypes.c_int * 3)(12, 16, 1), (ctypes.c_double * 3)(1, 1, 1))
    trap = g.Trap(0, (ctypes.c_double * 3)(1, 1, 1), 0.0, 0.0, None)
    par = (g.Params * 1)(g.Params(0, 0, 0, 0))
    assert L.gpsoc_create(ctypes.byref(grid), ctypes.byref(trap), par, 1, None, ctypes.byref(h)) == 1
    assert b"power" in L.gpsoc_last_error()
    grid = g.Grid(4, (ctypes.c_int * 3)(16, 16, 1), (ctypes.c_double * 3)(1, 1, 1))
    assert L.gpsoc_create(ctypes.byref(grid), ctypes.byref(trap), par, 1, None, ctypes.byref(h)) == 1
    grid = g.Grid(2, (ctypes.c_int * 3)(16, 16, 1), (ctypes.c_double * 3)(1, -1, 1))
    assert L.gpsoc_create(ctypes.byref(grid), ctypes.byref(trap), par, 1, None, ctypes.byref(h)) == 1
    par = (g.Params * 1)(g.Params(float("nan"), 0, 0, 0))
    grid = g.Grid(2, (ctypes.c_int * 3)(16, 16, 1), (ctypes.c_double * 3)(1, 1, 1))
    assert L.gpsoc_create(ctypes.byref(grid), ctypes.byref(trap), par, 1, None, ctypes.byref(h)) == 1
    assert L.gpsoc_solve(None, None, None) == 1
