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
    assert ctypes.sizeof(g.Result) == 8 * 4 + 8 * 7 + 4 * 8 + 4 * 8 + 8 * 8


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


def test_struct_layout_matches_header_via_gcc(tmp_path):
    # the C compiler's sizeof / offsetof of every ABI struct against the ctypes mirrors
    import subprocess
    from paper_2602_17950_gb300 import gpsoc as g
    structs = {"gpsoc_grid": g.Grid, "gpsoc_trap": g.Trap, "gpsoc_params": g.Params, "gpsoc_opts": g.Opts,
               "gpsoc_result": g.Result, "gpsoc_server_opts": g.ServerOpts}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gpsoc.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, field, val = line.split()
            got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_server_argument_checks_without_gpu(lib):
    # server creation and submission validate their arguments before any device work
    import numpy as np
    from paper_2602_17950_gb300 import gpsoc as g
    L = g.library()
    h = ctypes.c_void_p()
    bad = g.ServerOpts(0.0, 4, 0, 16)
    assert L.gpsoc_server_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    ok = g.ServerOpts(1e9, 4, 0, 16)
    assert L.gpsoc_server_create(ctypes.byref(ok), ctypes.byref(h)) == 0
    try:
        grid = g.Grid(2, (ctypes.c_int * 3)(16, 16, 1), (ctypes.c_double * 3)(5, 5, 1))
        trap = g.Trap(0, (ctypes.c_double * 3)(1, 1, 1), 0.0, 0.0, None)
        par = g.Params(0.1, 0.2, 10.0, 0.0)
        psi = np.zeros((3, 16, 16), dtype=np.complex128)
        tk = ctypes.c_uint64(0)
        o = g.Problem.opts(tol=1e-10)
        assert L.gpsoc_server_submit(h, ctypes.byref(grid), ctypes.byref(trap), ctypes.byref(par),
                                     psi.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o), ctypes.byref(tk)) == 0
        o.precond = 7
        assert L.gpsoc_server_submit(h, ctypes.byref(grid), ctypes.byref(trap), ctypes.byref(par),
                                     psi.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o), ctypes.byref(tk)) == 1
        assert b"preconditioner" in L.gpsoc_last_error()
        o = g.Problem.opts(tol=1e-10, cm_levels=2)
        assert L.gpsoc_server_submit(h, ctypes.byref(grid), ctypes.byref(trap), ctypes.byref(par),
                                     psi.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o), ctypes.byref(tk)) == 1
        q = ctypes.c_int(-1)
        assert L.gpsoc_server_stats(h, None, None, ctypes.byref(q)) == 0 and q.value == 1
    finally:
        L.gpsoc_server_destroy(h)
