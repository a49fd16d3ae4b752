"""The C-ABI library loads and exports every symbol include/tsp.h declares, and
argument validation that happens before any CUDA call reports the documented
status codes (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2608_16960_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(tsp_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    names = declared_symbols()
    assert "tsp_forward" in names and "tsp_adjoint" in names and "tsp_grid_create" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert L.tsp_version() >= 1


def _grid(r, t, p):
    L = _lib.load()
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (r, t, p)]
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    st = L.tsp_grid_create(ptr(arrs[0]), len(arrs[0]), ptr(arrs[1]), len(arrs[1]), ptr(arrs[2]), len(arrs[2]),
                           ctypes.byref(h))
    return st, L.tsp_last_error().decode()


@pytest.mark.parametrize("edges,status", [
    (([1, 2, 2, 3], [0, 1, 2], [0, 1, 2]), 2),          # repeated radial edge -> TSP_ENOTMONO
    (([1, 2, 3], [0, 2, 1], [0, 1, 2]), 2),             # decreasing polar edges
    (([-1, 2, 3], [0, 1, 2], [0, 1, 2]), 1),            # negative radius -> TSP_EINVAL
    (([1, 2, 3], [0, 1, 4], [0, 1, 2]), 1),             # polar edge beyond pi
    (([1, 2, 3], [0, 1, 2], [0, 4, 7]), 1),             # azimuth span beyond 2 pi
    (([1], [0, 1, 2], [0, 1, 2]), 1),                   # too few edges
    (([1, float("nan"), 3], [0, 1, 2], [0, 1, 2]), 1),  # non-finite edge
])
def test_grid_validation_status_codes(edges, status):
    st, msg = _grid(*edges)
    assert st == status, (st, msg)
    assert msg


def test_null_arguments_rejected():
    L = _lib.load()
    assert L.tsp_grid_create(None, 3, None, 3, None, 3, None) == 1
    assert L.tsp_forward(None, None, None, None, 1, None) == 1
    assert L.tsp_adjoint(None, None, None, None, 1, 0, None) == 1
    n = ctypes.c_int64()
    assert L.tsp_geom_num_rays(None, ctypes.byref(n)) == 1
    assert L.tsp_geom_cone(0, None, None, None, 4, 4, 30.0, 30.0, None) == 1
    assert L.tsp_autotune_store(None, None, None, None) == 1


def test_stall_hook_rejects_bad_budgets():
    """tsp_debug_tc_stall takes 1 .. 2e9 cycles (host-side check, no device)."""
    L = _lib.load()
    assert L.tsp_debug_tc_stall(0) == 1  # TSP_EINVAL
    assert L.tsp_debug_tc_stall(3_000_000_000) == 1
    assert b"wait_cycles" in L.tsp_last_error()
