"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/gw.h (no GPU needed: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "gw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gw_[a-z0-9_]+)\s*\(", src)))


def test_builds_and_exports_every_declared_symbol():
    from paper_1408_3036_gb300 import _build
    lib_path = _build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared()
    assert "gw_setup" in names and "gw_lanczos" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_1408_3036_gb300 as g
    assert set(declared()) <= set(g.EXPORTS)


def test_null_context_is_an_error_not_a_crash():
    from paper_1408_3036_gb300 import _build
    lib = ctypes.CDLL(_build.build())
    lib.gw_npw.restype = ctypes.c_int
    assert lib.gw_npw(None) == 0
    lib.gw_stats.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    assert lib.gw_stats(None, None, 0) != 0
    lib.gw_setup.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                             ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    out = ctypes.c_void_p()
    # invalid grid size is rejected before any device work
    assert lib.gw_setup(ctypes.byref(out), 10.0, 7 * 11, 5.0, None, 0, None) == 1
