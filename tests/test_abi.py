"""The C-ABI library builds, loads and exports every symbol that
include/feast_gb300.h declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re

from helpers import ROOT, lib


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "feast_gb300.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(feast_\w+)\s*\(", txt)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("feast_create", "feast_filter", "feast_rayleigh_ritz", "feast_solve", "feast_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    fg = lib()
    so = ctypes.CDLL(fg.LIB_PATH)
    for name in declared_functions():
        assert hasattr(so, name), name
    assert set(fg.SYMBOLS) == set(declared_functions())


def test_status_strings_and_defaults():
    fg = lib()
    assert fg.status_str(0) == "ok"
    assert "singular" in fg.status_str(fg.FEAST_ERR_SINGULAR_SHIFT)
    o = fg.make_options()
    assert o.tol == 1e-10 and o.max_iter == 20 and o.cand_tol == 1e-4
