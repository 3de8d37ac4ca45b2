"""The C-ABI library builds, loads and exports every symbol include/ph_hydro.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ph_hydro.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"^\s*(?:int|const char\*|void)\s+\**(ph_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_symbols()
    assert "ph_create" in names and "ph_step" in names and len(names) >= 20


def test_library_exports_all_declared_symbols():
    import paper_2202_12309_gb300 as ph
    from paper_2202_12309_gb300 import build as B
    B.build()
    L = ctypes.CDLL(ph.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(L, name), name
    assert set(ph.EXPORTS) == set(declared_symbols())


def test_config_struct_layout_matches_header():
    # the ctypes mirror must have the C struct's size: 3*4*2 + 6*8 + 2*4 + 6*8 + 2*4 + 6*8 + 4 + 12
    import paper_2202_12309_gb300 as ph
    expected = 24 + 48 + 8 + 48 + 8 + 48 + 4 + 12
    assert ctypes.sizeof(ph.Config) == expected


def test_invalid_config_rejected_without_gpu_work():
    import paper_2202_12309_gb300 as ph
    L = ph.lib()
    cfg = ph.make_config((2, 16, 16), (1, 1, 1))   # nx < 4: rejected before any CUDA call
    h = ctypes.c_void_p()
    rc = L.ph_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert rc == -1
    assert b"nx" in L.ph_last_error()
