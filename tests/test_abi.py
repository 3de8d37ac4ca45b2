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
    # the ctypes mirror must have the C struct's size:
    # 3*4*2 + 6*8 + 2*4 + 6*8 + 2*4 + 6*8 + 4 + 12 + 6*4 + 4 + 4
    import paper_2202_12309_gb300 as ph
    expected = 24 + 48 + 8 + 48 + 8 + 48 + 4 + 12 + 24 + 8
    assert ctypes.sizeof(ph.Config) == expected


def test_invalid_config_rejected_without_gpu_work():
    import paper_2202_12309_gb300 as ph
    L = ph.lib()
    cfg = ph.make_config((2, 16, 16), (1, 1, 1))   # nx < 4: rejected before any CUDA call
    h = ctypes.c_void_p()
    rc = L.ph_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert rc == -1
    assert b"nx" in L.ph_last_error()


BAD_CONFIGS = [
    dict(nx=(16, 16, 16), nb=(0, 1, 1)),                       # no blocks
    dict(nx=(16, 16, 16), nb=(1, 1, 1), xmin=(0, 0, 0), xmax=(0, 1, 1)),  # empty domain
    dict(nx=(16, 16, 16), nb=(1, 1, 1), max_level=5),          # deeper than the supported tree
    dict(nx=(15, 16, 16), nb=(1, 1, 1), max_level=1),          # odd block on a multi-level mesh
    dict(nx=(16, 16, 16), nb=(1, 1, 1), gamma=1.0),            # gamma must exceed 1
    dict(nx=(16, 16, 16), nb=(1, 1, 1), cfl=0.0),
    dict(nx=(16, 16, 16), nb=(1, 1, 1), tile=(24, 8, 16)),     # unsupported tile
    dict(nx=(16, 16, 16), nb=(1, 1, 1), tile=(16, 16, 17)),    # chunk deeper than the block
    dict(nx=(16, 16, 16), nb=(1, 1, 1), bc=("periodic", "outflow") + ("periodic",) * 4),  # half periodic
    dict(nx=(16, 16, 16), nb=(1, 1, 1), bc=(0, 0, 3, 3, 0, 0)),  # unknown boundary kind
    dict(nx=(16, 16, 16), nb=(1, 1, 1), nscalars=3),           # more passive scalars than supported
    dict(nx=(16, 16, 16), nb=(1, 1, 1), nscalars=1, tile=(32, 8, 16)),  # tile without a scalar kernel
]


@pytest.mark.parametrize("kw", BAD_CONFIGS)
def test_invalid_configs_rejected_before_any_cuda_call(kw):
    import paper_2202_12309_gb300 as ph
    L = ph.lib()
    kw = dict(kw)
    nx, nb = kw.pop("nx"), kw.pop("nb")
    cfg = ph.make_config(nx, nb, **kw)
    h = ctypes.c_void_p()
    assert L.ph_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1
    assert h.value is None
    assert len(L.ph_last_error()) > 0


def test_bad_precision_and_batch_arguments_rejected():
    import paper_2202_12309_gb300 as ph
    L = ph.lib()
    cfg = ph.make_config((16, 16, 16), (1, 1, 1))
    cfg.precision = 7
    h = ctypes.c_void_p()
    assert L.ph_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1
    # batches: mixed precision, two-level member
    a = ph.make_config((16, 16, 16), (1, 1, 1))
    b = ph.make_config((16, 16, 16), (1, 1, 1), precision="fp32")
    arr = (ph.Config * 2)(a, b)
    assert L.ph_batch_create(arr, 2, None, ctypes.byref(h)) == -1
    c = ph.make_config((16, 16, 16), (1, 1, 1), max_level=1)
    arr = (ph.Config * 1)(c)
    assert L.ph_batch_create(arr, 1, None, ctypes.byref(h)) == -1
    assert L.ph_batch_create(arr, 0, None, ctypes.byref(h)) == -1


def test_null_handles_rejected():
    import paper_2202_12309_gb300 as ph
    L = ph.lib()
    assert L.ph_step(None, 1) == -1
    assert L.ph_num_blocks(None, None) == -1
    assert L.ph_destroy(None) == 0
    assert L.ph_batch_destroy(None) == 0
    # allocator hooks come in pairs
    assert L.ph_set_allocator(ctypes.c_void_p(1), None, None) == -1
    # no-allocation totals: checks happen before any device work
    out = ctypes.c_void_p(8)
    n3 = (ctypes.c_int32 * 3)(4, 4, 4)
    vol = (ctypes.c_double * 2)(1.0, 0.125)
    assert L.ph_totals_noalloc(None, 0, n3, 5, 1, None, vol, 1, out, None) == -1
    assert L.ph_totals_noalloc(ctypes.c_void_p(8), 3, n3, 5, 1, None, vol, 1, out, None) == -1
    assert L.ph_totals_noalloc(ctypes.c_void_p(8), 0, n3, 5, 1 << 20, None, vol, 1, out, None) == -1
    assert L.ph_totals_noalloc(ctypes.c_void_p(8), 0, n3, 8, 1, None, vol, 1, out, None) == -1
    assert L.ph_totals_noalloc(ctypes.c_void_p(8), 0, n3, 5, 1, None, vol, 2, out, None) == -1
    assert L.ph_totals_noalloc(ctypes.c_void_p(8), 0, n3, 5, 1, None, None, 1, out, None) == -1


def test_load_validates_the_file_before_any_device_work(tmp_path):
    import paper_2202_12309_gb300 as ph
    L = ph.lib()
    h = ctypes.c_void_p()
    assert L.ph_load(os.fsencode(str(tmp_path / "missing.phr")), None, ctypes.byref(h)) == -7
    assert not h.value
    junk = tmp_path / "junk.phr"
    junk.write_bytes(b"not a restart file" * 64)
    assert L.ph_load(os.fsencode(str(junk)), None, ctypes.byref(h)) == -1
    short = tmp_path / "short.phr"
    short.write_bytes(b"PHYDRST1")
    assert L.ph_load(os.fsencode(str(short)), None, ctypes.byref(h)) == -7
    assert L.ph_load(None, None, ctypes.byref(h)) == -1
    assert L.ph_save(None, os.fsencode(str(junk)), 0) == -1
