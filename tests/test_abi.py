"""The C-ABI library loads and exports every function include/hmpcg.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hmpcg.h")


def _ensure_built():
    from paper_2605_13343_gb300 import LIB_PATH
    if not os.path.exists(LIB_PATH):
        from paper_2605_13343_gb300 import build
        build.build()
    return LIB_PATH


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hmpcg_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    path = _ensure_built()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    import paper_2605_13343_gb300 as h
    assert set(declared_functions()) == set(h.EXPORTS)


def test_host_only_calls():
    _ensure_built()
    import paper_2605_13343_gb300 as h
    assert h.status_string(0) == "ok"
    assert "breakdown" in h.status_string(-4).lower()
    # packed widths: learned P of Sec. 4.4 and the svdh layout
    assert h.packed_width(8192, 64, 16, h.PRE_LEARNED) == 128 * 4096 + 127 * 256 + 2 * 8192 * 16 + 8192
    assert h.packed_width(1024, 64, 16, h.PRE_SVDH) == 16 * 4096 + 15 * 256 + 4 * 1024 * 16
    assert h.packed_width(1000, 64, 16, h.PRE_LEARNED) == -1
    lib = h.lib()
    dims = (ctypes.c_int32 * 3)(32, 16, 16)
    assert lib.hmpcg_system_bytes(3, dims) >= 8192 * 60
    bad = (ctypes.c_int32 * 3)(30, 16, 16)
    assert lib.hmpcg_system_bytes(3, bad) == -1


def test_invalid_arguments_rejected_on_host():
    _ensure_built()
    import paper_2605_13343_gb300 as h
    lib = h.lib()
    assert lib.hmpcg_destroy(None) == h.E_INVALID
    assert lib.hmpcg_create(None, None, None, 0, None) == h.E_INVALID
    assert lib.hmpcg_apply(None, None, None, None, 1, None) == h.E_INVALID
    assert lib.hmpcg_solve(None, None, None, None, None, None, None, None) == h.E_INVALID
