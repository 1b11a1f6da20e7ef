"""The C-ABI library builds, loads and exports every symbol include/jfof.h
declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "jfof.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jfof_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_26851_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert len(syms) >= 17
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    import paper_2510_26851_gb300 as j
    assert sorted(j.EXPORTED) == declared_symbols()


def test_host_side_argument_checks(lib):
    # pure host logic: no device is touched by these calls
    n = ctypes.c_int32()
    lib.jfof_max_cells_per_axis.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.POINTER(ctypes.c_int32)]
    assert lib.jfof_max_cells_per_axis(100.0, 0.625, ctypes.byref(n)) == 0
    assert n.value == 158  # floor(100 / (1.01 * 0.625))
    assert lib.jfof_max_cells_per_axis(10.0, 4.0, ctypes.byref(n)) == 0
    assert n.value == 1  # floor(10 / 4.04) = 2 -> 1 (a 2-cell stencil would repeat cells)
    lib.jfof_default_cells_per_axis.argtypes = [ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                                                ctypes.POINTER(ctypes.c_int32)]
    assert lib.jfof_default_cells_per_axis(32768, 100.0, 0.625, ctypes.byref(n)) == 0
    assert n.value == 32
    assert lib.jfof_default_cells_per_axis(1 << 30, 1000.0, 0.1953125, ctypes.byref(n)) == 0
    assert n.value == 1024
    assert lib.jfof_default_cells_per_axis(10, 10.0, 6.0, ctypes.byref(n)) == 1  # b >= L/2
    assert lib.jfof_default_cells_per_axis(0, 10.0, 1.0, ctypes.byref(n)) == 1   # N < 1
    sz = ctypes.c_size_t()
    lib.jfof_fof_bytes.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
    assert lib.jfof_fof_bytes(1000, 2, ctypes.byref(sz)) == 1
    assert lib.jfof_fof_bytes(1000, 8, ctypes.byref(sz)) == 0 and sz.value > 32 * 1000
    lib.jfof_strerror.restype = ctypes.c_char_p
    assert b"workspace" in lib.jfof_strerror(3)
