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


def _dense_ok(N, L, b, n):
    # the host's rule for the sub-cell path of dense cells (k <= 9 sub-cells of
    # side s/k with sqrt(3)(s/k + 2 eps) <= b (1 - 1e-4) and b + 2 eps < 2 s/k)
    import math
    s = L / n
    k = max(1, math.ceil(s * math.sqrt(3.0) * 1.02 / b))
    sf = s / k
    eps = 4.0 * L * 2.0 ** -24
    return (n >= 5 and k <= 9 and math.sqrt(3.0) * (sf + 2 * eps) <= b * (1 - 1e-4)
            and (b + 2 * eps) / sf < 2.0)


def test_default_grid_keeps_the_dense_path(lib):
    # the default grid is the largest legal n with n^3 <= N, raised (by at most
    # max(2, n/8)) to the first n whose cells are narrow enough for 9 sub-cells
    import synth
    n = ctypes.c_int32()
    lib.jfof_default_cells_per_axis.argtypes = [ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                                                ctypes.POINTER(ctypes.c_int32)]
    raised = 0
    for N, L in [(73228, 129.0), (32876, 395.0), (243739, 338.0), (1203185, 220.0), (6417007, 318.0),
                 (32 ** 3, 100.0), (40 ** 3 + 1000, 75.0), (150_000, 50.0), (1 << 24, 250.0)]:
        b = synth.linking_length(L, N)
        assert lib.jfof_default_cells_per_axis(N, L, b, ctypes.byref(n)) == 0
        n0 = 3
        while (n0 + 1) ** 3 <= N:
            n0 += 1
        cands = [m for m in range(n0, n0 + max(2, n0 // 8) + 1) if _dense_ok(N, L, b, m)]
        if cands:
            assert n.value == cands[0], (N, L, n.value, cands)
            raised += n.value > n0
        else:
            assert n.value == n0
    assert raised >= 1  # 73228 particles in L = 129: n = 41 has k = 10, so 42
