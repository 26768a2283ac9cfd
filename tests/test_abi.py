"""The C-ABI library loads, exports every symbol include/lbm.h declares, and
validates its arguments -- all without a GPU (no compute calls here).  Its
lattice constants, solved by its own method, agree with the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "lbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lbmlib):
    from paper_1606_06107_gb300 import lbm
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lbmlib, name), name
        assert name in lbm.SIGNATURES, name


@pytest.mark.parametrize("name,kind", [("D1Q7", 1), ("D2Q37", 2), ("D2Q49", 3), ("D3Q343", 4)])
def test_library_lattice_matches_oracle(lbmlib, orc, name, kind):
    from paper_1606_06107_gb300 import lbm
    r, e, w = lbm.lattice_info(name)
    ro, eo, wo, _ = orc.lattice(kind)
    assert abs(r - ro) < 1e-13
    assert np.array_equal(e, eo)
    assert np.allclose(w, wo, rtol=1e-12, atol=1e-16)


def _create(lib, D, lattice, n, tau):
    h = ctypes.c_void_p()
    rc = lib.lbm_create(D, lattice, n, tau, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("args", [(0, 1, 4, 0.7), (2, 1, 4, 0.7), (1, 1, -1, 0.7), (1, 1, 4, 0.0),
                                  (1, 1, 4, -1.0), (2, 9, 3, 0.7), (2, 4, 0, 0.7),
                                  (1, 1, 4, float("nan"))])
def test_create_rejects_bad_arguments(lbmlib, args):
    rc, h = _create(lbmlib, *args)
    assert rc == -1 and not h.value


def test_grid_validation_and_sizes(lbmlib):
    rc, h = _create(lbmlib, 2, 3, 3, 2 / 3)
    assert rc == 0
    try:
        sb, wb = ctypes.c_size_t(), ctypes.c_size_t()
        shape = (ctypes.c_int64 * 3)(1000, 70000, 1)
        bc = (ctypes.c_int * 3)(0, 1, 0)
        assert lbmlib.lbm_set_grid(h, shape, bc, ctypes.byref(sb), ctypes.byref(wb)) == -2
        shape = (ctypes.c_int64 * 3)(1000, 16, 1)
        bad_bc = (ctypes.c_int * 3)(0, 7, 0)
        assert lbmlib.lbm_set_grid(h, shape, bad_bc, ctypes.byref(sb), ctypes.byref(wb)) == -1
        assert lbmlib.lbm_set_grid(h, shape, bc, ctypes.byref(sb), ctypes.byref(wb)) == 0
        assert sb.value == 4 * (49 + 7) * 1024 * 16      # rows padded to 32 floats
        assert wb.value > 0
        assert lbmlib.lbm_set_mode(h, 1, 10) == -6       # mode after grid: out of order
        assert lbmlib.lbm_step(h, 1) == -6               # no state yet
        assert lbmlib.lbm_step(h, -1) == -1
        assert b"lbm_set_macro" in lbmlib.lbm_last_error(h) or lbmlib.lbm_last_error(h)
    finally:
        lbmlib.lbm_destroy(h)


def test_mode_validation(lbmlib):
    rc, h = _create(lbmlib, 1, 1, 4, 2 / 3)
    assert rc == 0
    try:
        assert lbmlib.lbm_set_mode(h, 1, 0) == -1
        assert lbmlib.lbm_set_mode(h, 5, 1) == -1
        assert lbmlib.lbm_set_mode(h, 1, 10) == 0
    finally:
        lbmlib.lbm_destroy(h)


def test_product_path_has_no_oracle_dependency():
    """The package never imports or links the oracle (test infrastructure)."""
    pkg = os.path.join(os.path.dirname(HEADER), "..", "paper_1606_06107_gb300")
    pat = re.compile(r"^\s*(import|from)\s+oracle\b|liborc|lbm_oracle", re.M)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                assert not pat.search(open(os.path.join(root, f)).read()), f


def test_batch_create_validation_and_sizes(lbmlib):
    L = (ctypes.c_int64 * 3)(10, 40, 33)
    n = (ctypes.c_int * 3)(2, 4, 0)
    tau = (ctypes.c_double * 3)(0.7, 0.6, 1.0)
    h = ctypes.c_void_p()
    assert lbmlib.lbm_batch_create(0, L, n, tau, 1, 10, ctypes.byref(h)) == -1
    assert lbmlib.lbm_batch_create(3, L, n, tau, 1, 0, ctypes.byref(h)) == -1
    bad_tau = (ctypes.c_double * 3)(0.7, -1.0, 1.0)
    assert lbmlib.lbm_batch_create(3, L, n, bad_tau, 1, 10, ctypes.byref(h)) == -1
    assert lbmlib.lbm_batch_create(3, L, n, tau, 1, 10, ctypes.byref(h)) == 0
    try:
        sb, wb, tn = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int64()
        assert lbmlib.lbm_batch_sizes(h, ctypes.byref(sb), ctypes.byref(wb), ctypes.byref(tn)) == 0
        assert tn.value == 83
        assert sb.value == 4 * 14 * (32 + 64 + 64)  # each problem padded to 32 floats
        assert lbmlib.lbm_batch_run(h, 1) == -6      # no state yet
        assert lbmlib.lbm_batch_set_block(h, 100, 0) == -1
        assert lbmlib.lbm_batch_set_block(h, 512, -1) == -1
        assert lbmlib.lbm_batch_set_block(h, 512, 2) == 0
        # watch ranges: 0 <= lo <= hi <= length per problem, both or neither
        IA = ctypes.c_int * 3
        assert lbmlib.lbm_batch_set_watch(h, IA(0, 5, 10), IA(10, 35, 33)) == 0
        assert lbmlib.lbm_batch_set_watch(h, IA(0, 5, 10), IA(11, 35, 33)) == -1  # hi > length
        assert lbmlib.lbm_batch_set_watch(h, IA(0, 6, 10), IA(10, 5, 33)) == -1   # lo > hi
        assert lbmlib.lbm_batch_set_watch(h, IA(-1, 0, 0), IA(10, 40, 33)) == -1  # lo < 0
        assert lbmlib.lbm_batch_set_watch(h, IA(0, 0, 0), None) == -1            # one of two
        assert lbmlib.lbm_batch_set_watch(h, None, None) == 0                   # whole problems
    finally:
        lbmlib.lbm_batch_destroy(h)


def test_node_reference_storage_sizes_and_limits(lbmlib):
    """Per-node reference storage (LBM_STORE_F16_NODE = 3, BF16_NODE = 4):
    the state buffer holds the 16-bit populations, then, 256-byte aligned, one
    16-byte record per node; STREAM on the 1-D and 2-D lattices only.  Host
    calls only."""
    sb, wb = ctypes.c_size_t(), ctypes.c_size_t()
    shape = (ctypes.c_int64 * 3)(100, 10, 1)
    bc = (ctypes.c_int * 3)(0, 0, 0)
    for storage, rest in ((3, 1), (4, 2)):
        sizes = {}
        for st in (storage, rest):
            rc, h = _create(lbmlib, 2, 3, 3, 2 / 3)  # D2Q49 + D1Q7
            assert rc == 0
            try:
                assert lbmlib.lbm_set_storage(h, st) == 0
                assert lbmlib.lbm_set_grid(h, shape, bc, ctypes.byref(sb), ctypes.byref(wb)) == 0
                sizes[st] = sb.value
            finally:
                lbmlib.lbm_destroy(h)
        S = 128 * 10  # pitch of 100 halves rounded up to 64, times Y
        assert sizes[rest] == 2 * 56 * S
        assert sizes[storage] == (2 * 56 * S + 255) // 256 * 256 + 16 * S
    # FD transport and D3Q343 are refused at lbm_set_grid
    rc, h = _create(lbmlib, 1, 1, 4, 2 / 3)
    try:
        assert lbmlib.lbm_set_mode(h, 1, 10) == 0
        assert lbmlib.lbm_set_storage(h, 3) == 0
        assert lbmlib.lbm_set_grid(h, (ctypes.c_int64 * 3)(64, 1, 1), bc, ctypes.byref(sb),
                                   ctypes.byref(wb)) == -1
    finally:
        lbmlib.lbm_destroy(h)
    rc, h = _create(lbmlib, 3, 4, 0, 2 / 3)
    try:
        assert lbmlib.lbm_set_storage(h, 4) == 0
        assert lbmlib.lbm_set_grid(h, (ctypes.c_int64 * 3)(8, 8, 8), bc, ctypes.byref(sb),
                                   ctypes.byref(wb)) == -1
        assert lbmlib.lbm_set_storage(h, 5) == -1  # unknown storage
    finally:
        lbmlib.lbm_destroy(h)
