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


def test_d3q343_weights_are_the_d1q7_tensor_product(lbmlib):
    """The D3Q343 step forms each weight as (w_a w_b) w_c from the D1Q7
    weights (the in-plane factor an immediate, the plane factor per plane),
    so the library's D3Q343 set must be exactly that product with the index
    i = (c * 7 + b) * 7 + a for e = (a - 3, b - 3, c - 3).  Host calls only."""
    from paper_1606_06107_gb300 import lbm
    r1, e1, w1 = lbm.lattice_info("D1Q7")
    r3, e3, w3 = lbm.lattice_info("D3Q343")
    assert r3 == r1
    assert np.array_equal(e1[:, 0], np.arange(-3, 4))
    for i in range(343):
        a, b, c = i % 7, (i // 7) % 7, i // 49
        assert tuple(e3[i]) == (a - 3, b - 3, c - 3)
        assert abs(w3[i] - w1[a] * w1[b] * w1[c]) <= 1e-15 * w3[i]


def test_row_quartic_expansion():
    """The D3Q343 16-bit step evaluates the equilibrium polynomial of a row
    (e_y, e_z fixed) as a quartic in e_x: with c = C0 + e_x v and s = S0 + r2
    e_x^2, P = A0(s) + A1(s) c + A2(s) c^2 + k6 c^3 + k24 c^4 equals b0 + b1 e_x
    + b2 e_x^2 + b3 e_x^3 + b4 e_x^4 with the coefficients written out in the
    kernel's comments (A0 = a00 + a01 s + a02 s^2, A1 = a10 + a11 s, A2 = a20
    + a21 s at s = S0).  Checked here in double precision on random
    coefficients at the seven e_x of a row, and the pair form E +- O."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        a00, a01, a02, a10, a11, a20, a21, k6, k24 = rng.normal(size=9)
        C0, S0, v = rng.normal(size=3)
        r2 = 1.0 + rng.random()

        def P(t):
            s, c = S0 + r2 * t * t, C0 + v * t
            return (a00 + a01 * s + a02 * s * s + (a10 + a11 * s) * c + (a20 + a21 * s) * c * c
                    + k6 * c ** 3 + k24 * c ** 4)

        A0, A1, A2 = a00 + a01 * S0 + a02 * S0 * S0, a10 + a11 * S0, a20 + a21 * S0
        b0 = A0 + C0 * (A1 + C0 * (A2 + C0 * (k6 + C0 * k24)))
        b1 = v * (A1 + C0 * (2 * A2 + C0 * (3 * k6 + 4 * k24 * C0)))
        b2 = r2 * (a01 + 2 * a02 * S0 + a11 * C0 + a21 * C0 * C0) + v * v * (A2 + C0 * (3 * k6 + 6 * k24 * C0))
        b3 = v * (r2 * (a11 + 2 * a21 * C0) + v * v * (k6 + 4 * k24 * C0))
        b4 = a02 * r2 * r2 + a21 * r2 * v * v + k24 * v ** 4
        for t in range(-3, 4):
            want = P(t)
            got = b0 + b1 * t + b2 * t * t + b3 * t ** 3 + b4 * t ** 4
            assert abs(got - want) <= 1e-11 * (1 + abs(want)), (t, got, want)
        for k in (1, 2, 3):
            E, O = b0 + b2 * k * k + b4 * k ** 4, k * (b1 + b3 * k * k)
            assert abs(E + O - P(k)) <= 1e-11 * (1 + abs(P(k)))
            assert abs(E - O - P(-k)) <= 1e-11 * (1 + abs(P(-k)))
