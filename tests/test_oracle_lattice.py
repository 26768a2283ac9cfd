"""Pins for the oracle's lattices (Tables I and II) against what the paper and
the mathematics fix: the Gauss-Hermite moment equations (closed form), the
printed tables, the equal-r requirement, and the group structure of D2Q37."""
import itertools
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gauss_1d(k):
    """E[x^k] for x ~ N(0, 1): 0 for odd k, (k-1)!! for even k."""
    if k % 2:
        return 0.0
    return float(np.prod(np.arange(k - 1, 0, -2))) if k > 0 else 1.0


@pytest.mark.parametrize("kind,degree", [(1, 9), (2, 9), (3, 9)])
def test_lattice_reproduces_normal_moments(orc, kind, degree):
    """Every monomial moment up to the quadrature degree equals the unit
    normal's (Tables I/II are Gauss-Hermite quadratures)."""
    r, e, w, _ = orc.lattice(kind)
    xi = r * e.astype(float)
    D = orc.LATTICE_DIM[kind]
    worst = 0.0
    for powers in itertools.product(range(degree + 1), repeat=D):
        if sum(powers) > degree:
            continue
        mono = np.prod([xi[:, a] ** powers[a] for a in range(D)], axis=0)
        lat = float(np.sum(w * mono))
        exact = float(np.prod([gauss_1d(p) for p in powers]))
        worst = max(worst, abs(lat - exact) / max(1.0, abs(exact)))
    assert worst < 1e-13


def test_d1q7_matches_table_II(orc):
    gold = json.load(open(os.path.join(GOLD, "tables_I_II.json")))
    r, e, w, _ = orc.lattice(orc.D1Q7)
    assert e[:, 0].tolist() == [-3, -2, -1, 0, 1, 2, 3]
    for k, wp in zip(gold["D1Q7"]["abs_e"], gold["D1Q7"]["w"]):
        ours = w[e[:, 0] == k][0]
        assert abs(ours - wp) / wp < 1e-7
    assert abs(r - gold["r"]) / gold["r"] < 1e-8


def test_d2q37_matches_table_I(orc):
    gold = json.load(open(os.path.join(GOLD, "tables_I_II.json")))["D2Q37"]
    r, e, w, _ = orc.lattice(orc.D2Q37)
    assert len(w) == 37 and np.all(e[:, 2] == 0)
    for (a, b), k, wp in zip(gold["groups"], gold["members"], gold["w"]):
        key = (max(a, b), min(a, b))
        members = [i for i in range(37)
                   if (max(abs(e[i, 0]), abs(e[i, 1])), min(abs(e[i, 0]), abs(e[i, 1]))) == key]
        assert len(members) == k
        assert np.allclose(w[members], w[members[0]], rtol=0, atol=0)
        # printed to ~9 digits, whose sum misses 1 by 1e-8: agree within 5e-9
        assert abs(w[members[0]] - wp) < 5e-9


def test_equal_scaling_factor(orc):
    """Sec. IV: the g and h lattices must share r; both solves agree."""
    r37 = orc.lattice(orc.D2Q37)[0]
    r7 = orc.lattice(orc.D1Q7)[0]
    assert abs(r37 - r7) < 1e-14


def test_tensor_lattice_is_product(orc):
    r7, e7, w7, _ = orc.lattice(orc.D1Q7)
    r49, e49, w49, _ = orc.lattice(orc.D2Q49)
    assert r49 == r7
    for i in range(49):
        ex, ey = e49[i, 0], e49[i, 1]
        assert i == (ey + 3) * 7 + (ex + 3)
        assert w49[i] == pytest.approx(w7[ex + 3] * w7[ey + 3], rel=1e-15)


def test_order_is_ez_ey_ex_ascending(orc):
    for kind in (1, 2, 3):
        e = orc.lattice(kind)[1]
        keys = [(z, y, x) for x, y, z in e]
        assert keys == sorted(keys)
