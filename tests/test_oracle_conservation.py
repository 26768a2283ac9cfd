"""Pins for the oracle's global conservation sums (orc_conservation).

Sec. II defines the conserved totals: the mass sum of rho, the momentum sum
of rho u and the total energy of Eq. Total, rho (E + u^2/2) with the
translational part sum_i g_i xi_i^2 / 2 and the rotational part rho times
sum_j h_j (n/2) eta_j^2 (the rotational distribution is normalised,
sum_j h_j = 1, Eq. FFeqRhoEta).  These tests compute the same four numbers
without the oracle's node code: the populations are gathered with NumPy
index arithmetic (pull pre-image in STREAM mode, the stored values in FD
mode, wrap or clamp at the ends) and summed with the velocities of the
lattice, and, separately, from the oracle's rho, u, T through Eq. Total.
A sum that drops the density on the rotational energy, uses the wrong pull
direction at clamped ends, or takes a signed instead of an absolute
deviation of sum_j h_j fails one of them."""
import zlib

import numpy as np
import pytest


def _random_state(orc, kind, n, shape, rng):
    """Positive, non-equilibrium populations; each node's h sums to 1."""
    r, e, w, _ = orc.lattice(kind)
    N = int(np.prod(shape))
    rho = 1.0 + 0.3 * rng.random(N)
    ft = w[:, None] * rho[None, :] * (1.0 + 0.2 * rng.standard_normal((len(w), N)))
    fr = None
    if n > 0:
        fr = orc.heq(1.0)[:, None] * (1.0 + 0.3 * rng.random((7, N)))
        fr /= fr.sum(axis=0, keepdims=True)
    return r, e, ft, fr


def _gather(ft, e, shape, bc, mode):
    """g_i(x) = ft_i(bc(x - e_i)) (STREAM) or ft_i(x) (FD), x fastest."""
    if mode == 1:
        return ft.copy()
    D = len(shape)
    grids = np.meshgrid(*[np.arange(s) for s in shape[::-1]], indexing="ij")
    coords = grids[::-1]  # coords[a] has the array shape (Z.., Y, X)
    out = np.empty_like(ft)
    for i in range(ft.shape[0]):
        flat = np.zeros(coords[0].shape, dtype=np.int64)
        stride = 1
        for a in range(D):
            src = coords[a] - e[i, a]
            src = np.mod(src, shape[a]) if bc[a] == 0 else np.clip(src, 0, shape[a] - 1)
            flat += src * stride
            stride *= shape[a]
        out[i] = ft[i][flat.ravel()]
    return out


@pytest.mark.parametrize("kind,shape,n,bc,mode", [
    ("D2Q49", (7, 5), 3, (0, 0), 0),
    ("D2Q49", (6, 5), 3, (1, 0), 0),
    ("D2Q37", (5, 6), 0, (1, 1), 0),
    ("D1Q7", (11,), 4, (1,), 0),
    ("D1Q7", (9,), 2, (0,), 1),
    ("D2Q49", (5, 4), 3, (1, 1), 1),
])
def test_conservation_against_numpy_sums(orc, kind, shape, n, bc, mode):
    code = getattr(orc, kind)
    rng = np.random.default_rng(zlib.crc32(repr((kind, shape, n, bc, mode)).encode()))
    r, e, ft, fr = _random_state(orc, code, n, shape, rng)
    D = len(shape)
    sim = orc.Sim(code, n, 0.8, shape, bc, mode=mode)
    sim.set_state(ft, fr)
    got = sim.conservation()

    g = _gather(ft, e, shape, bc, mode)
    xi = r * e[:, :D].astype(float)                       # xi_i = r e_i
    rho = g.sum(axis=0)
    mom = xi.T @ g                                        # [D, N]
    K = 0.5 * ((xi ** 2).sum(axis=1) @ g)                 # sum_i g_i xi_i^2 / 2
    if n > 0:
        eta2 = (r * (np.arange(7) - 3.0)) ** 2            # D1Q7 eta_j^2
        R = 0.5 * n * (eta2 @ fr)                         # per unit mass
        hdev = np.abs(fr.sum(axis=0) - 1.0).max()
    else:
        R = np.zeros_like(rho)
        hdev = 0.0
    want = np.concatenate([[rho.sum()], mom.sum(axis=1), [(K + rho * R).sum(), hdev]])
    assert got.shape == (3 + D,)
    np.testing.assert_allclose(got[:-1], want[:-1], rtol=1e-13, atol=1e-13)
    assert got[-1] == pytest.approx(want[-1], abs=1e-14)

    # the same totals from the oracle's rho, u, T through Eq. Total:
    # rho (E + u^2/2) with E = (D + n) T / 2
    rr, uu, TT = sim.moments()
    energy = (rr * ((D + n) * TT / 2.0 + 0.5 * (uu ** 2).sum(axis=0))).sum()
    assert got[0] == pytest.approx(rr.sum(), rel=1e-13)
    np.testing.assert_allclose(got[1:1 + D], (rr[None, :] * uu).sum(axis=1), rtol=1e-12,
                               atol=1e-12)
    assert got[1 + D] == pytest.approx(energy, rel=1e-12)
    # a rotational energy summed without rho would differ measurably
    if n > 0:
        assert abs((K + R).sum() - got[1 + D]) > 1e-3 * abs(got[1 + D])


def test_conservation_planted_h_deviation(orc):
    """max_x |sum_j h_j - 1| picks the largest absolute deviation: one node
    raised by 3e-3 and another lowered by 5e-3 give exactly 5e-3."""
    rng = np.random.default_rng(5)
    shape, n = (8, 6), 3
    r, e, ft, fr = _random_state(orc, orc.D2Q49, n, shape, rng)
    fr[:, 10] *= 1.0 + 3e-3
    fr[:, 31] *= 1.0 - 5e-3
    sim = orc.Sim(orc.D2Q49, n, 0.8, shape, (0, 0))
    sim.set_state(ft, fr)
    assert sim.conservation()[-1] == pytest.approx(5e-3, abs=1e-14)
    fr[:, 31] /= 1.0 - 5e-3
    sim.set_state(ft, fr)
    assert sim.conservation()[-1] == pytest.approx(3e-3, abs=1e-14)
