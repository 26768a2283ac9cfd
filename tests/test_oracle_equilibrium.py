"""Pins for the oracle's equilibria (Sec. IV), moments (Sec. V steps 3-4,
Eq. T) and collision (Eq. DisEvolI / EvoEtaJ relaxation terms).

The defining property of a 4th-order Hermite equilibrium is that its lattice
moments equal the Maxwellian's up to order 4; the Maxwellian's raw moments
have a closed form.  A second, independent evaluation contracts explicit
Hermite tensors.  The collision must conserve mass, momentum and the total
(translational + rotational) energy exactly."""
import itertools

import numpy as np
import pytest


def normal_raw_1d(k, mu, var):
    """E[x^k] for x ~ N(mu, var), k <= 4 (closed form)."""
    return [1.0, mu, mu * mu + var, mu ** 3 + 3 * mu * var,
            mu ** 4 + 6 * mu * mu * var + 3 * var * var][k]


def lattice_moments(orc, kind, f):
    r, e, w, _ = orc.lattice(kind)
    xi = r * e.astype(float)
    D = orc.LATTICE_DIM[kind]
    out = {}
    for powers in itertools.product(range(5), repeat=D):
        if sum(powers) <= 4:
            mono = np.prod([xi[:, a] ** powers[a] for a in range(D)], axis=0)
            out[powers] = float(np.sum(f * mono))
    return out


CASES = [(1.0, (0.0, 0.0), 1.0), (1.3, (0.3, -0.2), 0.8), (0.7, (-0.45, 0.1), 1.25),
         (2.0, (0.05, 0.4), 0.6)]


@pytest.mark.parametrize("kind", [1, 2, 3])
@pytest.mark.parametrize("rho,u,theta", CASES)
def test_geq_moments_equal_maxwellian(orc, kind, rho, u, theta):
    D = orc.LATTICE_DIM[kind]
    u = u[:D]
    g = orc.geq(kind, rho, u, theta)
    mom = lattice_moments(orc, kind, g)
    for powers, val in mom.items():
        exact = rho * np.prod([normal_raw_1d(powers[a], u[a], theta) for a in range(D)])
        assert abs(val - exact) < 1e-12 * max(1.0, abs(exact)), powers


def test_printed_equilibrium_fails_the_pin(orc):
    """The equilibrium as printed in Sec. IV (garbled a2, a3, a4 terms) does not
    reproduce the Maxwellian's moments, so the moment pin discriminates the
    reading the oracle takes from the literal text."""
    kind = orc.D2Q37
    r, e, w, _ = orc.lattice(kind)
    rho, u, th = 1.3, np.array([0.3, -0.2]), 0.8
    xi = r * e[:, :2].astype(float)
    c = xi @ u
    u2 = u @ u
    s = (xi * xi).sum(1)
    t = th - 1.0
    D = 2
    a2 = c * c + t * (th * th - D) - u2
    a3 = c * (c * c - 3 * u2 + 3 * t * (u2 - D - 2))
    a4 = (c ** 4 - 6 * c * c * u2 + 3 * u2 * u2 + 6 * t * (c * c * (u2 - D - 4) + (D + 2 - u2) * s)
          + 3 * t * t * (u2 * u2 - 2 * (D + 2) * u2 + D * (D + 2)))
    g_lit = w * rho * (1 + c + a2 / 2 + a3 / 6 + a4 / 24)
    mom = lattice_moments(orc, kind, g_lit)
    worst = max(abs(v - rho * np.prod([normal_raw_1d(p[a], u[a], th) for a in range(2)]))
                for p, v in mom.items())
    assert worst > 1e-3


def hermite_tensors(x, D):
    """Probabilists' Hermite tensors H0..H4 of a D-vector x (explicit)."""
    I = np.eye(D)
    H1 = x
    H2 = np.einsum("i,j->ij", x, x) - I
    H3 = (np.einsum("i,j,k->ijk", x, x, x) - np.einsum("i,jk->ijk", x, I)
          - np.einsum("j,ik->ijk", x, I) - np.einsum("k,ij->ijk", x, I))
    xx = np.einsum("i,j->ij", x, x)
    H4 = (np.einsum("i,j,k,l->ijkl", x, x, x, x)
          - np.einsum("ij,kl->ijkl", xx, I) - np.einsum("ik,jl->ijkl", xx, I)
          - np.einsum("il,jk->ijkl", xx, I) - np.einsum("jk,il->ijkl", xx, I)
          - np.einsum("jl,ik->ijkl", xx, I) - np.einsum("kl,ij->ijkl", xx, I)
          + np.einsum("ij,kl->ijkl", I, I) + np.einsum("ik,jl->ijkl", I, I)
          + np.einsum("il,jk->ijkl", I, I))
    return H1, H2, H3, H4


def hermite_coeffs(u, theta, D):
    """Hermite coefficients a^(k)/rho of a Gaussian with mean u, variance theta."""
    I = np.eye(D)
    t = theta - 1.0
    a1 = u
    a2 = np.einsum("i,j->ij", u, u) + t * I
    a3 = (np.einsum("i,j,k->ijk", u, u, u) + t * (np.einsum("i,jk->ijk", u, I)
          + np.einsum("j,ik->ijk", u, I) + np.einsum("k,ij->ijk", u, I)))
    uu = np.einsum("i,j->ij", u, u)
    a4 = (np.einsum("i,j,k,l->ijkl", u, u, u, u)
          + t * (np.einsum("ij,kl->ijkl", uu, I) + np.einsum("ik,jl->ijkl", uu, I)
                 + np.einsum("il,jk->ijkl", uu, I) + np.einsum("jk,il->ijkl", uu, I)
                 + np.einsum("jl,ik->ijkl", uu, I) + np.einsum("kl,ij->ijkl", uu, I))
          + t * t * (np.einsum("ij,kl->ijkl", I, I) + np.einsum("ik,jl->ijkl", I, I)
                     + np.einsum("il,jk->ijkl", I, I)))
    return a1, a2, a3, a4


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_geq_equals_tensor_contraction(orc, kind):
    D = orc.LATTICE_DIM[kind]
    r, e, w, _ = orc.lattice(kind)
    rho, u, theta = 1.1, np.array([0.25, -0.35])[:D], 0.9
    a1, a2, a3, a4 = hermite_coeffs(u, theta, D)
    ref = np.empty(len(w))
    for i in range(len(w)):
        x = r * e[i, :D].astype(float)
        H1, H2, H3, H4 = hermite_tensors(x, D)
        ref[i] = w[i] * rho * (1 + np.sum(a1 * H1) + np.sum(a2 * H2) / 2
                               + np.sum(a3 * H3) / 6 + np.sum(a4 * H4) / 24)
    assert np.allclose(orc.geq(kind, rho, u, theta), ref, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("theta", [0.6, 1.0, 1.4])
def test_heq_moments(orc, theta):
    """h^eq on D1Q7: unit mass, variance theta and 4th moment 3 theta^2
    (Eq. FeqRhoEta, FeqEEta)."""
    r, e, w, _ = orc.lattice(orc.D1Q7)
    eta = r * e[:, 0]
    h = orc.heq(theta)
    assert abs(h.sum() - 1) < 1e-14
    assert abs((h * eta ** 2).sum() - theta) < 1e-13
    assert abs((h * eta ** 4).sum() - 3 * theta ** 2) < 1e-12
    assert abs((h * eta).sum()) < 1e-14 and abs((h * eta ** 3).sum()) < 1e-13


@pytest.mark.parametrize("kind,n", [(1, 4), (2, 3), (3, 3), (3, 0), (1, 2)])
def test_moments_of_equilibrium_round_trip(orc, kind, n):
    D = orc.LATTICE_DIM[kind]
    rho, u, T = 0.9, np.array([0.2, -0.1])[:D], 1.15
    g = orc.geq(kind, rho, u, T)
    h = orc.heq(T)
    rr, uu, TT, K, R = orc.node_moments(kind, n, g, h)
    assert abs(rr - rho) < 1e-14 and np.allclose(uu, u, atol=1e-14) and abs(TT - T) < 1e-13
    assert abs(K - rho * (0.5 * u @ u + 0.5 * D * T)) < 1e-13   # Eq. FeqEXi
    assert abs(R - 0.5 * n * T) < 1e-13                         # Eq. FeqEEta


def perturbed(orc, kind, rng):
    D = orc.LATTICE_DIM[kind]
    g = orc.geq(kind, 1.1, rng.uniform(-0.2, 0.2, D), 0.95)
    g *= 1 + 0.05 * rng.standard_normal(g.size)
    h = orc.heq(1.05) * (1 + 0.05 * rng.standard_normal(7))
    h /= h.sum()
    return g, h


@pytest.mark.parametrize("kind,n", [(1, 4), (2, 3), (3, 3), (3, 0)])
def test_collision_invariants(orc, kind, n):
    """BGK toward the decoupled equilibria conserves rho, rho u and the total
    energy K + rho R (Eq. Total) to rounding, and keeps sum_j h_j = 1; the
    translational energy alone is exchanged with the rotational one."""
    rng = np.random.default_rng(3)
    g, h = perturbed(orc, kind, rng)
    go, ho = orc.collide_node(kind, n, 1.5, g, h)
    r0, u0, T0, K0, R0 = orc.node_moments(kind, n, g, h)
    r1, u1, T1, K1, R1 = orc.node_moments(kind, n, go, ho)
    assert abs(r1 - r0) < 1e-14 * r0
    assert np.allclose(r1 * u1, r0 * u0, atol=1e-14)
    assert abs((K1 + r1 * R1) - (K0 + r0 * R0)) < 1e-13
    if n > 0:
        assert abs(ho.sum() - 1) < 1e-14
        assert abs(K1 - K0) > 1e-6   # exchange between g and h energies


def test_full_relaxation_reaches_equilibrium(orc):
    """omega = 1 maps a node onto its own equilibrium."""
    rng = np.random.default_rng(5)
    g, h = perturbed(orc, orc.D2Q49, rng)
    go, ho = orc.collide_node(orc.D2Q49, 3, 1.0, g, h)
    rho, u, T, _, _ = orc.node_moments(orc.D2Q49, 3, g, h)
    assert np.allclose(go, orc.geq(orc.D2Q49, rho, u, T), rtol=1e-13, atol=1e-16)
    assert np.allclose(ho, orc.heq(T), rtol=1e-13, atol=1e-16)
