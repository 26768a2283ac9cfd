"""Pins for the oracle's transport: the third-order upwind stencil (Sec. V),
pull streaming on the lattice, boundaries, and the global invariants a
periodic domain must keep (mass and momentum exactly; sum_j h_j = 1)."""
import numpy as np
import pytest

from paper_1606_06107_gb300 import workloads


@pytest.mark.parametrize("coeffs", [(1.0, 0, 0, 0), (0.3, 2.0, 0, 0), (0, 0, 1.0, 0),
                                    (0.1, -0.7, 0.4, 1.3)])
def test_upwind_exact_for_cubics(orc, coeffs):
    """Both one-sided stencils differentiate polynomials of degree <= 3
    exactly: nu * dF/dx at x=0 for F(x) = c0 + c1 x + c2 x^2 + c3 x^3."""
    x = np.arange(-2, 3, dtype=float)
    F = sum(c * x ** k for k, c in enumerate(coeffs))
    dF = coeffs[1]
    for nu in (0.7, -0.4):
        assert orc.upwind(nu, F) == pytest.approx(nu * dF, abs=1e-13)


def test_upwind_third_order(orc):
    """Error on a smooth wave falls as h^3 (third order, Sec. V)."""
    errs = []
    for h in (0.1, 0.05, 0.025):
        x = 0.3 + h * np.arange(-2, 3)
        approx = orc.upwind(1.0, np.sin(x)) / h
        errs.append(abs(approx - np.cos(0.3)))
    ratios = [errs[k] / errs[k + 1] for k in range(2)]
    assert all(7.0 < q < 9.0 for q in ratios), ratios


def test_pull_stream_direction(orc):
    """One STREAM step equals: g_i(x) = ft_i(x - e_i) (np.roll on a periodic
    grid), then the node-local BGK of each pulled node.  Rotational fr with
    zero velocity has no convection."""
    kind, n, tau = orc.D2Q49, 3, 0.8
    X, Y = 9, 7
    rng = np.random.default_rng(11)
    sim = orc.Sim(kind, n, tau, (X, Y), (orc.PERIODIC, orc.PERIODIC))
    r, e, w, _ = orc.lattice(kind)
    ft = np.empty((49, Y, X))
    for i in range(49):
        ft[i] = w[i] * (1 + 0.05 * rng.standard_normal((Y, X)))
    # make the momentum vanish at every pulled node so fr has no convection:
    # a uniform-in-space rotational state makes the upwind term zero anyway
    fr = np.tile(orc.heq(1.0)[:, None, None], (1, Y, X))
    sim.set_state(ft.reshape(49, -1), fr.reshape(7, -1))
    sim.step(1)
    got = sim.ft.reshape(49, Y, X)
    g = np.stack([np.roll(ft[i], shift=(e[i, 1], e[i, 0]), axis=(0, 1)) for i in range(49)])
    for y in range(Y):
        for x in range(X):
            go, _ = orc.collide_node(kind, n, 1.0 / tau, g[:, y, x], fr[:, y, x])
            assert np.allclose(got[:, y, x], go, rtol=1e-13, atol=1e-17)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
def test_uniform_state_is_fixed_point(orc, mode, bc):
    sim = orc.Sim(orc.D2Q37, 3, 2 / 3, (11, 6), (bc, bc), mode=mode, m_fd=4)
    rho = np.full((6, 11), 1.2)
    u = np.stack([np.full((6, 11), 0.1), np.full((6, 11), -0.05)])
    T = np.full((6, 11), 0.9)
    sim.set_macro(rho, u, T)
    ft0, fr0 = sim.state()
    sim.step(3)
    ft1, fr1 = sim.state()
    assert np.allclose(ft1, ft0, rtol=1e-13, atol=1e-16)
    assert np.allclose(fr1, fr0, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("kind,mode", [(3, 0), (2, 0), (1, 0), (3, 1), (1, 1)])
def test_periodic_global_conservation(orc, kind, mode):
    """Pull streaming is a permutation and the upwind stencil telescopes, so a
    periodic domain keeps total mass and momentum to rounding; sum_j h_j = 1
    holds at every node (Eq. FFeqRhoEta).  Total energy is not conserved
    exactly because h is advected in non-conservative form (Eq. EvoEtaJ)."""
    D = orc.LATTICE_DIM[kind]
    shape = (24,) if D == 1 else (16, 12)
    name = {1: "D1Q7", 2: "D2Q37", 3: "D2Q49"}[kind]
    wl = workloads.smooth_random(shape, seed=2, kind=name, n=3)
    sim = orc.Sim(kind, wl.n, wl.tau, shape, (orc.PERIODIC,) * D, mode=mode, m_fd=5)
    sim.set_macro(wl.rho, wl.u, wl.T)
    c0 = sim.conservation()
    sim.step(20)
    c1 = sim.conservation()
    assert abs(c1[0] - c0[0]) < 1e-12 * c0[0]
    for a in range(D):
        assert abs(c1[1 + a] - c0[1 + a]) < 1e-12 * c0[0]
    assert c1[2 + D] < 1e-13
    assert abs(c1[1 + D] - c0[1 + D]) < 1e-2 * c0[1 + D]


def test_set_macro_round_trip(orc):
    """The pull pre-image initial state gives back the input moments."""
    wl = workloads.smooth_random((20, 10), seed=4, kind="D2Q49", n=3)
    sim = orc.Sim(orc.D2Q49, 3, wl.tau, wl.shape, (orc.PERIODIC,) * 2)
    sim.set_macro(wl.rho, wl.u, wl.T)
    rho, u, T = sim.moments()
    assert np.allclose(rho, wl.rho.ravel(), atol=1e-14)
    assert np.allclose(u, wl.u.reshape(2, -1), atol=1e-14)
    assert np.allclose(T, wl.T.ravel(), atol=1e-13)


def test_copy_boundary_keeps_edges(orc):
    """Copy (zero-gradient) ends on a uniform state change nothing, and a
    left-moving disturbance does not wrap around to the right end."""
    X = 40
    sim = orc.Sim(orc.D1Q7, 4, 2 / 3, (X,), (orc.COPY,))
    rho = np.ones(X)
    rho[:3] = 1.05
    sim.set_macro(rho, np.zeros((1, X)), np.ones(X))
    sim.step(5)
    r, u, T = sim.moments()
    assert np.allclose(r[-10:], 1.0, atol=1e-12)
