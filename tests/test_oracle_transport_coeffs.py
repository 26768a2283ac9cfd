"""Chapman-Enskog transport coefficients of the scheme, measured on the oracle
from the decay of small periodic perturbations (Sec. III and the Appendix).

- Shear viscosity: a transverse wave u_y = U sin(kx) decays as exp(-nu k^2 t).
  The Appendix gives mu = P tau, i.e. kinematic nu = T tau.  With exact
  streaming (dt = dx/r) the time discretisation shifts it to T (tau - 1/2)
  per lattice step, the familiar lattice-BGK result; the paper's forward-Euler
  transport (FD mode) keeps T tau.
- Heat conduction: an isobaric temperature wave decays as exp(-chi k^2 t).
  The Appendix's kappa implies chi = T tau for every n.  Its decoupled
  rotational equation (Eq. EvoEtaJ) advects h with the fluid velocity only,
  so rotational energy is not conducted and the scheme itself gives
  chi = (D+2)/(D+n+2) T tau: this pins the oracle's h transport (advecting h
  with the particle velocity, or dropping it, would change the ratio).

Units: nodes and steps; xi = r e, so nu in nodes^2/step is T (tau - 1/2)/r^2
(STREAM) or T tau/(m r^2) (FD with dt = dx/(m r)).
"""
import numpy as np
import pytest


def decay_rate(series, start):
    ks = np.arange(len(series))
    return -np.polyfit(ks[start:], np.log(np.abs(series[start:])), 1)[0]


def shear_nu(orc, kind, n, tau, mode, m=10, X=32, Y=2, steps=200, U=1e-3):
    s = orc.Sim(kind, n, tau, (X, Y), (orc.PERIODIC, orc.PERIODIC), mode=mode, m_fd=m)
    x = (np.arange(X) + 0.5) / X
    u = np.zeros((2, Y, X))
    u[1] = U * np.sin(2 * np.pi * x)[None, :]
    s.set_macro(np.ones((Y, X)), u, np.ones((Y, X)))
    amp = []
    for _ in range(steps):
        _, uu, _ = s.moments()
        amp.append(np.sum(uu[1].reshape(Y, X)[0] * np.sin(2 * np.pi * x)))
        s.step(1)
    return decay_rate(np.array(amp), steps // 4) / (2 * np.pi / X) ** 2


def thermal_chi(orc, kind, n, tau, X=64, Y=2, steps=1000, eps=1e-3):
    s = orc.Sim(kind, n, tau, (X, Y), (orc.PERIODIC, orc.PERIODIC))
    x = (np.arange(X) + 0.5) / X
    T = 1 + eps * np.cos(2 * np.pi * x)
    s.set_macro(np.tile(1 / T, (Y, 1)), np.zeros((2, Y, X)), np.tile(T, (Y, 1)))
    amp = []
    for _ in range(steps):
        _, _, TT = s.moments()
        amp.append(np.sum((TT.reshape(Y, X)[0] - 1) * np.cos(2 * np.pi * x)))
        s.step(1)
    return decay_rate(np.array(amp), steps // 3) / (2 * np.pi / X) ** 2


@pytest.mark.parametrize("kind,n", [(2, 3), (3, 0)])
def test_shear_viscosity_stream(orc, kind, n):
    r = orc.lattice(kind)[0]
    tau = 0.8
    nu = shear_nu(orc, kind, n, tau, orc.STREAM)
    assert nu == pytest.approx((tau - 0.5) / r ** 2, rel=0.01)


def test_shear_viscosity_fd_is_the_papers(orc):
    """FD mode: mu = P tau (Appendix), nu = T tau per unit time."""
    r = orc.lattice(orc.D2Q37)[0]
    tau, m = 0.8, 10
    nu = shear_nu(orc, orc.D2Q37, 3, tau, orc.FD, m=m)
    assert nu == pytest.approx(tau / (m * r ** 2), rel=0.02)


@pytest.mark.parametrize("n", [0, 1, 3])
def test_thermal_diffusivity_of_the_scheme(orc, n):
    r = orc.lattice(orc.D2Q49)[0]
    tau, D = 0.8, 2
    chi = thermal_chi(orc, orc.D2Q49, n, tau)
    scheme = (D + 2) / (D + n + 2) * (tau - 0.5) / r ** 2
    assert chi == pytest.approx(scheme, rel=0.02)
    if n > 0:  # the Appendix's kappa (chi = T tau for all n) does not hold
        assert abs(chi / ((tau - 0.5) / r ** 2) - 1) > 0.1
