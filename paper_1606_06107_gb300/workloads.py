"""Seeded synthetic initial conditions for the shock-tube family of problems.

These generators produce macroscopic fields (rho, u, T) only; they hold none
of the lattice Boltzmann arithmetic and are shared by the CUDA path, the
oracle and the benchmark so that both sides start from the same inputs.
Fields are NumPy float64 arrays, x fastest: rho and T have shape ``shape[::-1]``
(i.e. [Z][Y][X]), u has shape ``(D,) + shape[::-1]``.

The equation of state P = rho T (dimensionless, theta0 = 1) converts a stated
pressure into a temperature.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Workload:
    name: str
    kind: str           # "D1Q7", "D2Q37", "D2Q49", "D3Q343"
    n: int              # rotational degrees of freedom
    tau: float          # relaxation time in lattice steps
    shape: tuple        # (X,), (X, Y) or (X, Y, Z)
    bc: tuple           # per axis: "periodic" or "copy"
    rho: np.ndarray
    u: np.ndarray
    T: np.ndarray
    steps: int
    note: str = ""

    @property
    def D(self) -> int:
        return len(self.shape)

    @property
    def nodes(self) -> int:
        return int(np.prod(self.shape))

    @property
    def gamma(self) -> float:
        return (self.D + self.n + 2.0) / (self.D + self.n)


def _two_state_1d(X, left, right):
    """Diaphragm at mid-domain: node centres x_i = (i + 1/2)/X, left state for i < X/2."""
    i = np.arange(X)
    is_left = i < X // 2
    rho = np.where(is_left, left[0], right[0]).astype(np.float64)
    p = np.where(is_left, left[2], right[2]).astype(np.float64)
    u = np.where(is_left, left[1], right[1]).astype(np.float64)
    return rho, u, p / rho


def sod_1d(X: int = 1000, steps: int = 2000) -> Workload:
    """Sod's shock tube in 1-D: left rho=1, p=1, u=0; right rho=0.125, p=0.1, u=0;
    gamma = 1.4 (D=1, n=4), tau = 2/3, copy (zero-gradient) ends."""
    rho, u, T = _two_state_1d(X, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    return Workload("sod_1d", "D1Q7", 4, 2.0 / 3.0, (X,), ("copy",), rho, u[None], T,
                    steps)


def stream_tube(X: int = 1000, Y: int = 1, kind: str = "D1Q7", steps: int = 200,
                rho_r: float = 0.25, p_r: float = 0.2) -> Workload:
    """A Sod-type tube with Sod's temperature ratio 0.8: left rho=1, p=1,
    u=0; right rho=rho_r, p=p_r, u=0.  The default (density ratio 4,
    pressure ratio 5) is the strongest such tube the STREAM transport keeps
    finite in double precision; rho_r=0.4, p_r=0.32 (ratios 2.5 and 3.1) the
    strongest it keeps finite in float32 for 400 steps.  gamma = 1.4 with
    n = 4 on D1Q7, or (kind "D2Q49", Y rows, periodic in y) gamma = 4/3 with
    n = 4; tau = 2/3, copy ends in x.  200 steps reach t = 200/(X r) = 0.167."""
    rho1, u1, T1 = _two_state_1d(X, (1.0, 0.0, 1.0), (rho_r, 0.0, p_r))
    if kind == "D1Q7":
        return Workload("stream_tube", kind, 4, 2.0 / 3.0, (X,), ("copy",), rho1, u1[None], T1,
                        steps)
    rho = np.tile(rho1, (Y, 1))
    T = np.tile(T1, (Y, 1))
    u = np.zeros((2, Y, X))
    return Workload("stream_tube", kind, 4, 2.0 / 3.0, (X, Y), ("copy", "periodic"), rho, u, T,
                    steps)


def paper_tube_2d(X: int = 1000, Y: int = 16, kind: str = "D2Q37",
                  steps: int = 180) -> Workload:
    """The paper's own validation run (Sec. VI): 1000 x 16, left rho=4, T=1;
    right rho=1, T=1; u=0; gamma=1.4 (D=2, n=3); tau=2/3; periodic in y and
    open (copy) ends in x."""
    rho1, u1, T1 = _two_state_1d(X, (4.0, 0.0, 4.0), (1.0, 0.0, 1.0))
    rho = np.tile(rho1, (Y, 1))
    T = np.tile(T1, (Y, 1))
    u = np.zeros((2, Y, X))
    return Workload("paper_tube_2d", kind, 3, 2.0 / 3.0, (X, Y), ("copy", "periodic"),
                    rho, u, T, steps)


def riemann_2d(X: int = 2048, Y: int = 2048, seed: int = 0, kind: str = "D2Q49",
               steps: int = 5000, mild: bool = False, band=None) -> Workload:
    """Four-quadrant 2-D Riemann problem, gamma=1.4 (D=2, n=3), tau=2/3,
    periodic.  Per quadrant, drawn from the seed: rho ~ U[0.1, 1.5],
    p ~ U[0.03, 1.5] and a velocity of uniform direction with |u| ~ U[0, 0.5].

    ``mild=True`` is the stable-envelope variant: rho ~ U[0.8, 1.2],
    T ~ U[0.8, 1.2], |u| ~ U[0, 0.1].  The stated draws reach T = p/rho of
    0.02..15 and density ratios near 10, where the scheme goes non-finite
    within a few steps; and the forward-Euler upwind advection of h is
    unstable once |u| reaches ~0.5 (diagonal) in 2-D, which stronger quadrant
    contrasts produce after a few thousand steps.

    ``band=(rho_lo, rho_hi, T_lo, T_hi, umax)`` draws rho ~ U[rho_lo, rho_hi],
    T ~ U[T_lo, T_hi] and |u| ~ U[0, umax] per quadrant instead (the same
    sequence of draws as ``mild``).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if band is not None:
        rho_q = rng.uniform(band[0], band[1], 4)
        T_q = rng.uniform(band[2], band[3], 4)
        umax = band[4]
    elif mild:
        rho_q = rng.uniform(0.8, 1.2, 4)
        T_q = rng.uniform(0.8, 1.2, 4)
        umax = 0.1
    else:
        rho_q = rng.uniform(0.1, 1.5, 4)
        T_q = rng.uniform(0.03, 1.5, 4) / rho_q
        umax = 0.5
    ang = rng.uniform(0.0, 2.0 * np.pi, 4)
    rad = rng.uniform(0.0, umax, 4)
    ux_q = rad * np.cos(ang)
    uy_q = rad * np.sin(ang)
    xs = np.arange(X) >= X // 2
    ys = np.arange(Y) >= Y // 2
    quad = (ys[:, None].astype(int) * 2 + xs[None, :].astype(int))  # [Y, X] in 0..3
    rho = rho_q[quad]
    T = T_q[quad]
    u = np.stack([ux_q[quad], uy_q[quad]])
    name = "riemann_2d_band" if band is not None else ("riemann_2d_mild" if mild else "riemann_2d")
    return Workload(name, kind, 3, 2.0 / 3.0, (X, Y), ("periodic", "periodic"),
                    rho, u, T, steps)


# The widest quadrant band that stays finite through 5000 STREAM steps at
# 2048^2 for seeds 0-3 (rho ~ U[0.8, 1.2], T ~ U[0.6, 1.4], |u| <= 0.1).
# Measured at the edges: T in [0.5, 1.5] fails for one seed of four near step
# 5000, rho in [0.5, 1.5] for two (by steps 750 and 2750), |u| <= 0.2 for one
# (by step 2750) and |u| <= 0.3 for three (by step 500).
WIDE_BAND = (0.8, 1.2, 0.6, 1.4, 0.1)


def riemann_2d_wide(X: int = 2048, Y: int = 2048, seed: int = 0, kind: str = "D2Q49",
                    steps: int = 5000) -> Workload:
    """The four-quadrant problem on WIDE_BAND (see riemann_2d)."""
    wl = riemann_2d(X, Y, seed=seed, kind=kind, steps=steps, band=WIDE_BAND)
    wl.name = "riemann_2d_wide"
    return wl


def blast_3d(L: int = 384, radius: float = 32.0, n: int = 0, steps: int = 2000,
             p_in: float = 1.0, p_out: float = 0.1) -> Workload:
    """3-D blast: uniform rho=1, p=0.1 background, central sphere of the given
    radius (in nodes) at p=1; periodic; D3Q343."""
    c = (np.arange(L) + 0.5) - L / 2.0
    r2 = c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2
    rho = np.ones((L, L, L))
    T = np.where(r2 <= radius * radius, p_in, p_out)
    u = np.zeros((3, L, L, L))
    return Workload("blast_3d", "D3Q343", n, 2.0 / 3.0, (L, L, L), ("periodic",) * 3,
                    rho, u, T, steps)


def smooth_random(shape, seed: int = 0, kind: str = None, n: int = 3, tau: float = 2.0 / 3.0,
                  bc=None, amp_rho=0.2, amp_u=0.1, amp_T=0.1, steps: int = 100, u_mean=None) -> Workload:
    """Smooth seeded random fields: a few low Fourier modes per field around
    rho=1, u=0, T=1 (periodic-compatible).  Used for parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    D = len(shape)
    kind = kind or {1: "D1Q7", 2: "D2Q49", 3: "D3Q343"}[D]
    bc = bc or ("periodic",) * D
    grids = np.meshgrid(*[np.arange(s) / s for s in shape[::-1]], indexing="ij")[::-1]

    def field(amp):
        f = np.zeros(shape[::-1])
        for _ in range(3):
            k = rng.integers(1, 3, D)
            ph = rng.uniform(0, 2 * np.pi)
            a = rng.uniform(-1, 1)
            arg = sum(2 * np.pi * k[d] * grids[d] for d in range(D)) + ph
            f += a * np.sin(arg)
        return amp * f / 3.0

    rho = 1.0 + field(amp_rho)
    T = 1.0 + field(amp_T)
    u = np.stack([field(amp_u) for _ in range(D)])
    if u_mean is not None:
        u += np.asarray(u_mean, dtype=np.float64).reshape((D,) + (1,) * D)
    return Workload("smooth_random", kind, n, tau, tuple(shape), tuple(bc), rho, u, T,
                    steps)


def batched_tubes(count: int = 4096, seed: int = 0, lmin: int = 256, lmax: int = 8192,
                  steps: int = 4000):
    """Ensemble of 1-D shock tubes of uneven length: lengths ~ U{lmin..lmax},
    gamma from {5/3, 1.4, 9/7, 1.25} (n = 2, 4, 6, 7 at D=1), left/right
    pressure ratio log-uniform in [2, 100], density ratio ~ U[1, 10],
    tau ~ U[0.55, 1.0]; left rho=1, p=1; copy ends.  Returns a list of
    Workload (one per tube)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lengths = rng.integers(lmin, lmax + 1, count)
    ns = rng.choice(np.array([2, 4, 6, 7]), count)
    pr = np.exp(rng.uniform(np.log(2.0), np.log(100.0), count))
    dr = rng.uniform(1.0, 10.0, count)
    taus = rng.uniform(0.55, 1.0, count)
    out = []
    for k in range(count):
        X = int(lengths[k])
        rho, u, T = _two_state_1d(X, (1.0, 0.0, 1.0), (1.0 / dr[k], 0.0, 1.0 / pr[k]))
        out.append(Workload(f"tube{k}", "D1Q7", int(ns[k]), float(taus[k]), (X,),
                            ("copy",), rho, u[None], T, steps))
    return out


def surrogate_tubes(count: int = 1024, L: int = 4096, seed: int = 0, tau: float = 0.8,
                    steps: int = 4000):
    """Tubes for the learned surrogate, drawn like ``batched_tubes`` but all of
    length L and with one relaxation time (the network's inputs are rho, u,
    T and gamma only, so tau is a property of the operator it learns):
    gamma from {5/3, 1.4, 9/7, 1.25}, left rho=1, p=1; right density
    1/U[1, 10], pressure 1/logU[2, 100]; diaphragm at mid-tube; copy ends."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.choice(np.array([2, 4, 6, 7]), count)
    pr = np.exp(rng.uniform(np.log(2.0), np.log(100.0), count))
    dr = rng.uniform(1.0, 10.0, count)
    out = []
    for k in range(count):
        rho, u, T = _two_state_1d(L, (1.0, 0.0, 1.0), (1.0 / dr[k], 0.0, 1.0 / pr[k]))
        out.append(Workload(f"stube{k}", "D1Q7", int(ns[k]), float(tau), (L,), ("copy",), rho,
                            u[None], T, steps))
    return out
