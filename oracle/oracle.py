"""FP64 CPU oracle for the decoupled Hermite-expansion LBM (arXiv 1606.06107).

TEST INFRASTRUCTURE.  This module is the independent reference the CUDA
library is checked against.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library in
``paper_1606_06107_gb300`` never does.  The arithmetic lives in plain C
(``lbm_oracle.c``, ``riemann_exact.c``), compiled here with gcc, double
precision, no fused multiply-add contraction, OpenMP over nodes.

Every function below cites the part of the paper it follows; the readings
taken where the paper is garbled or silent are listed in ``lbm_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_SOURCES = ["lbm_oracle.c", "riemann_exact.c"]

D1Q7, D2Q37, D2Q49, D3Q343 = 1, 2, 3, 4
LATTICE_DIM = {D1Q7: 1, D2Q37: 2, D2Q49: 2, D3Q343: 3}
LATTICE_Q = {D1Q7: 7, D2Q37: 37, D2Q49: 49, D3Q343: 343}
STREAM, FD = 0, 1
PERIODIC, COPY = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``_build/liborc.so`` (gcc, -O2, OpenMP)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _P = ctypes.POINTER
        dp = _P(ctypes.c_double)
        ip = _P(ctypes.c_int)
        _lib.orc_lattice_get.argtypes = [ctypes.c_int, dp, ip, dp, dp]
        _lib.orc_geq.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp]
        _lib.orc_heq.argtypes = [ctypes.c_double, dp]
        _lib.orc_node_moments.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        _lib.orc_collide_node.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          dp, dp, dp, dp]
        for name in ("orc_init", "orc_moments"):
            getattr(_lib, name).argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
        _lib.orc_step.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        _lib.orc_run.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, ctypes.c_long]
        _lib.orc_conservation.argtypes = [ctypes.c_void_p, dp, dp, dp]
        _lib.orc_upwind.argtypes = [ctypes.c_double, dp]
        _lib.orc_upwind.restype = ctypes.c_double
        _lib.orc_riemann.argtypes = [ctypes.c_double, dp, dp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, dp, dp, dp, dp, dp]
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class _Cfg(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("tau", ctypes.c_double),
                ("mode", ctypes.c_int), ("m_fd", ctypes.c_int),
                ("shape", ctypes.c_int * 3), ("bc", ctypes.c_int * 3)]


# --------------------------------------------------------------------------
# Lattices and equilibria (Sec. IV, Tables I and II)

def lattice(kind: int):
    """(r, e[Q,3] int, w[Q], moment residual) re-solved in FP64 (Tables I/II).

    Velocities are ordered by (ez, ey, ex) ascending; xi_i = r * e_i.
    """
    r = ctypes.c_double()
    res = ctypes.c_double()
    e = np.zeros((343, 3), dtype=np.int32)
    w = np.zeros(343)
    q = lib().orc_lattice_get(kind, ctypes.byref(r), e.ctypes.data_as(
        ctypes.POINTER(ctypes.c_int)), _dp(w), ctypes.byref(res))
    if q <= 0:
        raise RuntimeError("lattice solve failed")
    return r.value, e[:q].astype(np.int64), w[:q].copy(), res.value


def geq(kind: int, rho: float, u, theta: float) -> np.ndarray:
    """4th-order Hermite translational equilibrium g_i^eq (Sec. IV)."""
    uu = np.zeros(3)
    uu[:len(u)] = u
    out = np.zeros(343)
    q = lib().orc_geq(kind, float(rho), _dp(uu), float(theta), _dp(out))
    return out[:q].copy()


def heq(theta: float) -> np.ndarray:
    """4th-order Hermite rotational equilibrium h_j^eq on D1Q7 (Sec. IV)."""
    out = np.zeros(7)
    lib().orc_heq(float(theta), _dp(out))
    return out


def node_moments(kind: int, n: int, g, h):
    """(rho, u[D], T, K, R) of one node (Sec. V steps 3-4, Eq. T)."""
    D = LATTICE_DIM[kind]
    g = np.ascontiguousarray(g, dtype=np.float64)
    h = np.ascontiguousarray(h if h is not None else np.zeros(7), dtype=np.float64)
    out = np.zeros(4 + D)
    lib().orc_node_moments(kind, n, _dp(g), _dp(h), _dp(out))
    return out[0], out[1:1 + D].copy(), out[1 + D], out[2 + D], out[3 + D]


def collide_node(kind: int, n: int, omega: float, g, h):
    """BGK relaxation of one node toward its own equilibria (Eq. DisEvolI/EvoEtaJ)."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    h = np.ascontiguousarray(h if h is not None else np.zeros(7), dtype=np.float64)
    go = np.zeros_like(g)
    ho = np.zeros(7)
    lib().orc_collide_node(kind, n, float(omega), _dp(g), _dp(h), _dp(go), _dp(ho))
    return go, ho


def upwind(nu: float, f5) -> float:
    """Third-order upwind convection term nu*dF/dx from F at offsets -2..+2 (Sec. V)."""
    f = np.ascontiguousarray(f5, dtype=np.float64)
    return lib().orc_upwind(float(nu), _dp(f))


# --------------------------------------------------------------------------
# Whole-grid simulation

@dataclass
class Sim:
    """An oracle simulation: populations ft[Q, N] and fr[7 or 0, N] in FP64.

    shape is (X,), (X, Y) or (X, Y, Z) with x fastest in memory; bc holds one
    of PERIODIC / COPY per axis.
    """
    kind: int
    n: int
    tau: float
    shape: tuple
    bc: tuple
    mode: int = STREAM
    m_fd: int = 10
    ft: np.ndarray = field(default=None, repr=False)
    fr: np.ndarray = field(default=None, repr=False)

    def __post_init__(self):
        D = LATTICE_DIM[self.kind]
        if len(self.shape) != D or len(self.bc) != D:
            raise ValueError("shape/bc must have one entry per dimension")
        self._cfg = _Cfg()
        self._cfg.kind = self.kind
        self._cfg.n = self.n
        self._cfg.tau = self.tau
        self._cfg.mode = self.mode
        self._cfg.m_fd = self.m_fd
        for a in range(3):
            self._cfg.shape[a] = self.shape[a] if a < D else 1
            self._cfg.bc[a] = self.bc[a] if a < D else PERIODIC
        self.D = D
        self.Q = LATTICE_Q[self.kind]
        self.Qr = 7 if self.n > 0 else 0
        self.N = int(np.prod(self.shape))
        self.ft = np.zeros((self.Q, self.N))
        self.fr = np.zeros((max(self.Qr, 1), self.N))
        self.steps = 0

    @property
    def gamma(self) -> float:
        """gamma = (D+n+2)/(D+n) (Sec. III)."""
        return (self.D + self.n + 2.0) / (self.D + self.n)

    def _flat(self, a, rows=None):
        a = np.asarray(a, dtype=np.float64)
        if rows is None:
            return np.ascontiguousarray(a.reshape(self.N))
        return np.ascontiguousarray(a.reshape(rows, self.N))

    def set_macro(self, rho, u, T):
        """Equilibrium initial state at (rho, u[D], T); arrays are x-fastest.

        rho and T have ``N`` entries (any shape), u has ``D * N`` (SoA).
        """
        r = self._flat(rho)
        uu = self._flat(u, self.D)
        t = self._flat(T)
        rc = lib().orc_init(ctypes.byref(self._cfg), _dp(r), _dp(uu), _dp(t),
                            _dp(self.ft), _dp(self.fr))
        if rc:
            raise ValueError(f"orc_init failed ({rc})")
        self.steps = 0

    def step(self, k: int = 1):
        ft2 = np.empty_like(self.ft)
        fr2 = np.empty_like(self.fr)
        rc = lib().orc_run(ctypes.byref(self._cfg), _dp(self.ft), _dp(self.fr),
                           _dp(ft2), _dp(fr2), int(k))
        if rc:
            raise ValueError(f"orc_run failed ({rc})")
        self.steps += k

    def moments(self):
        """(rho[N], u[D, N], T[N]) at the current time."""
        rho = np.zeros(self.N)
        u = np.zeros((self.D, self.N))
        T = np.zeros(self.N)
        rc = lib().orc_moments(ctypes.byref(self._cfg), _dp(self.ft), _dp(self.fr),
                               _dp(rho), _dp(u), _dp(T))
        if rc:
            raise ValueError(f"orc_moments failed ({rc})")
        return rho, u, T

    def conservation(self) -> np.ndarray:
        """[sum rho, sum rho u (D), sum rho(E + u^2/2), max|sum_j h_j - 1|]."""
        out = np.zeros(3 + self.D)
        rc = lib().orc_conservation(ctypes.byref(self._cfg), _dp(self.ft), _dp(self.fr),
                                    _dp(out))
        if rc:
            raise ValueError(f"orc_conservation failed ({rc})")
        return out

    def state(self):
        """(ft[Q, N], fr[Qr, N]) copies of the stored populations."""
        return self.ft.copy(), self.fr[:self.Qr].copy()

    def set_state(self, ft, fr=None):
        self.ft[...] = np.asarray(ft, dtype=np.float64).reshape(self.Q, self.N)
        if self.Qr:
            self.fr[...] = np.asarray(fr, dtype=np.float64).reshape(7, self.N)


# --------------------------------------------------------------------------
# Exact Riemann solution and the error metric (Sec. VI)

def riemann(gamma: float, left, right, x, x0: float, t: float):
    """Exact Euler Riemann solution sampled at x: (rho, u, p, (p*, u*))."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    L = np.asarray(left, dtype=np.float64)
    R = np.asarray(right, dtype=np.float64)
    rho = np.zeros_like(x)
    u = np.zeros_like(x)
    p = np.zeros_like(x)
    star = np.zeros(2)
    rc = lib().orc_riemann(float(gamma), _dp(L), _dp(R), float(x0), float(t), x.size,
                           _dp(x), _dp(rho), _dp(u), _dp(p), _dp(star))
    if rc:
        raise ValueError("vacuum generated")
    return rho, u, p, (star[0], star[1])


def rel_l1(num, anal) -> float:
    """Relative L1 error sum|x_num - x_anal| / sum|x_anal| (Eq. Error)."""
    num = np.asarray(num, dtype=np.float64)
    anal = np.asarray(anal, dtype=np.float64)
    return float(np.abs(num - anal).sum() / np.abs(anal).sum())
