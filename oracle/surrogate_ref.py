"""FP64 CPU reference of the learned surrogate (the 1-D convolutional operator
that advances the macroscopic state of a tube by K lattice steps per call).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the library never
does.  The paper has no surrogate: the network is an extension of the method,
and its definition is the contract of the ``lbm_nn_*`` entry points in
``include/lbm.h``, restated here as plain NumPy in double precision:

    features  a[b,l,:] = ((rho-1)/s0, u/s1, (T-1)/s2, (gamma-1.4)/s3)
    lift      x0       = bf16(a Wl^T + bl)                       (C channels)
    layer i   z_i      = conv(x_i; W_i, d_i) + b_i,   W_i[t][co][ci], k taps,
                         tap t reads position l + (t - k//2) d_i, zero outside
                         the tube
              x_{i+1}  = bf16(x_i + gelu(z_i))
    head      out      = x_N Wp^T + bp                            (3 channels)
    update    (rho,u,T)' = (rho,u,T) + out * out_scale

(patches of P consecutive nodes may form one position: 4P features in, 3P
outputs; the functions below take the feature and output counts from the
array shapes) with gelu the tanh form of the Gaussian error linear unit and
bf16() rounding
to bfloat16 (nearest, ties to even) at the points where the GPU path stores a
bfloat16 tensor.  Training minimises the mean squared error between ``out``
and the scaled change of the LBM state over K steps.  The backward pass is
written out by hand (no automatic differentiation): the residual stream and
the input gradients in FP64, the operands the GPU path feeds to its tensor
cores (z for the activation derivative, the pre-activation gradient g_z)
rounded to bfloat16 exactly where the GPU path rounds them.

Parity pins (tests/test_oracle_surrogate.py): the analytic gradient against
central finite differences with the rounding switched off; the convolution
against numpy.correlate channel by channel and a one-hot kernel against a
plain shift; bfloat16 rounding against torch's conversion; gelu against the
erf form within the published error of the tanh approximation; one Adam step
against its closed form.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    The input is first rounded to float32 (the GPU path holds every value it
    rounds to bfloat16 in a float32 register)."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def gelu(x):
    """x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))."""
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + GELU_A * x ** 3)))


def gelu_grad(x):
    """Derivative of ``gelu`` (product and chain rule on the tanh form)."""
    th = np.tanh(GELU_C * (x + GELU_A * x ** 3))
    return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th * th) * GELU_C * (1.0 + 3.0 * GELU_A * x * x)


def shift(x, s):
    """y[:, l, :] = x[:, l + s, :], zero where l + s falls outside [0, L)."""
    B, L, C = x.shape
    y = np.zeros_like(x)
    if s >= 0:
        if s < L:
            y[:, :L - s] = x[:, s:]
    else:
        if -s < L:
            y[:, -s:] = x[:, :L + s]
    return y


def conv1d(x, W, d):
    """z[b,l,co] = sum_t sum_ci x[b, l + (t - k//2) d, ci] W[t,co,ci]."""
    k = W.shape[0]
    z = np.zeros(x.shape[:2] + (W.shape[1],))
    for t in range(k):
        z += shift(x, (t - k // 2) * d) @ W[t].T
    return z


def conv1d_input_grad(g, W, d):
    """Adjoint of conv1d in x: gx[b,l,ci] = sum_t sum_co g[b, l - (t - k//2) d, co] W[t,co,ci]."""
    k = W.shape[0]
    gx = np.zeros(g.shape[:2] + (W.shape[2],))
    for t in range(k):
        gx += shift(g, -(t - k // 2) * d) @ W[t]
    return gx


def conv1d_weight_grad(g, x, k, d):
    """Adjoint of conv1d in W: gW[t,co,ci] = sum_{b,l} g[b,l,co] x[b, l + (t - k//2) d, ci]."""
    gW = np.zeros((k, g.shape[2], x.shape[2]))
    g2 = g.reshape(-1, g.shape[2])
    for t in range(k):
        gW[t] = g2.T @ shift(x, (t - k // 2) * d).reshape(-1, x.shape[2])
    return gW


@dataclass
class Params:
    """Network parameters in FP64 (the float32 masters of the GPU path)."""
    Wl: np.ndarray            # [C, 4]
    bl: np.ndarray            # [C]
    W: list                   # N x [k, C, C]
    b: list                   # N x [C]
    Wp: np.ndarray            # [3, C]
    bp: np.ndarray            # [3]
    dil: list                 # N dilations

    def arrays(self):
        return [self.Wl, self.bl, *self.W, *self.b, self.Wp, self.bp]


def init_params(C=128, k=5, dil=(1, 1, 2, 2, 4, 4, 1, 1, 2, 2, 4, 4), seed=0) -> Params:
    """Seeded He-style initialisation (scaled so the residual stream starts small)."""
    rng = np.random.default_rng(seed)
    N = len(dil)
    Wl = rng.normal(0, 1.0 / math.sqrt(4), (C, 4))
    W = [rng.normal(0, 0.5 / math.sqrt(k * C * N), (k, C, C)) for _ in range(N)]
    Wp = rng.normal(0, 0.1 / math.sqrt(C), (3, C))
    return Params(Wl, np.zeros(C), W, [np.zeros(C) for _ in range(N)], Wp, np.zeros(3),
                  list(dil))


def features(rho, u, T, gamma_per_tube, in_scale):
    """a[b,l,:] = ((rho-1)/s0, u/s1, (T-1)/s2, (gamma-1.4)/s3); rho, u, T are [B, L]."""
    B, L = rho.shape
    g = np.broadcast_to(np.asarray(gamma_per_tube, float)[:, None], (B, L))
    return np.stack([(rho - 1.0) / in_scale[0], u / in_scale[1], (T - 1.0) / in_scale[2],
                     (g - 1.4) / in_scale[3]], axis=-1)


def forward(p: Params, a, emulate_bf16=True):
    """Forward pass; returns (out [B,L,3], cache for ``backward``)."""
    rnd = bf16_round if emulate_bf16 else (lambda v: np.asarray(v, float))
    W = [rnd(w) for w in p.W]
    x = rnd(a @ p.Wl.T + p.bl)
    xs, zs = [x], []
    for i, d in enumerate(p.dil):
        z = conv1d(x, W[i], d) + p.b[i]
        zs.append(rnd(z))
        x = rnd(x + gelu(z))
        xs.append(x)
    out = x @ p.Wp.T + p.bp
    return out, {"a": a, "xs": xs, "zs": zs, "W": W}


def mse(out, target):
    """loss = mean((out - target)^2), gradient 2 (out - target) / count."""
    d = out - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(p: Params, cache, gout, emulate_bf16=True):
    """Gradients of a scalar loss with d loss / d out = gout; same order as Params.arrays()."""
    rnd = bf16_round if emulate_bf16 else (lambda v: np.asarray(v, float))
    xs, zs, W, a = cache["xs"], cache["zs"], cache["W"], cache["a"]
    N = len(p.dil)
    k = p.W[0].shape[0] if N else 1
    g2 = gout.reshape(-1, gout.shape[-1])
    gWp = g2.T @ xs[N].reshape(-1, xs[N].shape[-1])
    gbp = g2.sum(0)
    gx = gout @ p.Wp
    gW, gb = [None] * N, [None] * N
    for i in reversed(range(N)):
        gz = rnd(gx * gelu_grad(zs[i]))
        gW[i] = conv1d_weight_grad(gz, xs[i], k, p.dil[i])
        gb[i] = gz.reshape(-1, gz.shape[-1]).sum(0)
        gx = gx + conv1d_input_grad(gz, W[i], p.dil[i])
    gWl = gx.reshape(-1, gx.shape[-1]).T @ a.reshape(-1, a.shape[-1])
    gbl = gx.reshape(-1, gx.shape[-1]).sum(0)
    return [gWl, gbl, *gW, *gb, gWp, gbp]


def adam_step(param, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """One Adam update (Kingma and Ba, with bias correction); returns (param, m, v)."""
    g = grad + wd * param
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v


def conservation_residual(rho, u, T, rho2, u2, T2, n, D=1):
    """Per tube: max of the relative changes of total mass, momentum (scaled by
    the mass) and total energy sum rho ((D+n)/2 T + u^2/2) between two states.
    rho, u, T are [B, L]; n is the rotational degree count per tube."""
    cv = (D + np.asarray(n, float)) / 2.0
    m1, m2 = rho.sum(1), rho2.sum(1)
    j1, j2 = (rho * u).sum(1), (rho2 * u2).sum(1)
    e1 = (rho * (cv[:, None] * T + 0.5 * u * u)).sum(1)
    e2 = (rho2 * (cv[:, None] * T2 + 0.5 * u2 * u2)).sum(1)
    return np.maximum(np.abs(m2 - m1) / m1, np.maximum(np.abs(j2 - j1) / m1, np.abs(e2 - e1) / e1))


def l1_error(rho, u, T, rho_ref, u_ref, T_ref, gamma):
    """Per tube: max over (rho, u, T) of the relative L1 error, velocity taken
    relative to the local sound speed sqrt(gamma T) (a Mach-number error)."""
    g = np.asarray(gamma, float)[:, None]
    er = np.abs(rho - rho_ref).sum(1) / np.abs(rho_ref).sum(1)
    eu = np.abs(u - u_ref).sum(1) / np.sqrt(g * T_ref).sum(1)
    eT = np.abs(T - T_ref).sum(1) / np.abs(T_ref).sum(1)
    return np.maximum(er, np.maximum(eu, eT))
