"""Learned surrogate of the 1-D method: a convolutional operator that advances
the macroscopic state (rho, u, T) of shock tubes by K lattice steps per call,
trained on the GPU on trajectories the lattice Boltzmann solver generates,
with that solver as its fallback and the reference it is measured against.

Argument marshalling only: the network, its training and every check run in
the CUDA kernels behind the ``lbm_nn_*`` entry points of ``liblbm.so``;
PyTorch provides device memory and the stream.  The network is defined in
include/lbm.h (features, lift, residual dilated conv layers with GELU, linear
head); this module sequences its layers.

What the surrogate learns.  For a state s of a tube, the target is the
method restarted from local equilibrium: L_K(s) = the macroscopic moments
after ``set_macro(s)`` and K steps of the plain solver (FD transport).
A rollout of the surrogate is compared with the rollout of L_K, and the
fallback replaces a prediction by L_K(s) itself.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from .lbm import LbmBatch, LbmError, load_library

DEFAULT_DILATIONS = (1, 1, 2, 2, 4, 4, 1, 1, 2, 2, 4, 4)
# gamma = (D + n + 2) / (D + n) at D = 1
GAMMA_OF_N = {n: (n + 3.0) / (n + 1.0) for n in range(16)}


def _fp(x):
    return ctypes.c_void_p(0 if x is None else x.data_ptr())


def _f32(vals):
    return (ctypes.c_float * len(vals))(*[float(v) for v in vals])


class ConvOperator:
    """The network: parameters (float32 masters, bfloat16 copies for the
    tensor cores), Adam state and activation buffers on one device.

    ``patch`` consecutive nodes form one position of the network (4 patch
    features in, 3 patch outputs), so the body runs on L / patch positions.
    ``impl`` 3 runs the convolutions on the tensor cores (tcgen05, persistent,
    128 channels x 256 positions per tile; layers whose halo (k - 1) d
    exceeds 64 positions take impl 0), 0 on the persistent tensor-core form
    with 128 x 128 tiles, 2 on the tensor cores one output tile per block, 1
    on the CUDA cores.
    """

    def __init__(self, C=128, k=5, dilations=DEFAULT_DILATIONS, patch=1, seed=0, device=None,
                 impl=3, in_scale=(1.0, 1.0, 1.0, 0.25), out_scale=(1.0, 1.0, 1.0)):
        import torch

        self.torch = torch
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise LbmError(-3, "no CUDA device")
        if C % 128 or k % 2 == 0:
            raise LbmError(-1, "C must be a multiple of 128 and k odd")
        self.device = torch.device(device if device is not None else "cuda")
        self.C, self.k, self.dil, self.patch, self.impl = C, k, tuple(dilations), patch, impl
        self.N = len(self.dil)
        self.F, self.Fo = 4 * patch, 3 * patch
        self.in_scale = tuple(float(v) for v in in_scale)
        self.out_scale = tuple(float(v) for v in out_scale)
        shapes = [("Wl", (C, self.F)), ("bl", (C,)), ("W", (self.N, k, C, C)),
                  ("b", (self.N, C)), ("Wp", (self.Fo, C)), ("bp", (self.Fo,))]
        self.offsets, off = {}, 0
        for name, shp in shapes:
            self.offsets[name] = (off, shp)
            off += -(-int(np.prod(shp)) // 4) * 4        # 16-byte aligned segments
        self.size = off
        self.n_params = sum(int(np.prod(s)) for _, s in shapes)
        with torch.cuda.device(self.device):
            z = lambda: torch.zeros(self.size, dtype=torch.float32, device=self.device)
            self.params, self.grads, self.m, self.v = z(), z(), z(), z()
            nw = self.N * k * C * C
            self.wb = torch.empty(nw, dtype=torch.bfloat16, device=self.device)
            self.wt = torch.empty(nw, dtype=torch.bfloat16, device=self.device)
            self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
            self.loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.step_count = 0
        self._bufs = {}
        self.set_params(self.initial_params(seed))

    # ------------------------------------------------------------ parameters
    def initial_params(self, seed):
        """Seeded initialisation: unit-variance lift, conv weights scaled by
        1/sqrt(k C N) so that the residual stream starts close to the lift,
        small head, zero biases."""
        rng = np.random.default_rng(seed)
        C, k, N = self.C, self.k, self.N
        return ([rng.normal(0, 1 / math.sqrt(self.F), (C, self.F)), np.zeros(C)]
                + [rng.normal(0, 0.5 / math.sqrt(k * C * N), (k, C, C)) for _ in range(N)]
                + [np.zeros(C) for _ in range(N)]
                + [rng.normal(0, 0.1 / math.sqrt(C), (self.Fo, C)), np.zeros(self.Fo)])

    def _view(self, buf, name, i=None):
        off, shp = self.offsets[name]
        n = int(np.prod(shp))
        v = buf[off:off + n].view(*shp)
        return v if i is None else v[i]

    def _ptr(self, buf, name, i=None):
        off, shp = self.offsets[name]
        per = int(np.prod(shp[1:])) if i is not None else 0
        return ctypes.c_void_p(buf.data_ptr() + 4 * (off + (i or 0) * per))

    def set_params(self, arrays):
        """Arrays in the order Wl, bl, W_0..W_{N-1}, b_0..b_{N-1}, Wp, bp."""
        t = self.torch
        N = self.N
        Wl, bl, Ws, bs, Wp, bp = arrays[0], arrays[1], arrays[2:2 + N], arrays[2 + N:2 + 2 * N], \
            arrays[2 + 2 * N], arrays[3 + 2 * N]
        for name, val in [("Wl", Wl), ("bl", bl), ("W", np.stack(Ws)), ("b", np.stack(bs)),
                          ("Wp", Wp), ("bp", bp)]:
            self._view(self.params, name).copy_(t.as_tensor(np.asarray(val, np.float32)))
        self.m.zero_(), self.v.zero_()
        self.step_count = 0
        self._cast()

    def _arrays(self, buf):
        g = lambda name: self._view(buf, name).detach().cpu().numpy().astype(np.float64)
        W, b = g("W"), g("b")
        return [g("Wl"), g("bl"), *list(W), *list(b), g("Wp"), g("bp")]

    def get_params(self):
        return self._arrays(self.params)

    def get_grads(self):
        return self._arrays(self.grads)

    def _cast(self):
        s = self.torch.cuda.current_stream(self.device).cuda_stream
        self._check(self.lib.lbm_nn_cast_weights(self._ptr(self.params, "W"), _fp(self.wb),
                                                 _fp(self.wt), self.N, self.C, self.k, s))

    def _check(self, rc, what="lbm_nn"):
        if rc != 0:
            raise LbmError(rc, what)

    # --------------------------------------------------------------- buffers
    def _buffers(self, B, Lp, train):
        key = (B, Lp, train)
        if key in self._bufs:
            return self._bufs[key]
        t = self.torch
        P = B * Lp
        bf = lambda: t.empty(P * self.C, dtype=t.bfloat16, device=self.device)
        nx = self.N + 1 if train else 2
        bufs = {"x": [bf() for _ in range(nx)],
                "z": [bf() for _ in range(self.N)] if train else [],
                "out": t.empty(P * self.Fo, dtype=t.float32, device=self.device)}
        if train:
            bufs["gx"] = t.empty(P * self.C, dtype=t.float32, device=self.device)
            bufs["gz"] = [bf(), bf()]
            bufs["gout"] = t.empty(P * self.Fo, dtype=t.float32, device=self.device)
        self._bufs = {key: bufs}          # keep one shape at a time
        return bufs

    def _wb(self, i):
        return ctypes.c_void_p(self.wb.data_ptr() + 2 * i * self.k * self.C * self.C)

    def _wt(self, i):
        return ctypes.c_void_p(self.wt.data_ptr() + 2 * i * self.k * self.C * self.C)

    # -------------------------------------------------------------- forward
    def forward(self, feat, B, L, train=False):
        """feat: float32 [B*L*4] node features (lbm_nn_features).  Returns the
        float32 head output [B*L*3] (a view into an internal buffer)."""
        lib, s = self.lib, self.torch.cuda.current_stream(self.device).cuda_stream
        if L % self.patch:
            raise LbmError(-1, "tube length must be a multiple of the patch")
        Lp = L // self.patch
        P = B * Lp
        bufs = self._buffers(B, Lp, train)
        x = bufs["x"]
        self._check(lib.lbm_nn_lift(_fp(feat), self._ptr(self.params, "Wl"),
                                    self._ptr(self.params, "bl"), _fp(x[0]), P, self.F, self.C, s),
                    "lbm_nn_lift")
        for i, d in enumerate(self.dil):
            src, dst = (x[i], x[i + 1]) if train else (x[i % 2], x[(i + 1) % 2])
            z = bufs["z"][i] if train else None
            self._check(lib.lbm_nn_conv_forward(_fp(src), self._wb(i), self._ptr(self.params, "b", i),
                                                _fp(dst), _fp(z), B, Lp, self.C, self.k, d,
                                                self.conv_impl(d), _fp(self.status), s),
                        "lbm_nn_conv_forward")
        last = x[self.N] if train else x[self.N % 2]
        self._check(lib.lbm_nn_head(_fp(last), self._ptr(self.params, "Wp"),
                                    self._ptr(self.params, "bp"), _fp(bufs["out"]), P, self.C,
                                    self.Fo, s), "lbm_nn_head")
        return bufs["out"]

    def conv_impl(self, d):
        """Kernel code for a layer of dilation d (impl 3 holds a halo of
        (k - 1) d <= 64 positions per window)."""
        if self.impl == 3 and (self.k - 1) * d > 64:
            return 0
        return self.impl

    def backward(self, feat, gout, B, L):
        """Gradients of the loss with d loss / d out = gout into self.grads
        (zeroed first), after ``forward(feat, B, L, train=True)``."""
        lib, s = self.lib, self.torch.cuda.current_stream(self.device).cuda_stream
        Lp = L // self.patch
        P = B * Lp
        bufs = self._buffers(B, Lp, True)
        x, z, gx, gz = bufs["x"], bufs["z"], bufs["gx"], bufs["gz"]
        g = self.grads
        g.zero_()
        self._check(lib.lbm_nn_head_backward(_fp(gout), _fp(x[self.N]),
                                             self._ptr(self.params, "Wp"), _fp(z[self.N - 1]),
                                             _fp(gx), _fp(gz[0]), self._ptr(g, "Wp"),
                                             self._ptr(g, "bp"), P, self.C, self.Fo, s),
                    "lbm_nn_head_backward")
        cur = 0
        for i in reversed(range(self.N)):
            d = self.dil[i]
            self._check(lib.lbm_nn_bias_grad(_fp(gz[cur]), self._ptr(g, "b", i), P, self.C, s),
                        "lbm_nn_bias_grad")
            self._check(lib.lbm_nn_conv_backward_weight(_fp(gz[cur]), _fp(x[i]), self._ptr(g, "W", i),
                                                        B, Lp, self.C, self.k, d,
                                                        self.conv_impl(d), _fp(self.status), s),
                        "lbm_nn_conv_backward_weight")
            zp, gzp = (z[i - 1], gz[1 - cur]) if i > 0 else (None, None)
            self._check(lib.lbm_nn_conv_backward_data(_fp(gz[cur]), self._wt(i), _fp(gx), _fp(zp),
                                                      _fp(gzp), B, Lp, self.C, self.k, d,
                                                      self.conv_impl(d), _fp(self.status), s),
                        "lbm_nn_conv_backward_data")
            cur = 1 - cur
        self._check(lib.lbm_nn_lift_backward(_fp(gx), _fp(feat), self._ptr(g, "Wl"),
                                             self._ptr(g, "bl"), P, self.F, self.C, s),
                    "lbm_nn_lift_backward")

    def loss_and_grad(self, feat, target, B, L):
        """Forward, mean squared error against target [B*L*3] and backward.
        Returns the loss as a device tensor (float64, one element)."""
        s = self.torch.cuda.current_stream(self.device).cuda_stream
        out = self.forward(feat, B, L, train=True)
        gout = self._buffers(B, L // self.patch, True)["gout"]
        self.loss.zero_()
        self._check(self.lib.lbm_nn_mse(_fp(out), _fp(target), _fp(gout), _fp(self.loss),
                                        out.numel(), s), "lbm_nn_mse")
        self.backward(feat, gout, B, L)
        return self.loss

    def adam(self, lr, b1=0.9, b2=0.999, eps=1e-8, weight_decay=0.0):
        s = self.torch.cuda.current_stream(self.device).cuda_stream
        self.step_count += 1
        self._check(self.lib.lbm_nn_adam(_fp(self.params), _fp(self.grads), _fp(self.m),
                                         _fp(self.v), self.size, lr, b1, b2, eps, self.step_count,
                                         weight_decay, s), "lbm_nn_adam")
        self._cast()

    def check_status(self):
        st = int(self.status.item())
        if st:
            raise LbmError(-5, f"tensor-core kernel timed out (status {st})")

    # -------------------------------------------------------------- helpers
    def features(self, rho, u, T, gamma, B, L, out=None):
        t = self.torch
        s = t.cuda.current_stream(self.device).cuda_stream
        feat = out if out is not None else t.empty(B * L * 4, dtype=t.float32, device=self.device)
        self._check(self.lib.lbm_nn_features(_fp(rho), _fp(u), _fp(T), _fp(gamma), _fp(feat), B, L,
                                             _f32(self.in_scale), s), "lbm_nn_features")
        return feat

    def targets(self, rho, u, T, rho2, u2, T2, out=None):
        t = self.torch
        s = t.cuda.current_stream(self.device).cuda_stream
        n = rho.numel()
        tgt = out if out is not None else t.empty(n * 3, dtype=t.float32, device=self.device)
        self._check(self.lib.lbm_nn_targets(_fp(rho), _fp(u), _fp(T), _fp(rho2), _fp(u2), _fp(T2),
                                            _fp(tgt), n, _f32(self.out_scale), s), "lbm_nn_targets")
        return tgt

    def predict(self, rho, u, T, gamma, B, L):
        """One call: (rho, u, T) after K steps as predicted by the network."""
        t = self.torch
        s = t.cuda.current_stream(self.device).cuda_stream
        feat = self.features(rho, u, T, gamma, B, L)
        out = self.forward(feat, B, L, train=False)
        r2, u2, T2 = (t.empty_like(rho) for _ in range(3))
        self._check(self.lib.lbm_nn_apply(_fp(rho), _fp(u), _fp(T), _fp(out), _fp(r2), _fp(u2),
                                          _fp(T2), rho.numel(), _f32(self.out_scale), s),
                    "lbm_nn_apply")
        return r2, u2, T2


# --------------------------------------------------------------------- data
def _rows(lib, torch, device, fields, rows, offsets, W, row_len, out=None):
    """Gather rows (or windows) of three float fields with lbm_nn_gather."""
    count = int(rows.numel())
    s = torch.cuda.current_stream(device).cuda_stream
    if out is None:
        out = [torch.empty(count * W, dtype=torch.float32, device=device) for _ in range(3)]
    rc = lib.lbm_nn_gather(_fp(fields[0]), _fp(fields[1]), _fp(fields[2]), _fp(rows),
                           _fp(offsets), count, row_len, W, _fp(out[0]), _fp(out[1]), _fp(out[2]),
                           s)
    if rc != 0:
        raise LbmError(rc, "lbm_nn_gather")
    return out


def _scatter(lib, torch, device, packed, rows, offsets, W, row_len, fields):
    s = torch.cuda.current_stream(device).cuda_stream
    rc = lib.lbm_nn_scatter(_fp(packed[0]), _fp(packed[1]), _fp(packed[2]), _fp(rows),
                            _fp(offsets), int(rows.numel()), row_len, W, _fp(fields[0]),
                            _fp(fields[1]), _fp(fields[2]), s)
    if rc != 0:
        raise LbmError(rc, "lbm_nn_scatter")


@dataclass
class Trajectories:
    """Restarted-method trajectories of B tubes of L nodes: rho[j], u[j],
    T[j] are [B*L] device tensors for windows j = 0..J (state after j*K
    steps), ``ok`` marks the tubes the solver kept finite."""
    rho: object
    u: object
    T: object
    n: np.ndarray
    gamma: np.ndarray
    tau: float
    K: int
    L: int
    ok: np.ndarray

    @property
    def B(self):
        return len(self.n)

    @property
    def J(self):
        return self.rho.shape[0] - 1


def restarted_trajectories(rho0, u0, T0, n, tau, L, K, windows, m_fd=10, device=None):
    """state_{j+1} = moments after set_macro(state_j) and K FD steps, for B
    tubes of L nodes given as [B*L] arrays.  All on the device."""
    import torch
    dev = torch.device(device if device is not None else "cuda")
    B = len(n)
    lb = LbmBatch([L] * B, n, [tau] * B, mode="fd", m_fd=m_fd, device=dev)
    rho = torch.empty(windows + 1, B * L, dtype=torch.float32, device=dev)
    u, T = torch.empty_like(rho), torch.empty_like(rho)
    for f, v in ((rho, rho0), (u, u0), (T, T0)):
        f[0].copy_(torch.as_tensor(np.asarray(v, np.float32)))
    bad = np.zeros(B, dtype=bool)
    for j in range(windows):
        lb.set_macro(rho[j], u[j], T[j])
        lb.run(K)
        r, uu, tt = lb.moments()
        rho[j + 1].copy_(r), u[j + 1].copy_(uu), T[j + 1].copy_(tt)
        st, nbad = lb.status()
        bad |= st != 0
    lb.close()
    gam = np.array([GAMMA_OF_N[int(v)] for v in n])
    return Trajectories(rho, u, T, np.asarray(n), gam, tau, K, L, ~bad)


def output_scales(tr: Trajectories, sample=64):
    """Per-channel standard deviation of the K-step change over a sample of
    windows (host side, from a few rows copied back)."""
    idx = np.linspace(0, tr.J - 1, min(sample, tr.J)).astype(int)
    keep = np.repeat(tr.ok, tr.L)
    out = []
    for f in (tr.rho, tr.u, tr.T):
        d = (f[idx + 1] - f[idx]).cpu().numpy()[:, keep]
        out.append(float(np.sqrt(np.mean(d * d))) or 1.0)
    return tuple(out)


class Trainer:
    """Minibatch training of a ConvOperator on restarted-method pairs
    (state_j -> state_{j+1}) of the tubes the solver kept finite.

    ``step(lr)`` runs one step from the host (minibatch drawn by NumPy).
    ``run(lrs)`` runs ``len(lrs)`` steps with the learning-rate schedule
    ``lrs`` as replays of one CUDA graph: the minibatch is drawn on the
    device (lbm_nn_sample_pairs), the learning rate and Adam's bias
    corrections come from a device step counter (lbm_nn_adam_scheduled), so
    a step costs one graph launch."""

    def __init__(self, net: ConvOperator, tr: Trajectories, batch=32, seed=0, max_steps=1 << 20):
        import torch
        self.net, self.tr, self.batch, self.torch = net, tr, batch, torch
        self.seed = seed
        self.rng = np.random.default_rng(seed)
        self.good = np.flatnonzero(tr.ok)
        if self.good.size == 0:
            raise LbmError(-1, "no finite trajectories to train on")
        dev = net.device
        self.gamma = torch.as_tensor(tr.gamma.astype(np.float32), device=dev)
        self.good_dev = torch.as_tensor(self.good.astype(np.int32), device=dev)
        self.rows_src = torch.empty(batch, dtype=torch.int64, device=dev)
        self.rows_dst = torch.empty(batch, dtype=torch.int64, device=dev)
        self.gam_b = torch.empty(batch, dtype=torch.float32, device=dev)
        L = tr.L
        self.a = [torch.empty(batch * L, dtype=torch.float32, device=dev) for _ in range(3)]
        self.b = [torch.empty(batch * L, dtype=torch.float32, device=dev) for _ in range(3)]
        self.feat = torch.empty(batch * L * 4, dtype=torch.float32, device=dev)
        self.target = torch.empty(batch * L * 3, dtype=torch.float32, device=dev)
        self.max_steps = max_steps
        self.lr_table = torch.zeros(max_steps, dtype=torch.float32, device=dev)
        self.step_dev = torch.zeros(1, dtype=torch.int64, device=dev)
        self.hyper = torch.zeros(3, dtype=torch.float32, device=dev)
        self.graph = None

    def sample(self):
        tr, B = self.tr, self.batch
        tubes = self.rng.choice(self.good, B)
        js = self.rng.integers(0, tr.J, B)
        t = self.torch
        self.rows_src.copy_(t.as_tensor(js * tr.B + tubes))
        self.rows_dst.copy_(t.as_tensor((js + 1) * tr.B + tubes))
        self.gam_b.copy_(t.as_tensor(tr.gamma[tubes].astype(np.float32)))
        return self.rows_src, self.rows_dst

    def load(self, rows_src, rows_dst):
        net, tr = self.net, self.tr
        t = self.torch
        fields = (tr.rho.view(-1), tr.u.view(-1), tr.T.view(-1))
        _rows(net.lib, t, net.device, fields, rows_src, None, tr.L, tr.L, self.a)
        _rows(net.lib, t, net.device, fields, rows_dst, None, tr.L, tr.L, self.b)
        net.features(*self.a, self.gam_b, self.batch, tr.L, out=self.feat)
        net.targets(*self.a, *self.b, out=self.target)

    def step(self, lr):
        self.load(*self.sample())
        loss = self.net.loss_and_grad(self.feat, self.target, self.batch, self.tr.L)
        self.net.adam(lr)
        return loss

    # ------------------------------------------------------- graph replays
    def _device_step(self):
        net, tr, lib = self.net, self.tr, self.net.lib
        s = self.torch.cuda.current_stream(net.device).cuda_stream
        rc = lib.lbm_nn_sample_pairs(_fp(self.good_dev), int(self.good.size), tr.J, tr.B,
                                     _fp(self.gamma), self.seed, _fp(self.step_dev), self.batch,
                                     _fp(self.rows_src), _fp(self.rows_dst), _fp(self.gam_b), s)
        if rc != 0:
            raise LbmError(rc, "lbm_nn_sample_pairs")
        self.load(self.rows_src, self.rows_dst)
        net.loss_and_grad(self.feat, self.target, self.batch, tr.L)
        rc = lib.lbm_nn_adam_scheduled(_fp(net.params), _fp(net.grads), _fp(net.m), _fp(net.v),
                                       net.size, _fp(self.lr_table), self.max_steps,
                                       _fp(self.step_dev), _fp(self.hyper), 0.9, 0.999, 1e-8,
                                       0.0, s)
        if rc != 0:
            raise LbmError(rc, "lbm_nn_adam_scheduled")
        net._cast()

    def _capture(self):
        t = self.torch
        side = t.cuda.Stream(device=self.net.device)
        side.wait_stream(t.cuda.current_stream(self.net.device))
        saved = [x.clone() for x in (self.net.params, self.net.m, self.net.v, self.step_dev)]
        with t.cuda.stream(side):       # one eager step: buffers, kernel attributes
            self._device_step()
        t.cuda.current_stream(self.net.device).wait_stream(side)
        g = t.cuda.CUDAGraph()
        with t.cuda.graph(g):
            self._device_step()
        for dst, src in zip((self.net.params, self.net.m, self.net.v, self.step_dev), saved):
            dst.copy_(src)
        self.net._cast()
        self.graph = g

    def reset(self):
        """Adam moments and the device step counter back to zero."""
        self.net.m.zero_(), self.net.v.zero_(), self.step_dev.zero_()
        self.net.step_count = 0

    def run(self, lrs):
        """len(lrs) steps, step i with learning rate lrs[i], continuing the
        device step counter; returns the last step's loss (device tensor)."""
        n = len(lrs)
        done = int(self.step_dev.item())
        if done + n > self.max_steps:
            raise LbmError(-1, "schedule longer than max_steps")
        table = np.full(self.max_steps, float(lrs[-1]), np.float32)
        table[done:done + n] = np.asarray(lrs, np.float32)
        self.lr_table.copy_(self.torch.as_tensor(table))
        if self.graph is None:
            self._capture()
        for _ in range(n):
            self.graph.replay()
        return self.net.loss


def cosine_lr(step, total, peak=1e-3, warmup=100, floor=0.02):
    if step < warmup:
        return peak * (step + 1) / warmup
    f = (step - warmup) / max(1, total - warmup)
    return peak * (floor + (1 - floor) * 0.5 * (1 + math.cos(math.pi * min(1.0, f))))


# ------------------------------------------------------------------ runtime
def fallback_windows(L: int, width: int, margin: int):
    """Windows that recompute a tube of L nodes exactly: interiors of `width`
    nodes tile [0, L) (the last one moved back to end at L, overlapping its
    neighbour), each inside a window of S = width + 2 margin nodes placed so
    that every interior node is at least `margin` nodes from a window edge
    that is not a tube end.  Returns (S, interior starts, window starts);
    one window, the whole tube, when L <= S."""
    width = max(1, min(int(width), L))
    S = min(L, width + 2 * margin)
    if S == L:
        return L, np.zeros(1, np.int64), np.zeros(1, np.int64)
    nw = -(-L // width)
    istart = np.minimum(np.arange(nw, dtype=np.int64) * width, L - width)
    wstart = np.clip(istart - margin, 0, L - S)
    return S, istart, wstart


def _latency_block(length: int) -> int:
    """Block size of an ensemble run whose time is one problem's latency (a
    few problems, or one wave of short ones): one node per thread, up to
    1024.  The ensemble kernel steps a problem with one block, so a 4096-node
    tube at 256 threads makes each thread update 16 nodes in turn per step
    (32 steps: 1.02 ms, against 0.45 ms at 1024 threads; 1024 windows of 384
    nodes: 0.368 ms at 256 threads, 0.355 ms at 384)."""
    return int(min(1024, max(32, -(-length // 32) * 32)))


class SurrogateRunner:
    """Advance B tubes of L nodes by K steps per call with the network, check
    every prediction and fall back to the method where a check fails.

    Checks per tube: the conservation residual of the prediction (totals of
    mass, momentum and energy against the input state) and the L1 error on a
    spot-check window of ``window`` nodes centred on the node where the
    prediction changes rho most, against the method run on that window with a
    margin of 2K nodes on each side (the FD stencil reaches two nodes per
    step, so the window interior is exactly what the full-tube run gives).  A
    tube whose residual or L1 exceeds ``tol``, or whose prediction is not
    finite, is recomputed by the method from the same input state; a tube on
    which the method itself fails (non-finite or non-positive rho, T) keeps
    the prediction and is not sent to the method again (``quarantined``).  With
    ``timing`` the wall time of each phase is accumulated in ``self.times``
    (CUDA events, milliseconds).
    """

    def __init__(self, net: ConvOperator, n, tau, L, K, tol=5e-3, window=256, m_fd=10,
                 timing=False, fallback_window=512):
        import torch
        self.net, self.torch = net, torch
        self.n = np.asarray(n)
        self.B, self.L, self.K, self.tau, self.tol, self.m_fd = len(n), L, K, tau, tol, m_fd
        # fallback tubes are recomputed as windows of fallback_window nodes
        # (plus the 2K-node margins), each an exact piece of the full run
        self.fb_window = max(1, min(int(fallback_window), L))
        self.gamma_np = np.array([GAMMA_OF_N[int(v)] for v in self.n])
        dev = net.device
        self.gamma = torch.as_tensor(self.gamma_np.astype(np.float32), device=dev)
        self.half_dof = torch.as_tensor(((1 + self.n) / 2.0).astype(np.float32), device=dev)
        self.margin = 2 * K
        self.window = min(window, L - 2 * self.margin)
        if self.window < 1:
            raise LbmError(-1, "tube too short for a spot-check window")
        self.span = self.window + 2 * self.margin
        B = self.B
        self.spot = LbmBatch([self.span] * B, self.n, [tau] * B, mode="fd", m_fd=m_fd, device=dev)
        self.spot.set_block(_latency_block(self.span))
        self.rows = torch.arange(B, dtype=torch.int64, device=dev)
        self.starts = torch.zeros(2 * B, dtype=torch.int32, device=dev)
        self.inner = torch.full((B,), self.margin, dtype=torch.int32, device=dev)
        self.residual = torch.empty(B, dtype=torch.float32, device=dev)
        self.l1 = torch.empty(B, dtype=torch.float32, device=dev)
        self._checks_h = torch.empty((2, B), dtype=torch.float32).pin_memory()
        self.stats = {"calls": 0, "fallback_tubes": 0, "max_residual": 0.0, "max_l1": 0.0,
                      "max_l1_accepted": 0.0,
                      "method_failed": 0}
        self.quarantined = np.zeros(self.B, dtype=bool)
        self._solvers = {}
        self.timing = timing
        self.times = {}

    def _mark(self, name, ev):
        if self.timing:
            e = self.torch.cuda.Event(enable_timing=True)
            e.record()
            if ev is not None:
                prev_name, prev = ev
                e.synchronize()
                self.times[prev_name] = self.times.get(prev_name, 0.0) + prev.elapsed_time(e)
            return (name, e)
        return None

    def advance(self, rho, u, T):
        """One call on [B*L] device fields; returns the new fields and the
        indices of the tubes that fell back to the method."""
        t, net, lib = self.torch, self.net, self.net.lib
        s = t.cuda.current_stream(net.device).cuda_stream
        B, L = self.B, self.L
        ev = self._mark("predict", None)
        r2, u2, T2 = net.predict(rho, u, T, self.gamma, B, L)
        ev = self._mark("residual", ev)
        rc = lib.lbm_nn_tube_checks(_fp(rho), _fp(u), _fp(T), _fp(r2), _fp(u2), _fp(T2),
                                    _fp(self.half_dof), None, _fp(self.residual), None,
                                    _fp(self.starts), self.span, self.margin, B, L, 0, L, s)
        if rc != 0:
            raise LbmError(rc, "lbm_nn_tube_checks")
        # spot check: the method on [start, start + span), compared on the
        # interior [start + margin, start + margin + window)
        ev = self._mark("spot_check", ev)
        win_in = _rows(lib, t, net.device, (rho, u, T), self.rows, self.starts, self.span, L)
        self.spot.set_macro(*win_in)
        self.spot.run(self.K)
        ref = self.spot.moments()
        off_in = self.starts[B:]
        pred_w = _rows(lib, t, net.device, (r2, u2, T2), self.rows, off_in, self.window, L)
        ref_w = _rows(lib, t, net.device, ref, self.rows, self.inner, self.window, self.span)
        rc = lib.lbm_nn_tube_checks(_fp(pred_w[0]), _fp(pred_w[1]), _fp(pred_w[2]), _fp(ref_w[0]),
                                    _fp(ref_w[1]), _fp(ref_w[2]), None, _fp(self.gamma), None,
                                    _fp(self.l1), None, 0, 0, B, self.window, 0, self.window, s)
        if rc != 0:
            raise LbmError(rc, "lbm_nn_tube_checks")
        ev = self._mark("decide", ev)
        self._checks_h[0].copy_(self.residual, non_blocking=True)
        self._checks_h[1].copy_(self.l1, non_blocking=True)
        t.cuda.current_stream(net.device).synchronize()
        res = self._checks_h[0].numpy().copy()
        l1 = self._checks_h[1].numpy().copy()
        bad = ~np.isfinite(res) | (res > self.tol) | ~np.isfinite(l1) | (l1 > self.tol)
        # a tube on which the method itself has failed is not sent back to it
        fallback = np.flatnonzero(bad & ~self.quarantined)
        ev = self._mark("fallback", ev)
        if fallback.size:
            self._fallback(rho, u, T, (r2, u2, T2), fallback)
        self._mark("end", ev)
        self.stats["calls"] += 1
        self.stats["fallback_tubes"] += int(fallback.size)
        fin = np.isfinite(res)
        if fin.any():
            self.stats["max_residual"] = max(self.stats["max_residual"], float(res[fin].max()))
        fin = np.isfinite(l1)
        if fin.any():
            self.stats["max_l1"] = max(self.stats["max_l1"], float(l1[fin].max()))
        kept = ~bad & ~self.quarantined  # predictions that passed both checks
        if kept.any():
            self.stats["max_l1_accepted"] = max(self.stats["max_l1_accepted"], float(l1[kept].max()))
        return (r2, u2, T2), fallback

    def _fallback(self, rho, u, T, out, tubes):
        """Recompute `tubes` with the method.  Each tube is cut into windows
        whose interiors (fb_window nodes) tile it, each window carrying the
        2K-node margins on its inner sides: the method on a window gives its
        interior bit for bit as the full-tube run does (the spot check's
        property), and short windows run many to a launch with their state
        in shared memory.  Only a window's interior may set its status word
        (lbm_batch_set_watch), so a window fails exactly where the full-tube
        run fails; a tube on which any window fails keeps its prediction and
        is quarantined."""
        t, net, lib = self.torch, self.net, self.net.lib
        L = self.L
        S, istart, wstart = fallback_windows(L, self.fb_window, self.margin)
        Wi = L if S == L else min(self.fb_window, L)
        nw = istart.size
        f = len(tubes)
        count = f * nw
        # a pool of solvers with room for 1, 2, 4, ... windows of S nodes,
        # retargeted to this call's windows (lbm_batch_set_problems); slot i
        # is always window i % nw, so the window geometry (offsets, watch
        # ranges) is fixed per pool entry; the free slots repeat the last
        # tube and their results are dropped
        cap = 1 << (count - 1).bit_length()
        ent = self._solvers.get(cap)
        if ent is None:
            lb = LbmBatch([S] * cap, [0] * cap, [self.tau] * cap, mode="fd", m_fd=self.m_fd,
                          device=net.device)
            lb.set_block(_latency_block(S))
            slot = np.arange(cap) % nw
            inner = (istart - wstart)[slot]
            # only the exact interiors report failures (the margins carry the
            # windows' artificial ends)
            lb.set_watch(inner, inner + Wi)
            dev = net.device
            ent = {"lb": lb,
                   "woff": t.as_tensor(wstart[slot].astype(np.int32), device=dev),
                   "inner": t.as_tensor(inner.astype(np.int32), device=dev),
                   "ioff": t.as_tensor(istart[slot].astype(np.int32), device=dev),
                   "all": t.arange(cap, dtype=t.int64, device=dev),
                   "rows_h": t.empty(cap, dtype=t.int64).pin_memory(),
                   "rows": t.empty(cap, dtype=t.int64, device=dev)}
            self._solvers[cap] = ent
        lb = ent["lb"]
        win_tube = np.repeat(np.asarray(tubes, np.int64), nw)
        rows_np = np.concatenate([win_tube, np.full(cap - count, win_tube[-1])])
        lb.set_problems(self.n[rows_np], self.tau)
        ent["rows_h"].numpy()[:] = rows_np
        rows = ent["rows"]
        rows.copy_(ent["rows_h"], non_blocking=True)
        packed = _rows(lib, t, net.device, (rho, u, T), rows, ent["woff"], S, L)
        lb.set_macro(*packed)
        lb.run(self.K)
        res = lb.moments()
        # where the method itself fails (non-finite or non-positive rho, T from
        # a state at the edge of its stability), the prediction is kept and the
        # tube is counted; everywhere else the method's result replaces it
        st, _ = lb.status()      # (synchronises: rows_h may be rewritten after it)
        failed = (st[:count] != 0).reshape(f, nw).any(1)
        if not failed.any():
            sel, dst_rows, dst_off, inner = (ent["all"][:count], rows[:count],
                                             ent["ioff"][:count], ent["inner"][:count])
        else:
            self.stats["method_failed"] += int(failed.sum())
            self.quarantined[np.asarray(tubes)[failed]] = True
            keep = np.flatnonzero(np.repeat(~failed, nw))
            if keep.size == 0:
                return
            dev = net.device
            slot = keep % nw
            sel = t.as_tensor(keep, device=dev)
            dst_rows = t.as_tensor(win_tube[keep], device=dev)
            dst_off = t.as_tensor(istart[slot].astype(np.int32), device=dev)
            inner = t.as_tensor((istart - wstart)[slot].astype(np.int32), device=dev)
        interiors = _rows(lib, t, net.device, res, sel, inner, Wi, S)
        _scatter(lib, t, net.device, interiors, dst_rows, dst_off, Wi, L, out)
