"""Thin ctypes binding over liblbm.so (the C ABI of include/lbm.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``liblbm.so``.  PyTorch provides the device memory (two state buffers and
a work buffer, owned by the ``Lbm`` object) and the CUDA stream.  There is no
CPU fallback: if the library is missing or a CUDA device is not available the
calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm.so")

LATTICES = {"D1Q7": 1, "D2Q37": 2, "D2Q49": 3, "D3Q343": 4}
LATTICE_DIM = {"D1Q7": 1, "D2Q37": 2, "D2Q49": 2, "D3Q343": 3}
LATTICE_Q = {"D1Q7": 7, "D2Q37": 37, "D2Q49": 49, "D3Q343": 343}
BCS = {"periodic": 0, "copy": 1}
MODES = {"stream": 0, "fd": 1}
STORAGES = {"f32": 0, "f16": 1, "bf16": 2, "f16_node": 3, "bf16_node": 4}
STATUS = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ESIZE", -3: "LBM_ECUDA",
          -4: "LBM_ENONFINITE", -5: "LBM_ETIMEOUT", -6: "LBM_ESTATE"}

# Every symbol include/lbm.h declares, with its ctypes signature.
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
SIGNATURES = {
    "lbm_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.POINTER(_vp)]),
    "lbm_set_mode": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "lbm_set_storage": (ctypes.c_int, [_vp, ctypes.c_int]),
    "lbm_set_grid": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_size_t),
                                    ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_bind": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t, _vp]),
    "lbm_set_macro": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_step": (ctypes.c_int, [_vp, _i64]),
    "lbm_get_moments": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_conservation": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "lbm_conservation_noalloc": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    "lbm_get_state": (ctypes.c_int, [_vp, _vp, _vp]),
    "lbm_set_state": (ctypes.c_int, [_vp, _vp, _vp]),
    "lbm_sample_state": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "lbm_status": (ctypes.c_int, [_vp]),
    "lbm_steps": (_i64, [_vp]),
    "lbm_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_lattice_info": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double)]),
    "lbm_launch_count": (_i64, [_vp]),
    "lbm_destroy": (None, [_vp]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_i64),
                                        ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(_vp)]),
    "lbm_batch_set_problems": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_double)]),
    "lbm_batch_set_watch": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_sizes": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_i64)]),
    "lbm_batch_bind": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t,
                                      _vp]),
    "lbm_batch_set_macro": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_batch_run": (ctypes.c_int, [_vp, _i64]),
    "lbm_batch_get_moments": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_batch_status": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_set_block": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "lbm_batch_autotune": (ctypes.c_int, [_vp, _i64, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_launch_count": (_i64, [_vp]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_batch_destroy": (None, [_vp]),
    # learned surrogate (include/lbm.h, lbm_nn_*)
    "lbm_nn_conv_forward": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp] + [ctypes.c_int] * 6
                            + [_vp, _vp]),
    "lbm_nn_conv_backward_data": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp] + [ctypes.c_int] * 6
                                  + [_vp, _vp]),
    "lbm_nn_conv_backward_weight": (ctypes.c_int, [_vp, _vp, _vp] + [ctypes.c_int] * 6
                                    + [_vp, _vp]),
    "lbm_nn_cast_weights": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, _vp]),
    "lbm_nn_lift": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.c_int, ctypes.c_int, _vp]),
    "lbm_nn_lift_backward": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.c_int,
                                            ctypes.c_int, _vp]),
    "lbm_nn_head": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.c_int, ctypes.c_int, _vp]),
    "lbm_nn_head_backward": (ctypes.c_int, [_vp] * 8 + [_i64, ctypes.c_int, ctypes.c_int,
                                                        _vp]),
    "lbm_nn_bias_grad": (ctypes.c_int, [_vp, _vp, _i64, ctypes.c_int, _vp]),
    "lbm_nn_adam": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_float, ctypes.c_int,
                                   ctypes.c_float, _vp]),
    "lbm_nn_mse": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _vp]),
    "lbm_nn_adam_scheduled": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _vp, _i64, _vp, _vp,
                                             ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                             ctypes.c_float, _vp]),
    "lbm_nn_sample_pairs": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp,
                                           ctypes.c_uint64, _vp, ctypes.c_int, _vp, _vp, _vp,
                                           _vp]),
    "lbm_nn_features": (ctypes.c_int, [_vp] * 5 + [ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_float), _vp]),
    "lbm_nn_targets": (ctypes.c_int, [_vp] * 7 + [_i64, ctypes.POINTER(ctypes.c_float), _vp]),
    "lbm_nn_apply": (ctypes.c_int, [_vp] * 7 + [_i64, ctypes.POINTER(ctypes.c_float), _vp]),
    "lbm_nn_tube_checks": (ctypes.c_int, [_vp] * 11 + [ctypes.c_int] * 6 + [_vp]),
    "lbm_nn_wait_selftest": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_int, _vp, _vp]),
    "lbm_nn_gather": (ctypes.c_int, [_vp] * 5 + [ctypes.c_int, _i64, ctypes.c_int]
                      + [_vp] * 4),
    "lbm_nn_scatter": (ctypes.c_int, [_vp] * 5 + [ctypes.c_int, _i64, ctypes.c_int]
                       + [_vp] * 4),
}


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        self.code = code
        super().__init__(f"{STATUS.get(code, code)}: {msg}")


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblbm.so (built by ``_build.build()``); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise LbmError(-6, f"{path} not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def lattice_info(lattice: str):
    """The library's own (r, e[Q,3], w[Q]) in double precision."""
    lib = load_library()
    r = ctypes.c_double()
    e = (ctypes.c_int * (343 * 3))()
    w = (ctypes.c_double * 343)()
    q = lib.lbm_lattice_info(LATTICES[lattice], ctypes.byref(r), e, w)
    if q < 0:
        raise LbmError(q, f"lattice {lattice}")
    return r.value, np.array(e[:3 * q]).reshape(q, 3), np.array(w[:q])


class Lbm:
    """One solver instance on one CUDA device.

    Parameters follow include/lbm.h: ``lattice`` in LATTICES, ``n`` rotational
    degrees of freedom, ``tau`` relaxation time in lattice steps, ``shape``
    (X,), (X, Y) or (X, Y, Z) with x fastest, ``bc`` per axis in BCS,
    ``mode`` "stream" or "fd" (with ``m_fd`` sub-steps), ``storage`` in
    STORAGES: "f32"; "f16" / "bf16" deviations from the rest equilibrium;
    "f16_node" / "bf16_node" deviations from each node's own reference
    equilibrium (STREAM mode, lattices other than D3Q343).
    """

    def __init__(self, lattice: str, n: int, tau: float, shape, bc, mode: str = "stream",
                 m_fd: int = 10, device=None, stream=None, storage: str = "f32"):
        import torch

        self.torch = torch
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise LbmError(-3, "no CUDA device")
        self.device = torch.device(device if device is not None else "cuda")
        self.lattice = lattice
        self.D = LATTICE_DIM[lattice]
        self.Q = LATTICE_Q[lattice]
        self.Qr = 7 if n > 0 else 0
        self.n = n
        self.tau = tau
        self.shape = tuple(int(s) for s in shape)
        self.N = int(np.prod(self.shape))
        if len(self.shape) != self.D or len(bc) != self.D:
            raise LbmError(-1, "shape and bc need one entry per dimension")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            h = ctypes.c_void_p()
            self._check(self.lib.lbm_create(self.D, LATTICES[lattice], n, float(tau),
                                            ctypes.byref(h)), None)
            self.h = h
            self._check(self.lib.lbm_set_mode(h, MODES[mode], int(m_fd)))
            self._check(self.lib.lbm_set_storage(h, STORAGES[storage]))
            self.storage = storage
            shp = (ctypes.c_int64 * 3)(*self.shape, *([1] * (3 - self.D)))
            bcs = (ctypes.c_int * 3)(*[BCS[b] for b in bc], *([0] * (3 - self.D)))
            sb = ctypes.c_size_t()
            wb = ctypes.c_size_t()
            self._check(self.lib.lbm_set_grid(h, shp, bcs, ctypes.byref(sb), ctypes.byref(wb)))
            self.state_bytes = sb.value
            self.work_bytes = wb.value
            # torch's caching allocator returns 512-byte aligned blocks
            self.buf_a = torch.empty(self.state_bytes, dtype=torch.uint8, device=self.device)
            self.buf_b = torch.empty(self.state_bytes, dtype=torch.uint8, device=self.device)
            self.work = torch.zeros(self.work_bytes, dtype=torch.uint8, device=self.device)
            self._check(self.lib.lbm_bind(h, self.buf_a.data_ptr(), self.buf_b.data_ptr(),
                                          self.state_bytes, self.work.data_ptr(),
                                          self.work_bytes, self.stream.cuda_stream))

    # -- helpers -----------------------------------------------------------
    def _check(self, rc: int, h="self"):
        if rc != 0:
            msg = ""
            if h is not None and getattr(self, "h", None) is not None:
                msg = self.lib.lbm_last_error(self.h).decode()
            raise LbmError(rc, msg)

    def _field(self, a, rows=None):
        t = self.torch
        x = t.as_tensor(a, device=self.device, dtype=t.float32)
        x = x.reshape(-1) if rows is None else x.reshape(rows, self.N)
        if x.numel() != self.N * (rows or 1):
            raise LbmError(-1, "field has the wrong number of entries")
        return x.contiguous()

    @property
    def gamma(self) -> float:
        return (self.D + self.n + 2.0) / (self.D + self.n)

    # -- API -----------------------------------------------------------------
    def set_macro(self, rho, u, T):
        """Equilibrium state from (rho[N], u[D, N], T[N]); any array-likes."""
        with self.torch.cuda.device(self.device):
            r = self._field(rho)
            uu = self._field(u, self.D)
            tt = self._field(T)
            self._keep = (r, uu, tt)  # alive until the stream has consumed them
            self._check(self.lib.lbm_set_macro(self.h, r.data_ptr(), uu.data_ptr(), tt.data_ptr()))

    def step(self, k: int = 1):
        with self.torch.cuda.device(self.device):
            self._check(self.lib.lbm_step(self.h, int(k)))

    def moments(self):
        """(rho[N], u[D, N], T[N]) as float32 CUDA tensors."""
        t = self.torch
        with t.cuda.device(self.device):
            rho = t.empty(self.N, dtype=t.float32, device=self.device)
            u = t.empty(self.D, self.N, dtype=t.float32, device=self.device)
            T = t.empty(self.N, dtype=t.float32, device=self.device)
            self._check(self.lib.lbm_get_moments(self.h, rho.data_ptr(), u.data_ptr(), T.data_ptr()))
            return rho, u, T

    def conservation(self, check: bool = True) -> np.ndarray:
        """[sum rho, sum rho u (D), sum rho(E+u^2/2), max|sum_j h_j - 1|]."""
        out = (ctypes.c_double * (3 + self.D))()
        with self.torch.cuda.device(self.device):
            rc = self.lib.lbm_conservation(self.h, out)
        if rc != 0 and (check or rc != -4):
            self._check(rc)
        return np.array(out[:])

    def state(self):
        """(ft[Q, N], fr[Qr, N]) float32 CUDA tensors in canonical order."""
        t = self.torch
        with t.cuda.device(self.device):
            ft = t.empty(self.Q, self.N, dtype=t.float32, device=self.device)
            fr = t.empty(max(self.Qr, 1), self.N, dtype=t.float32, device=self.device)
            self._check(self.lib.lbm_get_state(self.h, ft.data_ptr(), fr.data_ptr()))
            return ft, fr[:self.Qr]

    def set_state(self, ft, fr=None):
        t = self.torch
        with t.cuda.device(self.device):
            a = self._field(ft, self.Q)
            b = self._field(fr, self.Qr) if self.Qr else t.zeros(1, device=self.device)
            self._keep = (a, b)
            self._check(self.lib.lbm_set_state(self.h, a.data_ptr(), b.data_ptr()))

    def sample(self, nodes):
        """All populations of the given nodes (indices x + X (y + Y z)) as a
        [len(nodes), Q + Qr] float32 array (lbm_sample_state)."""
        t = self.torch
        with t.cuda.device(self.device):
            idx = t.as_tensor(np.asarray(nodes, dtype=np.int64), device=self.device)
            out = t.empty((idx.numel(), self.Q + self.Qr), dtype=t.float32, device=self.device)
            self._check(self.lib.lbm_sample_state(self.h, idx.data_ptr(), idx.numel(),
                                                  out.data_ptr()))
            return out.cpu().numpy()

    def status(self) -> int:
        with self.torch.cuda.device(self.device):
            return self.lib.lbm_status(self.h)

    @property
    def steps(self) -> int:
        return self.lib.lbm_steps(self.h)

    @property
    def launches(self) -> int:
        return self.lib.lbm_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            self.lib.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LbmBatch:
    """An ensemble of independent 1-D problems (D1Q7 + D1Q7, copy ends)
    advanced together by one persistent launch (include/lbm.h, lbm_batch_*).

    ``lengths``, ``n`` and ``tau`` give each problem's node count, rotational
    degrees of freedom and relaxation time.  Macro fields are concatenated:
    problem k occupies nodes ``offsets[k] : offsets[k] + lengths[k]``.
    """

    def __init__(self, lengths, n, tau, mode: str = "fd", m_fd: int = 10, device=None,
                 stream=None):
        import torch

        self.torch = torch
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise LbmError(-3, "no CUDA device")
        self.device = torch.device(device if device is not None else "cuda")
        self.lengths = np.asarray(lengths, dtype=np.int64)
        self.count = int(self.lengths.size)
        self.offsets = np.concatenate([[0], np.cumsum(self.lengths)[:-1]]).astype(np.int64)
        nn = np.ascontiguousarray(n, dtype=np.int32)
        tt = np.ascontiguousarray(tau, dtype=np.float64)
        L = np.ascontiguousarray(self.lengths)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            h = ctypes.c_void_p()
            rc = self.lib.lbm_batch_create(
                self.count, L.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                tt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), MODES[mode], int(m_fd),
                ctypes.byref(h))
            if rc != 0:
                raise LbmError(rc, "lbm_batch_create")
            self.h = h
            sb, wb, tn = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int64()
            self._check(self.lib.lbm_batch_sizes(h, ctypes.byref(sb), ctypes.byref(wb),
                                                 ctypes.byref(tn)))
            self.state_bytes, self.work_bytes, self.N = sb.value, wb.value, tn.value
            self.buf_a = torch.empty(self.state_bytes, dtype=torch.uint8, device=self.device)
            self.buf_b = torch.empty(self.state_bytes, dtype=torch.uint8, device=self.device)
            self.work = torch.zeros(self.work_bytes, dtype=torch.uint8, device=self.device)
            self._check(self.lib.lbm_batch_bind(h, self.buf_a.data_ptr(), self.buf_b.data_ptr(),
                                                self.state_bytes, self.work.data_ptr(),
                                                self.work_bytes, self.stream.cuda_stream))

    def _check(self, rc: int):
        if rc != 0:
            raise LbmError(rc, self.lib.lbm_batch_last_error(self.h).decode())

    def _field(self, a):
        t = self.torch
        x = t.as_tensor(a, device=self.device, dtype=t.float32).reshape(-1).contiguous()
        if x.numel() != self.N:
            raise LbmError(-1, "field has the wrong number of entries")
        return x

    def set_macro(self, rho, u, T):
        with self.torch.cuda.device(self.device):
            r, uu, tt = self._field(rho), self._field(u), self._field(T)
            self._keep = (r, uu, tt)
            self._check(self.lib.lbm_batch_set_macro(self.h, r.data_ptr(), uu.data_ptr(),
                                                     tt.data_ptr()))

    def run(self, k: int):
        with self.torch.cuda.device(self.device):
            self._check(self.lib.lbm_batch_run(self.h, int(k)))

    def moments(self):
        t = self.torch
        with t.cuda.device(self.device):
            rho = t.empty(self.N, dtype=t.float32, device=self.device)
            u = t.empty(self.N, dtype=t.float32, device=self.device)
            T = t.empty(self.N, dtype=t.float32, device=self.device)
            self._check(self.lib.lbm_batch_get_moments(self.h, rho.data_ptr(), u.data_ptr(),
                                                       T.data_ptr()))
            return rho, u, T

    def status(self):
        """(per-problem status words, number of problems flagged)."""
        st = (ctypes.c_int * self.count)()
        bad = ctypes.c_int()
        with self.torch.cuda.device(self.device):
            self._check(self.lib.lbm_batch_status(self.h, st, ctypes.byref(bad)))
        return np.array(st[:]), bad.value

    def set_problems(self, n, tau):
        """New rotational degree counts and relaxation times for the same
        problem lengths (lbm_batch_set_problems); set_macro must follow."""
        nn = np.ascontiguousarray(np.broadcast_to(n, (self.count,)), dtype=np.int32)
        tt = np.ascontiguousarray(np.broadcast_to(tau, (self.count,)), dtype=np.float64)
        with self.torch.cuda.device(self.device):
            self._check(self.lib.lbm_batch_set_problems(
                self.h, nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                tt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def set_watch(self, lo=None, hi=None):
        """Only nodes [lo[k], hi[k]) of problem k set its status word
        (lbm_batch_set_watch); no arguments: whole problems."""
        if lo is None:
            self._check(self.lib.lbm_batch_set_watch(self.h, None, None))
            return
        ll = np.ascontiguousarray(np.broadcast_to(lo, (self.count,)), dtype=np.int32)
        hh = np.ascontiguousarray(np.broadcast_to(hi, (self.count,)), dtype=np.int32)
        with self.torch.cuda.device(self.device):
            self._check(self.lib.lbm_batch_set_watch(
                self.h, ll.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                hh.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))

    def set_block(self, threads: int, blocks_per_sm: int = 0):
        self._check(self.lib.lbm_batch_set_block(self.h, int(threads), int(blocks_per_sm)))

    def autotune(self, sample_steps: int = 20):
        """(threads per block, resident blocks per SM) of the fastest launch."""
        t, b = ctypes.c_int(), ctypes.c_int()
        with self.torch.cuda.device(self.device):
            self._check(self.lib.lbm_batch_autotune(self.h, int(sample_steps), ctypes.byref(t),
                                                    ctypes.byref(b)))
        return t.value, b.value

    @property
    def launches(self) -> int:
        return self.lib.lbm_batch_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            self.lib.lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
