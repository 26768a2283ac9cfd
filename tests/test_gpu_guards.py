"""Out-of-bounds writes, caught without a sanitizer: every device buffer a
kernel writes (and the inputs it reads) sits inside a larger allocation
filled with a canary byte; after the calls the bytes on both sides of each
buffer must be unchanged.  Ragged sizes make the last tile, block or row of
every kernel reach past the data."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GUARD = 4096          # bytes on each side, a multiple of the library's 256-byte alignment
CANARY = 0xA5


def _t():
    import torch
    return torch


class Guarded:
    """`nbytes` usable bytes with a canary band on both sides."""

    def __init__(self, nbytes, fill=None):
        torch = _t()
        self.n = int(nbytes)
        self.raw = torch.full((self.n + 2 * GUARD,), CANARY, dtype=torch.uint8, device="cuda")
        if fill is not None:
            self.view(fill.dtype)[:] = fill

    @property
    def ptr(self):
        return ctypes.c_void_p(self.raw.data_ptr() + GUARD)

    def view(self, dtype):
        return self.raw[GUARD:GUARD + self.n].view(dtype)

    def intact(self):
        return bool((self.raw[:GUARD] == CANARY).all()) and \
            bool((self.raw[GUARD + self.n:] == CANARY).all())


def f32(a):
    torch = _t()
    return torch.tensor(np.asarray(a, np.float32).ravel(), device="cuda")


def guarded_f32(a):
    x = f32(a)
    return Guarded(x.numel() * 4, fill=x)


LBM_CASES = [  # lattice, n, shape, bc, mode, storage
    ("D1Q7", 4, (1000,), ("copy",), "fd", "f32"),
    ("D1Q7", 0, (37,), ("periodic",), "stream", "f16"),
    ("D2Q49", 3, (130, 7), ("periodic", "copy"), "stream", "f32"),
    ("D2Q37", 3, (65, 5), ("copy", "periodic"), "fd", "bf16"),
    ("D2Q49", 2, (129, 3), ("copy", "copy"), "fd", "f16"),
    ("D3Q343", 2, (129, 3, 2), ("periodic", "copy", "periodic"), "stream", "f16"),
    ("D3Q343", 0, (33, 2, 3), ("periodic",) * 3, "stream", "f32"),
    ("D2Q49", 3, (131, 5), ("periodic", "copy"), "stream", "bf16"),
    ("D2Q49", 3, (130, 6), ("copy", "periodic"), "stream", "f16_node"),
    ("D2Q37", 0, (67, 3), ("periodic", "periodic"), "stream", "bf16_node"),
    ("D1Q7", 4, (259,), ("copy",), "stream", "bf16_node"),
]


@pytest.mark.parametrize("case", LBM_CASES)
def test_lbm_calls_write_only_their_buffers(lbmlib, case):
    from paper_1606_06107_gb300 import lbm, workloads
    torch = _t()
    kind, n, shape, bc, mode, storage = case
    D, Q = lbm.LATTICE_DIM[kind], lbm.LATTICE_Q[kind]
    Qr = 7 if n else 0
    N = int(np.prod(shape))
    lib = lbmlib
    h = ctypes.c_void_p()
    assert lib.lbm_create(D, lbm.LATTICES[kind], n, 2.0 / 3.0, ctypes.byref(h)) == 0
    try:
        assert lib.lbm_set_mode(h, lbm.MODES[mode], 10) == 0
        assert lib.lbm_set_storage(h, lbm.STORAGES[storage]) == 0
        shp = (ctypes.c_int64 * 3)(*shape, *([1] * (3 - D)))
        bcs = (ctypes.c_int * 3)(*[lbm.BCS[b] for b in bc], *([0] * (3 - D)))
        sb, wb = ctypes.c_size_t(), ctypes.c_size_t()
        assert lib.lbm_set_grid(h, shp, bcs, ctypes.byref(sb), ctypes.byref(wb)) == 0
        a, b = Guarded(sb.value), Guarded(sb.value)
        work = Guarded(wb.value, fill=torch.zeros(wb.value, dtype=torch.uint8, device="cuda"))
        s = torch.cuda.current_stream().cuda_stream
        assert lib.lbm_bind(h, a.ptr, b.ptr, sb.value, work.ptr, wb.value, s) == 0
        wl = workloads.smooth_random(shape, seed=5, kind=kind, n=n, bc=bc)
        rho, u, T = guarded_f32(wl.rho), guarded_f32(wl.u), guarded_f32(wl.T)
        assert lib.lbm_set_macro(h, rho.view(torch.float32).data_ptr(),
                                 u.view(torch.float32).data_ptr(),
                                 T.view(torch.float32).data_ptr()) == 0
        assert lib.lbm_step(h, 3) == 0
        mo = [Guarded(N * 4), Guarded(D * N * 4), Guarded(N * 4)]
        assert lib.lbm_get_moments(h, *(m.ptr for m in mo)) == 0
        out = (ctypes.c_double * 8)()
        assert lib.lbm_conservation(h, out) == 0
        ft, fr = Guarded(Q * N * 4), Guarded(max(Qr, 1) * N * 4)
        assert lib.lbm_get_state(h, ft.ptr, fr.ptr) == 0
        nodes = Guarded(3 * 8, fill=torch.tensor([0, N // 2, N - 1], dtype=torch.int64,
                                                 device="cuda"))
        samp = Guarded(3 * (Q + Qr) * 4)
        assert lib.lbm_sample_state(h, nodes.ptr, 3, samp.ptr) == 0
        assert lib.lbm_set_state(h, ft.ptr, fr.ptr) == 0
        assert lib.lbm_step(h, 2) == 0
        torch.cuda.synchronize()
        assert lib.lbm_status(h) == 0
        for name, g in [("state a", a), ("state b", b), ("work", work), ("rho", rho), ("u", u),
                        ("T", T), ("moments rho", mo[0]), ("moments u", mo[1]),
                        ("moments T", mo[2]), ("ft", ft), ("fr", fr), ("nodes", nodes),
                        ("sample", samp)]:
            assert g.intact(), name
    finally:
        lib.lbm_destroy(h)


def test_ensemble_writes_only_its_buffers(lbmlib):
    from paper_1606_06107_gb300 import workloads
    torch = _t()
    lib = lbmlib
    lengths = np.array([1, 7, 130, 257, 1000], dtype=np.int64)
    ns = np.array([2, 4, 0, 6, 7], dtype=np.int32)
    taus = np.array([0.7, 0.6, 0.9, 0.55, 1.0])
    h = ctypes.c_void_p()
    assert lib.lbm_batch_create(len(lengths), lengths.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                taus.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1, 10,
                                ctypes.byref(h)) == 0
    try:
        sb, wb, tn = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int64()
        assert lib.lbm_batch_sizes(h, ctypes.byref(sb), ctypes.byref(wb), ctypes.byref(tn)) == 0
        N = tn.value
        a, b = Guarded(sb.value), Guarded(sb.value)
        work = Guarded(wb.value, fill=torch.zeros(wb.value, dtype=torch.uint8, device="cuda"))
        s = torch.cuda.current_stream().cuda_stream
        assert lib.lbm_batch_bind(h, a.ptr, b.ptr, sb.value, work.ptr, wb.value, s) == 0
        fields = [np.concatenate(x) for x in zip(*[workloads._two_state_1d(
            int(L), (1.0, 0.0, 1.0), (0.8, 0.0, 0.7)) for L in lengths])]
        rho, u, T = (guarded_f32(f) for f in fields)
        assert lib.lbm_batch_set_macro(h, rho.ptr, u.ptr, T.ptr) == 0
        assert lib.lbm_batch_run(h, 17) == 0
        mo = [Guarded(N * 4) for _ in range(3)]
        assert lib.lbm_batch_get_moments(h, *(m.ptr for m in mo)) == 0
        torch.cuda.synchronize()
        for name, g in [("a", a), ("b", b), ("work", work), ("rho", rho), ("u", u), ("T", T),
                        ("m0", mo[0]), ("m1", mo[1]), ("m2", mo[2])]:
            assert g.intact(), name
    finally:
        lib.lbm_batch_destroy(h)


@pytest.mark.parametrize("impl", [0, 1, 2, 3])
def test_convolutions_write_only_their_buffers(lbmlib, impl):
    """Ragged tube length (77 positions: a 128-row tile and a 64-row weight
    block both reach past it) and three tubes."""
    torch = _t()
    lib = lbmlib
    B, L, C, k, d = 3, 77, 128, 5, 2
    n = B * L * C
    rng = np.random.default_rng(0)
    bf = lambda a: Guarded(a.size * 2, fill=torch.tensor(np.asarray(a, np.float32).ravel()).to(
        torch.bfloat16).cuda())
    x, zp, gz = bf(rng.normal(0, 1, n)), bf(rng.normal(0, 1, n)), bf(rng.normal(0, 1, n))
    w32 = guarded_f32(rng.normal(0, 0.05, k * C * C))
    wb, wt = Guarded(k * C * C * 2), Guarded(k * C * C * 2)
    bias = guarded_f32(rng.normal(0, 0.1, C))
    y, z, gzp = Guarded(n * 2), Guarded(n * 2), Guarded(n * 2)
    gx = guarded_f32(rng.normal(0, 1, n))
    gw = guarded_f32(np.zeros(k * C * C))
    st = Guarded(4, fill=torch.zeros(1, dtype=torch.int32, device="cuda"))
    s = torch.cuda.current_stream().cuda_stream
    assert lib.lbm_nn_cast_weights(w32.ptr, wb.ptr, wt.ptr, 1, C, k, s) == 0
    assert lib.lbm_nn_conv_forward(x.ptr, wb.ptr, bias.ptr, y.ptr, z.ptr, B, L, C, k, d, impl,
                                   st.ptr, s) == 0
    assert lib.lbm_nn_conv_backward_data(gz.ptr, wt.ptr, gx.ptr, zp.ptr, gzp.ptr, B, L, C, k, d,
                                         impl, st.ptr, s) == 0
    if impl != 2:
        assert lib.lbm_nn_conv_backward_weight(gz.ptr, x.ptr, gw.ptr, B, L, C, k, d, impl,
                                               st.ptr, s) == 0
    torch.cuda.synchronize()
    assert int(st.view(torch.int32)[0]) == 0
    for name, g in [("x", x), ("zprev", zp), ("gz", gz), ("w", w32), ("wb", wb), ("wt", wt),
                    ("bias", bias), ("y", y), ("z", z), ("gzprev", gzp), ("gx", gx),
                    ("gw", gw), ("status", st)]:
        assert g.intact(), name


def test_small_surrogate_kernels_write_only_their_buffers(lbmlib):
    torch = _t()
    lib = lbmlib
    B, L, C, P4 = 3, 77, 128, 4
    P = B * L
    rng = np.random.default_rng(1)
    s = torch.cuda.current_stream().cuda_stream
    feat = guarded_f32(rng.normal(0, 1, P * 4 * P4))
    Wl, bl = guarded_f32(rng.normal(0, 0.3, C * 4 * P4)), guarded_f32(rng.normal(0, 0.1, C))
    x0 = Guarded(P * C * 2)
    assert lib.lbm_nn_lift(feat.ptr, Wl.ptr, bl.ptr, x0.ptr, P, 4 * P4, C, s) == 0
    Wp, bp = guarded_f32(rng.normal(0, 0.1, 3 * P4 * C)), guarded_f32(np.zeros(3 * P4))
    out = Guarded(P * 3 * P4 * 4)
    assert lib.lbm_nn_head(x0.ptr, Wp.ptr, bp.ptr, out.ptr, P, C, 3 * P4, s) == 0
    gout = guarded_f32(rng.normal(0, 1, P * 3 * P4))
    gx, gz = Guarded(P * C * 4), Guarded(P * C * 2)
    gWp, gbp = guarded_f32(np.zeros(3 * P4 * C)), guarded_f32(np.zeros(3 * P4))
    assert lib.lbm_nn_head_backward(gout.ptr, x0.ptr, Wp.ptr, x0.ptr, gx.ptr, gz.ptr, gWp.ptr,
                                    gbp.ptr, P, C, 3 * P4, s) == 0
    gWl, gbl = guarded_f32(np.zeros(C * 4 * P4)), guarded_f32(np.zeros(C))
    assert lib.lbm_nn_lift_backward(gx.ptr, feat.ptr, gWl.ptr, gbl.ptr, P, 4 * P4, C, s) == 0
    gb = guarded_f32(np.zeros(C))
    assert lib.lbm_nn_bias_grad(gz.ptr, gb.ptr, P, C, s) == 0
    fields = [guarded_f32(1 + 0.1 * rng.random(B * L)) for _ in range(6)]
    hd, gam = guarded_f32(np.full(B, 2.5)), guarded_f32(np.full(B, 1.4))
    res, l1 = Guarded(B * 4), Guarded(B * 4)
    starts = Guarded(2 * B * 4)
    assert lib.lbm_nn_tube_checks(*(f.ptr for f in fields), hd.ptr, gam.ptr, res.ptr, l1.ptr,
                                  starts.ptr, 20, 4, B, L, 0, L, s) == 0
    rows = Guarded(2 * 8, fill=torch.tensor([2, 0], dtype=torch.int64, device="cuda"))
    offs = Guarded(2 * 4, fill=torch.tensor([5, 57], dtype=torch.int32, device="cuda"))
    packed = [Guarded(2 * 20 * 4) for _ in range(3)]
    assert lib.lbm_nn_gather(*(f.ptr for f in fields[:3]), rows.ptr, offs.ptr, 2, L, 20,
                             *(p.ptr for p in packed), s) == 0
    assert lib.lbm_nn_scatter(*(p.ptr for p in packed), rows.ptr, offs.ptr, 2, L, 20,
                              *(f.ptr for f in fields[3:]), s) == 0
    torch.cuda.synchronize()
    for name, g in [("feat", feat), ("x0", x0), ("out", out), ("gx", gx), ("gz", gz),
                    ("gWp", gWp), ("gbp", gbp), ("gWl", gWl), ("gbl", gbl), ("gb", gb),
                    ("res", res), ("l1", l1), ("starts", starts), ("rows", rows),
                    ("offs", offs)] + [(f"field{i}", f) for i, f in enumerate(fields)] + \
            [(f"packed{i}", p) for i, p in enumerate(packed)]:
        assert g.intact(), name
