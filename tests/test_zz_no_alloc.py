"""lbm_conservation_noalloc: the conservation sums for callers that cannot
hand the library any device scratch memory (their own allocator owns the
GPU, or their memory budget is fixed before the run).  Its partial sums live
in a static device array inside liblbm.so, so the call allocates nothing.

Checked through the C ABI against lbm_conservation (which uses the bound work
buffer) on two calls in a row, within the tolerance of the other
conservation checks (1e-6 relative; both run the same reduction kernel), for
every lattice, the 16-bit storages and a grid whose reduction uses the
largest block count (4 per SM).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1606_06107_gb300 import workloads

pytestmark = pytest.mark.gpu


def _noalloc(sim, state_ptr):
    out = (ctypes.c_double * (3 + sim.D))()
    rc = sim.lib.lbm_conservation_noalloc(sim.h, state_ptr, sim.stream.cuda_stream, out)
    return rc, np.array(out[:])


def _current_state(sim):
    return sim.buf_a.data_ptr() if sim.steps % 2 == 0 else sim.buf_b.data_ptr()


@pytest.mark.parametrize("kind,shape,n,storage", [
    ("D2Q49", (300, 41), 3, "f32"),
    ("D1Q7", (1000,), 4, "f32"),
    ("D2Q37", (64, 20), 0, "f32"),
    ("D2Q49", (100, 37), 3, "bf16"),
    ("D3Q343", (16, 16, 16), 0, "f16"),
    ("D3Q343", (12, 10, 9), 4, "bf16"),
    ("D2Q49", (90, 33), 3, "bf16_node"),
    # 196,608 nodes want 768 reduction blocks: capped at 4 per SM
    ("D2Q49", (2048, 96), 3, "f16"),
])
def test_noalloc_matches_bound_conservation(kind, shape, n, storage):
    from paper_1606_06107_gb300 import Lbm
    wl = workloads.smooth_random(shape, seed=8, kind=kind, n=n, u_mean=(0.05,) * len(shape))
    sim = Lbm(kind, wl.n, wl.tau, wl.shape, wl.bc, storage=storage)
    sim.set_macro(wl.rho, wl.u, wl.T)
    for steps in (3, 4):  # two calls in a row, on states in both buffers
        sim.step(steps)
        ref = sim.conservation()
        rc, got = _noalloc(sim, _current_state(sim))
        assert rc == 0, sim.lib.lbm_last_error(sim.h)
        scale = max(abs(ref[0]), 1.0)
        assert np.all(np.abs(got - ref) <= 1e-6 * scale), (got, ref)
    # the same state twice in a row gives the same sums
    rc, again = _noalloc(sim, _current_state(sim))
    assert rc == 0 and np.array_equal(again, got)


def test_noalloc_rejects_bad_pointers():
    """Null, misaligned and host pointers are refused on the host, before
    any kernel could read them."""
    import torch
    from paper_1606_06107_gb300 import Lbm
    wl = workloads.smooth_random((40,), seed=1, kind="D1Q7", n=2)
    sim = Lbm(wl.kind, wl.n, wl.tau, wl.shape, wl.bc)
    sim.set_macro(wl.rho, wl.u, wl.T)
    out = (ctypes.c_double * 4)()
    lib = sim.lib
    assert lib.lbm_conservation_noalloc(sim.h, None, None, out) == -1
    assert lib.lbm_conservation_noalloc(sim.h, sim.buf_a.data_ptr() + 4, None, out) == -1
    assert lib.lbm_conservation_noalloc(sim.h, sim.buf_a.data_ptr(), None, None) == -1
    # pinned host memory, 256-byte aligned
    pinned = torch.empty(sim.state_bytes + 512, dtype=torch.uint8, pin_memory=True)
    p = (pinned.data_ptr() + 255) // 256 * 256
    assert lib.lbm_conservation_noalloc(sim.h, p, None, out) == -1
    # ordinary (unregistered) host memory, 256-byte aligned
    host = np.zeros(sim.state_bytes + 512, dtype=np.uint8)
    q = (host.ctypes.data + 255) // 256 * 256
    assert lib.lbm_conservation_noalloc(sim.h, q, None, out) == -1
    # the valid call still works afterwards
    rc, _ = _noalloc(sim, _current_state(sim))
    assert rc == 0, lib.lbm_last_error(sim.h)
