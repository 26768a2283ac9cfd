"""The window geometry of the surrogate's fallback (host logic): the
interiors tile the tube, each lies inside its window, and every interior
node is at least `margin` nodes (the FD dependency cone of K steps, 2K)
from any window edge that is not a tube end, which is what makes the
method on a window exact on its interior."""
import numpy as np
import pytest

from paper_1606_06107_gb300.surrogate import fallback_windows


@pytest.mark.parametrize("margin", [0, 1, 7, 64])
def test_windows_cover_the_tube_with_exact_interiors(margin):
    for L in list(range(1, 70)) + [100, 255, 256, 511, 512, 640, 1000, 4096, 4097]:
        for width in (1, 2, 3, 7, 50, 100, 512, 5000):
            S, istart, wstart = fallback_windows(L, width, margin)
            w = min(max(width, 1), L)
            if S == L:                       # one window: the whole tube
                assert istart.tolist() == [0] and wstart.tolist() == [0]
                continue
            assert S == w + 2 * margin < L
            covered = np.zeros(L, bool)
            for i0, s0 in zip(istart.tolist(), wstart.tolist()):
                assert 0 <= s0 and s0 + S <= L                  # window inside the tube
                assert s0 <= i0 and i0 + w <= s0 + S            # interior inside the window
                covered[i0:i0 + w] = True
                if s0 > 0:                                      # artificial left edge
                    assert i0 - s0 >= margin
                if s0 + S < L:                                  # artificial right edge
                    assert (s0 + S - 1) - (i0 + w - 1) >= margin
            assert covered.all(), (L, width, margin)
            assert istart.size == -(-L // w)


def test_the_bench_shape():
    """4096-node tubes, 512-node interiors, K = 32: 8 windows of 640 nodes,
    each short enough for the shared-memory ensemble form (<= 864)."""
    S, istart, wstart = fallback_windows(4096, 512, 64)
    assert S == 640 and S <= 864
    assert istart.tolist() == [512 * j for j in range(8)]
    assert wstart.tolist() == [0, 448, 960, 1472, 1984, 2496, 3008, 3456]
