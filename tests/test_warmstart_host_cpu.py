"""Host logic of the warm-start workflow (no GPU): the window count of the restricted range keeps
the windows about as wide as the L = 8 layout at every lattice size, so a walker's work to converge
does not grow with L (Sec. 4.3 window layout, W = ceil(B / (1 + (h - 1)(1 - o))) with B = N bins)."""
import pytest

import oracle
from paper_1411_4212_gb300 import warmstart


def test_table_sizes_are_kept():
    for L, h in warmstart.WINDOWS.items():
        assert warmstart.windows_for(L) == h


@pytest.mark.parametrize("L,h", [(12, 61), (16, 149), (24, 509), (32, 1211)])
def test_larger_lattices_keep_the_window_width(L, h):
    N = 2 * L ** 3
    assert warmstart.windows_for(L) == h
    W8, _ = oracle.window_layout(2 * 8 ** 3, warmstart.windows_for(8), 0.75)
    W, starts = oracle.window_layout(N, h, 0.75)
    assert W8 == warmstart.WINDOW_BINS
    assert abs(W - W8) <= 2
    # the windows tile [0, N) with the stated overlap: first at 0, last ending at N
    assert starts[0] == 0 and starts[-1] + W == N


def test_window_count_grows_with_the_lattice():
    hs = [warmstart.windows_for(L) for L in range(4, 41)]
    assert all(a <= b for a, b in zip(hs, hs[1:]))
