"""The paper's weak-scaling measure (Sec. 5, Fig. 3) on one GPU: trial moves per walker to finish
the first Wang-Landau iteration.  The windows have a fixed size (about 64 bins at 75 % overlap) and their
number grows with the lattice; one serial walker over the whole range is the comparison.  From N = 128
to N = 8192 (5 to 509 windows) the windowed cost stays within a factor of 2 (it grows only with the
slowest of more walkers).  The serial cost grows roughly as N^2 (measured 0.30M -> 21M moves from
N = 128 to 1024)."""
import numpy as np
import pytest

import paper_1411_4212_gb300 as rw
from paper_1411_4212_gb300 import warmstart

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_first_iteration_cost_is_flat_with_windows_and_grows_without():
    J = (1.0, 0.5)
    sizes = (4, 8, 12, 16)
    jobs = {("rewl", L): warmstart.first_iteration_job(L, J, seed=100 + L) for L in sizes}
    jobs.update({("serial", L): warmstart.first_iteration_job(L, J, seed=200 + L, serial=True) for L in (4, 8)})
    with rw.Batch(list(jobs.values())) as b:
        ok, _ = b.run_to_convergence(max_intervals=20000, check_every=4)
    assert ok
    moves, windows = {}, {k: j.h for k, j in jobs.items()}
    for k, j in jobs.items():
        w = j.walkers()
        assert np.all(w["stage"] >= 1) and np.all(w["lnf"] == 0.5)
        moves[k] = w["steps"].mean()
        j.close()
    print({f"{k[0]} L={k[1]} ({windows[k]} windows)": f"{v:.0f}" for k, v in moves.items()})
    assert windows[("rewl", 8)] == 61 and windows[("rewl", 4)] == 5 and windows[("rewl", 16)] == 509
    rewl = [moves[("rewl", L)] for L in sizes]
    assert max(rewl) < 2 * min(rewl), moves
    assert moves[("serial", 8)] > 20 * moves[("serial", 4)], moves
    assert moves[("serial", 8)] > 20 * moves[("rewl", 8)], moves
