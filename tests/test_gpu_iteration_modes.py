"""The two readings of when a walker moves on to its next Wang-Landau iteration (Sec. 4.3): on its
own flat histogram (as written; the default), or together with the other walkers of its window
once all of them are flat, after averaging their ln g.  Production runs of both, 8 seeds each, on
a converging range; the accuracy (centred rms of each run's ln g against the mean of all 16) and
the moves to converge are compared."""
import numpy as np
import pytest

import paper_1411_4212_gb300 as rw

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_window_and_walker_iteration_converge_to_the_same_density_of_states():
    cfg = dict(kind=rw.BCC, mode=rw.PRODUCTION, L=4, J=(1.0, 0.5), e_min=-400.0, e_max=0.0, n_bins=120,
               n_windows=3, walkers_per_window=4, overlap=0.75, flatness=0.8, lnf_final=1e-5,
               exchange_interval=2000, group_size=1)
    jobs = {(it, s): rw.REWL(iteration=it, seed=100 + s, **cfg) for it in (0, 1) for s in range(8)}
    with rw.Batch(list(jobs.values())) as b:
        ok, _ = b.run_to_convergence(max_intervals=100000, check_every=16)
    assert ok
    lng = {k: j.merge()[0] for k, j in jobs.items()}
    ref = np.mean(list(lng.values()), axis=0)

    def rms(a):
        d = a - ref
        return float(np.sqrt(np.mean((d - d.mean()) ** 2)))

    res = {}
    for it in (0, 1):
        r = [rms(lng[(it, s)]) for s in range(8)]
        mv = [jobs[(it, s)].walkers()["steps"].mean() for s in range(8)]
        res[it] = (np.mean(r), np.mean(mv))
    print(f"walker iteration: rms {res[0][0]:.4f}, moves {res[0][1]:.3g}; "
          f"window iteration: rms {res[1][0]:.4f}, moves {res[1][1]:.3g}")
    for it in (0, 1):
        assert res[it][0] < 0.05
    # both readings estimate the same g(E): the mean of each mode's runs agree within their spread
    m0 = np.mean([lng[(0, s)] for s in range(8)], axis=0)
    m1 = np.mean([lng[(1, s)] for s in range(8)], axis=0)
    d = m0 - m1
    assert np.sqrt(np.mean((d - d.mean()) ** 2)) < 3 * max(res[0][0], res[1][0]) / np.sqrt(8) + 0.01
    for j in jobs.values():
        j.close()
