"""The learned warm start end to end at a small scale: a corpus of converged REWL runs over random
couplings (bcc L = 4, 5), the network trained on it by the library's kernels, then 8 held-out
coupling sets at L = 4 and at L = 5, each run 4 times from the network's ln g (ln f0 = 2^-10) and 4
times from scratch, to ln f = 1e-5.  Plain Wang-Landau finishes every run, so the warm runs must
reach the accuracy of a cold run (centred rms against an independent cold run) and, pooled over
the 64 runs per side, need fewer moves.  (Single runs differ by 10-30 % in moves to converge and
the warm start saves about 10 % at these sizes, so fewer runs could not resolve the gain.)"""
import numpy as np
import pytest

from paper_1411_4212_gb300 import warmstart, workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_warm_start_saves_moves_at_equal_accuracy():
    x, t, off, meta = warmstart.corpus(sizes=(4, 5), per_size=32, lnf_final=1e-4)
    assert meta["converged"] and len(off) == 65
    net, hist = warmstart.train(x, t, off, steps=3000, lr=2e-3)
    assert hist[-1] < hist[0] / 1000
    held_out = [workloads.random_couplings(10_000 + i) for i in range(8)]
    cold, warm, cold_rms, warm_rms = [], [], [], []
    for L in (4, 5):
        ok, res, _ = warmstart.warm_vs_cold(net, L, held_out, lnf_final=1e-5, replicas=4, lnf0=2.0 ** -10)
        assert ok
        for r in res:
            assert r["prediction_rms"] < 0.5, r          # the network has learned ln g (rms 0.1-0.2)
            cold += r["cold_moves"]
            warm += r["warm_moves"]
            cold_rms += r["cold_rms"]
            warm_rms += r["warm_rms"]
    ratio = np.mean(warm) / np.mean(cold)
    print(f"warm/cold moves to converge: {ratio:.3f} over {len(warm)} runs per side; "
          f"rms warm {np.mean(warm_rms):.3f} cold {np.mean(cold_rms):.3f}")
    assert np.mean(warm_rms) <= 1.5 * np.mean(cold_rms) + 0.02
    assert ratio < 1.0
    net.close()
