"""The learned warm start end to end at a small scale: a corpus of converged REWL runs over random
couplings (bcc L = 4, 5), the network trained on it by the library's kernels, then held-out
couplings at L = 5 run from the network's ln g at ln f0 = 2^-7 and from scratch.  Plain Wang-Landau
finishes both, so the warm runs must reach the accuracy of a cold run (centred rms against an
independent cold run) in fewer moves: averaged over 4 coupling sets x 3 replicas, whose spread in
moves to converge is under 15 % per run."""
import numpy as np
import pytest

from paper_1411_4212_gb300 import warmstart, workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_warm_start_saves_moves_at_equal_accuracy():
    x, t, off, meta = warmstart.corpus(sizes=(4, 5), per_size=32, lnf_final=1e-4)
    assert meta["converged"] and len(off) == 65
    net, hist = warmstart.train(x, t, off, steps=3000, lr=2e-3)
    assert hist[-1] < hist[0] / 1000
    held_out = [workloads.random_couplings(10_000 + i) for i in range(4)]
    ok, res, _ = warmstart.warm_vs_cold(net, 5, held_out, lnf_final=1e-5, replicas=3)
    assert ok
    cold = np.mean([m for r in res for m in r["cold_moves"]])
    warm = np.mean([m for r in res for m in r["warm_moves"]])
    cold_rms = np.mean([v for r in res for v in r["cold_rms"]])
    warm_rms = np.mean([v for r in res for v in r["warm_rms"]])
    for r in res:
        assert r["prediction_rms"] < 1.0, r
    assert warm_rms <= 1.5 * cold_rms + 0.02, (warm_rms, cold_rms)
    assert warm < 0.95 * cold, (warm, cold)
    net.close()
