"""The learned warm start end to end.
1. A corpus of converged REWL runs over random couplings (bcc L = 4, 5, 6).
2. The network, trained on it by the library's kernels.
3. Held-out coupling sets at L = 6 and L = 8, each run 4 times from the network's ln g (ln f0 = 2^-10)
   and 4 times from scratch, to ln f = 1e-5.

Accuracy is judged against an independent reference per coupling set: the mean of 3 further plain runs
converged to ln f = 1e-6.  Plain Wang-Landau finishes every warm run, so:
- the warm runs must be as close to the reference as the plain runs.  The per-set excess rms of warm
  over plain must not exceed twice its standard error over the sets (a paired test);
- pooled over the runs, the warm runs must need fewer moves to converge.
Single runs differ by 10-30 % in moves, and the gain is 10-25 % at these sizes, so fewer runs could
not resolve it."""
import numpy as np
import pytest

from paper_1411_4212_gb300 import warmstart, workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_warm_start_saves_moves_at_equal_accuracy():
    x, t, off, meta = warmstart.corpus(sizes=(4, 5, 6), per_size=32, lnf_final=1e-4)
    assert meta["converged"] and len(off) == 97
    net, hist = warmstart.train(x, t, off, steps=3000, lr=2e-3)
    assert hist[-1] < hist[0] / 1000
    held_out = [workloads.random_couplings(10_000 + i) for i in range(6)]
    cold, warm, excess, pred = [], [], [], []
    for L in (6, 8):
        ok, res, _ = warmstart.warm_vs_cold(net, L, held_out, lnf_final=1e-5, replicas=4, lnf0=2.0 ** -10,
                                            n_ref=3, lnf_ref=1e-6, seed0=900 + 10 * L)
        assert ok
        for r in res:
            pred.append(r["prediction_rms"] / (2 * L ** 3))
            cold += r["cold_moves"]
            warm += r["warm_moves"]
            excess.append(np.mean(r["warm_rms"]) - np.mean(r["cold_rms"]))
    d, se = warmstart.paired_excess(excess, np.zeros(len(excess)))
    ratio = np.mean(warm) / np.mean(cold)
    z = (np.mean(cold) - np.mean(warm)) / np.sqrt(np.var(cold, ddof=1) / len(cold) + np.var(warm, ddof=1) / len(warm))
    print(f"warm/plain moves to converge {ratio:.3f} over {len(warm)} runs per side (gain {z:.1f} standard errors); "
          f"excess rms of warm over plain against the reference {d:+.4f} +- {se:.4f} over {len(excess)} sets")
    print(f"prediction rms per spin (held out, up to L = 8 from a corpus at L <= 6): max {max(pred):.2e}")
    assert max(pred) < 3e-3                       # the network has learned ln g
    assert d <= 2.0 * se
    assert ratio < 1.0
    net.close()
