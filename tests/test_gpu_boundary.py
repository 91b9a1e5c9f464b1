"""C-ABI entry points that the interval runner does not cover, against the FP64 oracle: a Wang-Landau
iteration per call (rewl_run_stage, Sec. 4.2) and its caps, the standalone replica-exchange round
(rewl_exchange, Sec. 4.3, Eq. 5), the three split launches of an interval (rewl_walk, rewl_exchange,
rewl_flatness), and the temperature of the specific-heat peak (rewl_peak_temperature, Sec. 4.1, Eq. 3)."""
import ctypes as C
import io
import json

import numpy as np
import pytest

import oracle
import paper_1411_4212_gb300 as rw
from rewl_pairs import assert_same_state, make_pair

pytestmark = pytest.mark.gpu

# bins about as wide as the temperature, so that a stage ends in seconds
CONVERGING = dict(L=4, J=(1.0, 0.5), e_min=-400.0, e_max=0.0, n_bins=120, n_windows=4, walkers_per_window=2,
                  lnf_final=1e-3, exchange_interval=5000, seed=3)


def test_run_stage_is_one_wang_landau_iteration_and_matches_oracle():
    """Trajectory mode: every rewl_run_stage call ends once each walker that was active at its start
    has halved ln f; the oracle, run for the same number of intervals, is in the same state bit for bit
    after every stage, up to convergence."""
    gpu, orc = make_pair(**CONVERGING)
    gpu.init_walkers()
    orc.init_walkers()
    n_stages = 0
    while True:
        w0 = gpu.walkers()
        st = gpu.run_stage()
        assert not st["capped"]
        orc.run_intervals(st["intervals"])
        assert_same_state(gpu, orc)
        w1 = gpu.walkers()
        active = w0["lnf"] >= CONVERGING["lnf_final"]
        assert np.all(w1["stage"][active] > w0["stage"][active])
        assert st["n_halved"] == int((w1["stage"] - w0["stage"]).sum())
        assert st["moves"] == st["intervals"] * CONVERGING["exchange_interval"] * gpu.n_slots
        assert st["accepts"] == int((w1["accepts"] - w0["accepts"]).sum())
        assert st["n_done"] == int(np.sum(w1["lnf"] < CONVERGING["lnf_final"]))
        assert st["min_lnf"] == w1["lnf"].min() and st["max_lnf"] == w1["lnf"].max()
        n_stages += 1
        if st["all_done"]:
            break
        assert n_stages < 40
    assert np.all(gpu.walkers()["lnf"] < CONVERGING["lnf_final"])
    lg, _ = gpu.merge()
    lo, _ = orc.merge()
    assert np.array_equal(lg.view(np.int64), lo.view(np.int64))
    gpu.close()


@pytest.mark.parametrize("cap", ["moves", "timeout"])
def test_stage_caps_end_the_stage_with_etimeout(cap):
    """A stage that cannot finish (bcc L = 16 over [E_gs, 0]: the windows are far from flat after a few
    intervals) is ended by max_moves_per_stage or timeout_s: REWL_ETIMEOUT, with the stage statistics
    of the work done filled in.  run_to_convergence stops at the capped stage."""
    kw = dict(max_moves_per_stage=4 * 10000) if cap == "moves" else dict(timeout_s=1e-6)
    g = rw.REWL(kind=rw.BCC, L=16, J=(1.0, 0.5), n_bins=2000, n_windows=16, walkers_per_window=4, lnf_final=1e-8,
                seed=2, exchange_interval=10000, mode=rw.PRODUCTION, **kw)
    lib = rw.load_library()
    st = rw.StageStats()
    rc = lib.rewl_run_stage(g._h, C.byref(st))
    assert rc == rw.ETIMEOUT
    assert b"max_moves_per_stage or timeout_s" in lib.rewl_last_error(g._h)
    assert st.intervals == 4 and st.moves == 4 * 10000 * g.n_slots
    assert 0 < st.accepts < st.moves and st.exchange_attempts > 0 and st.elapsed_ms > 0
    assert st.n_halved == 0 and st.all_done == 0 and st.max_lnf == 1.0
    w = g.walkers()
    assert np.all(w["steps"] == 4 * 10000)
    stages = g.run_to_convergence(max_stages=5)
    assert len(stages) == 1 and stages[0]["capped"] and stages[0]["intervals"] == 4
    g.close()


@pytest.mark.parametrize("m", [2, 3])
def test_standalone_exchange_rounds_match_oracle(m):
    """rewl_exchange alone, round after round (alternating window parity, the walker shift a + t/2),
    against the oracle's exchange round: the permutation, energies, bins, counters and round trips bit
    for bit, and the stats report the round's attempts and acceptances."""
    gpu, orc = make_pair(L=4, J=(1.0, 0.5), n_bins=200, n_windows=4, walkers_per_window=m, exchange_interval=3000,
                         seed=5, lnf_final=1e-3)
    gpu.init_walkers()
    orc.init_walkers()
    gpu.run_intervals(3)
    orc.run_intervals(3)
    for _ in range(8):
        a0, b0 = orc.exchange_counts()
        st = gpu.exchange()
        orc.exchange()
        a1, b1 = orc.exchange_counts()
        assert st["exchange_attempts"] == int((a1 - a0).sum()) and st["exchange_accepts"] == int((b1 - b0).sum())
        assert st["moves"] == 0 and st["intervals"] == 0
        assert_same_state(gpu, orc, spins=False)
    assert gpu.info()["exchange_index"] == orc.exchange_index()
    assert_same_state(gpu, orc)
    gpu.close()


def test_split_launches_match_oracle_interval():
    """rewl_walk, rewl_exchange and rewl_flatness enqueued one by one (the benchmark's sequence) equal
    the oracle's moves, exchange round and flatness test."""
    gpu, orc = make_pair(**dict(CONVERGING, seed=11))
    gpu.init_walkers()
    orc.init_walkers()
    for _ in range(60):
        gpu.walk()
        gpu.exchange_async()
        gpu.flatness()
        orc.run_moves_only(CONVERGING["exchange_interval"])
        orc.exchange()
        orc.flatness()
    assert gpu.walkers()["stage"].max() > 0
    assert_same_state(gpu, orc)
    gpu.close()


def test_peak_temperature_matches_oracle():
    """The library's refinement of the C(T) maximum equals the oracle's on a measured curve and on the
    edge cases: maximum at either end of the grid, a tie (lowest index), a flat triple."""
    gpu, orc = make_pair(**CONVERGING)
    gpu.run_intervals(30)
    lng, cen = gpu.merge()
    T = np.linspace(1.5, 4.0, 2501)
    _, Cv, _ = rw.thermo(lng, cen, gpu.N, T)
    curves = [Cv, np.linspace(1.0, 0.0, 50), np.linspace(0.0, 1.0, 50), np.array([0.0, 1.0, 3.0, 1.0, 3.0, 0.5]),
              np.array([1.0, 2.0, 2.0, 2.0, 1.0]), np.array([5.0])]
    for c in curves:
        t = T[: c.size] if c.size > 1 else np.array([2.0])
        assert rw.peak_temperature(t, c) == oracle.peak(t, c)
    gpu.close()


def test_stage_log_reports_the_run():
    """run_to_convergence(log=...) writes one JSON line per stage: moves/s, accept rate, exchange
    acceptance per window pair, round trips, ln f, stage and flatness ratio per walker."""
    g = rw.REWL(kind=rw.BCC, mode=rw.PRODUCTION, group_size=1, **CONVERGING)
    buf = io.StringIO()
    stages = g.run_to_convergence(max_stages=40, log=buf)
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert len(lines) == len(stages) and stages[-1]["all_done"]
    last = lines[-1]
    assert last["stage_moves_per_s"] > 0 and 0 < last["accept_rate"] < 1
    assert len(last["exchange_acceptance"]) == g.h - 1 and all(0 <= a <= 1 for a in last["exchange_acceptance"])
    assert len(last["lnf"]) == g.n_slots and max(last["lnf"]) < CONVERGING["lnf_final"]
    for a, b in zip(lines, lines[1:]):      # every stage halves ln f of each walker still active at its start
        assert all(sb >= sa for sa, sb in zip(a["stage"], b["stage"]))
        assert all(sb > sa for sa, sb, f in zip(a["stage"], b["stage"], a["lnf"]) if f >= CONVERGING["lnf_final"])
    assert lines[-1]["stage"] == [int(v) for v in g.walkers()["stage"]]
    g.close()
