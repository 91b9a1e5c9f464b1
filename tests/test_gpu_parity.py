"""Trajectory-mode parity: the CUDA walker, exchange, flatness and merge kernels against the FP64
oracle, bit for bit (histograms, accept counts, ln g, energies, spins, exchange counters,
configuration permutation, merged ln g).  Sizes span several batches and a ragged tail, every group
size (summation order), every coupling shell count, table lattices, the shared-memory and the
global-memory lattice paths, and the degenerate single-window / single-walker layouts."""
import numpy as np
import pytest

from rewl_pairs import assert_same_state, make_pair

pytestmark = pytest.mark.gpu

CFG1 = dict(L=4, J=(1.0, 0.5), n_bins=200, n_windows=4, walkers_per_window=2, overlap=0.75, flatness=0.8,
            lnf_final=1e-3, seed=1)


def run_both(gpu, orc, intervals):
    gpu.init_walkers()
    orc.init_walkers()
    assert_same_state(gpu, orc)
    if intervals:
        gpu.run_intervals(intervals)
        orc.run_intervals(intervals)
    assert_same_state(gpu, orc)
    lg, cg = gpu.merge()
    lo, co = orc.merge()
    assert np.array_equal(lg.view(np.int64), lo.view(np.int64)), "merged ln g differs"
    assert np.array_equal(cg, co)


@pytest.mark.parametrize("G", [1, 2, 4, 8, 16, 32])
def test_cfg1_every_group_size(G):
    gpu, orc = make_pair(group_size=G, exchange_interval=1000, **CFG1)
    assert gpu.info()["pipelined"] == (1 if G == 1 else 0)
    run_both(gpu, orc, 6)
    gpu.close()


def test_cfg1_long_with_flatness_events():
    """Enough moves that walkers in the upper windows pass several ln f reductions."""
    gpu, orc = make_pair(group_size=8, exchange_interval=10000, **CFG1)
    run_both(gpu, orc, 40)
    w = gpu.walkers()
    assert w["stage"].max() >= 2, "expected ln f reductions within the run"
    a, b = gpu.exchange_counts()
    assert np.all(b > 0)
    gpu.close()


def test_three_shells_ragged():
    gpu, orc = make_pair(group_size=1, L=6, J=(1.0, 0.4, -0.1), n_bins=150, n_windows=5, walkers_per_window=3,
                         overlap=0.7, flatness=0.8, lnf_final=1e-3, seed=7, exchange_interval=777)
    run_both(gpu, orc, 4)
    gpu.close()


def test_four_shells():
    gpu, orc = make_pair(group_size=2, L=5, J=(1.0, 0.6, -0.05, -0.1), n_bins=120, n_windows=3,
                         walkers_per_window=2, overlap=0.75, flatness=0.8, lnf_final=1e-3, seed=3,
                         exchange_interval=500)
    run_both(gpu, orc, 4)
    gpu.close()


def test_single_window_single_walker_every_move_exchange():
    gpu, orc = make_pair(group_size=4, L=3, J=(1.0,), n_bins=40, n_windows=1, walkers_per_window=1,
                         overlap=0.0, flatness=0.8, lnf_final=1e-3, seed=11, exchange_interval=1)
    run_both(gpu, orc, 50)
    gpu.close()


def test_chain_table_lattice():
    gpu, orc = make_pair(kind="chain", group_size=1, L=10, J=(1.0,), n_bins=40, n_windows=2,
                         walkers_per_window=2, overlap=0.75, flatness=0.8, lnf_final=1e-4, seed=5,
                         exchange_interval=2000)
    run_both(gpu, orc, 10)
    gpu.close()


def test_explicit_table_lattice():
    """Ring of 24 spins with nearest and next-nearest couplings given as a table."""
    n = 24
    nbr = np.array([[(i - 1) % n for i in range(n)], [(i + 1) % n for i in range(n)],
                    [(i - 2) % n for i in range(n)], [(i + 2) % n for i in range(n)]], dtype=np.int32)
    Jt = np.array([[1.0] * n, [1.0] * n, [-0.3] * n, [-0.3] * n])
    for G in (1, 2):
        gpu, orc = make_pair(kind="table", group_size=G, nbr=nbr, Jt=Jt, e_min=-20.0, e_max=20.0, n_bins=60,
                             n_windows=3, walkers_per_window=2, overlap=0.75, flatness=0.8, lnf_final=1e-4,
                             seed=9, exchange_interval=1500)
        run_both(gpu, orc, 5)
        gpu.close()


def test_cfg2_size_shared_lattice():
    """bcc L=16 (8192 spins), 16 windows x 4 walkers, 2000 bins: the production workload's geometry."""
    gpu, orc = make_pair(group_size=1, L=16, J=(1.0, 0.5), n_bins=2000, n_windows=16, walkers_per_window=4,
                         overlap=0.75, flatness=0.8, lnf_final=1e-8, seed=1, exchange_interval=3000)
    assert gpu.info()["lattice_in_shared"] == 1 and gpu.info()["pipelined"] == 1
    run_both(gpu, orc, 2)
    gpu.close()


def test_global_memory_lattice_path():
    """bcc L=20 in FP64 (384 KB per lattice) does not fit in shared memory: global-memory path."""
    gpu, orc = make_pair(group_size=1, L=20, J=(1.0, 0.5), n_bins=400, n_windows=3, walkers_per_window=1,
                         overlap=0.75, flatness=0.8, lnf_final=1e-8, seed=2, exchange_interval=2000)
    assert gpu.info()["lattice_in_shared"] == 0 and gpu.info()["pipelined"] == 1
    run_both(gpu, orc, 2)
    gpu.close()


def test_global_memory_lattice_autotune_moves_are_ordinary_moves():
    """The conflict-table autotuner times ten walker launches (8192 .. 512 entries, twice; up to 32
    sites per entry): each is ordinary moves, so the oracle walking the same count agrees bit for bit,
    and so do the intervals after it on the chosen table."""
    gpu, orc = make_pair(group_size=1, L=20, J=(1.0, 0.5), n_bins=400, n_windows=3, walkers_per_window=1,
                         overlap=0.75, flatness=0.8, lnf_final=1e-8, seed=3, exchange_interval=1500)
    assert gpu.info()["conflict_entries"] == 2048
    gpu.init_walkers()
    orc.init_walkers()
    t = gpu.autotune(trial_moves=300)
    assert t["conflict_entries"] in (512, 1024, 2048, 4096, 8192) and t["trial_ms"] > 0
    assert gpu.info()["conflict_entries"] == t["conflict_entries"]
    orc.run_moves_only(10 * 300)
    assert_same_state(gpu, orc)
    gpu.run_intervals(2)
    orc.run_intervals(2)
    assert_same_state(gpu, orc)
    gpu.close()


def test_shared_lattice_autotune_moves_are_ordinary_moves():
    """With the lattice in shared memory the autotuner times the tables that fit beside it (1024 and 512
    entries at bcc L = 8, twice each): ordinary moves again, bit for bit with the oracle."""
    gpu, orc = make_pair(group_size=1, L=8, J=(1.0, 0.5), n_bins=600, n_windows=3, walkers_per_window=2,
                         overlap=0.75, flatness=0.8, lnf_final=1e-8, seed=5, exchange_interval=1500)
    assert gpu.info()["lattice_in_shared"] == 1 and gpu.info()["conflict_entries"] == 1024
    gpu.init_walkers()
    orc.init_walkers()
    t = gpu.autotune(trial_moves=300)
    assert t["conflict_entries"] in (512, 1024) and t["trial_ms"] > 0
    orc.run_moves_only(4 * 300)
    assert_same_state(gpu, orc)
    gpu.run_intervals(2)
    orc.run_intervals(2)
    assert_same_state(gpu, orc)
    gpu.close()


def test_autotune_leaves_single_table_walkers_alone():
    """bcc L = 4 (128 sites) has one table size to offer: no trial, no move."""
    gpu, _ = make_pair(group_size=1, exchange_interval=1000, **CFG1)
    gpu.init_walkers()
    steps = gpu.walkers()["steps"].copy()
    entries = gpu.info()["conflict_entries"]
    t = gpu.autotune(trial_moves=300)
    assert t == {"conflict_entries": entries, "trial_ms": 0.0}
    assert np.array_equal(gpu.walkers()["steps"], steps)
    gpu.close()


def test_frozen_walkers_and_set_initial_lng():
    """Warm start: set ln g and ln f below ln f_final for every walker (frozen), walk, compare."""
    gpu, orc = make_pair(group_size=8, exchange_interval=1000, **CFG1)
    B = gpu.B
    lng0 = np.linspace(0.0, 30.0, B) + np.sin(np.arange(B) / 7.0)
    gpu.set_initial_lng(lng0, 1e-4)
    orc.set_lng(lng0, 1e-4)
    run_both(gpu, orc, 3)
    w = gpu.walkers()
    assert np.all(w["H"] == 0)
    gpu.close()


def test_pipelined_walker_tiny_lattice_heavy_conflicts():
    """bcc L=3 (54 spins): nearly every move of a 64-move window conflicts; still bit-exact."""
    gpu, orc = make_pair(group_size=1, L=3, J=(1.0,), n_bins=60, n_windows=2, walkers_per_window=2,
                         overlap=0.75, flatness=0.8, lnf_final=1e-3, seed=21, exchange_interval=4000)
    assert gpu.info()["pipelined"] == 1
    run_both(gpu, orc, 3)
    gpu.close()


def test_pipelined_walker_partial_batches():
    """Exchange intervals of 1, 31, 33 and 65 moves (partial final batches, one- and two-batch runs)."""
    for ex in (1, 31, 33, 65):
        gpu, orc = make_pair(group_size=1, L=5, J=(1.0, 0.5, 0.25), n_bins=100, n_windows=3,
                             walkers_per_window=2, overlap=0.75, flatness=0.8, lnf_final=1e-3, seed=ex,
                             exchange_interval=ex)
        run_both(gpu, orc, 4)
        gpu.close()


def test_round_trips_on_a_converging_range():
    """Restricted range [-400, 0] (bins narrower than the temperature): configurations cross all
    four windows many times; round trips, exchanges and the walk agree bit for bit."""
    gpu, orc = make_pair(group_size=1, L=4, J=(1.0, 0.5), e_min=-400.0, e_max=0.0, n_bins=60, n_windows=4,
                         walkers_per_window=2, overlap=0.75, flatness=0.8, lnf_final=1e-6, seed=5,
                         exchange_interval=200)
    run_both(gpu, orc, 250)
    c, _ = gpu.round_trips()
    assert c.sum() > 5
    gpu.close()


@pytest.mark.parametrize("m,intervals,stages", [(3, 900, 2), (2, 40, 1)])
def test_window_synchronous_iteration(m, intervals, stages):
    """The walkers of a window move on together (ln g averaged bin by bin, then ln f halved): bit for
    bit against the oracle on a converging range (m = 3) and on the cfg1 geometry (m = 2)."""
    if m == 3:
        cfg = dict(L=4, J=(1.0, 0.5), e_min=-400.0, e_max=0.0, n_bins=60, n_windows=3, walkers_per_window=3,
                   overlap=0.75, flatness=0.8, lnf_final=1e-3, seed=9, exchange_interval=300)
    else:
        cfg = dict(CFG1, exchange_interval=10000)
    gpu, orc = make_pair(group_size=1, iteration=1, **cfg)
    run_both(gpu, orc, intervals)
    st = gpu.walkers()["stage"].reshape(-1, m)
    assert st.max() >= stages and np.all(st == st[:, :1])
    gpu.close()
