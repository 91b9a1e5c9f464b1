"""Batched jobs: many REWL handles in one persistent walker launch replayed from a CUDA graph.

Trajectory mode: every job of a batch must match its own FP64 oracle bit for bit (the batch only
changes which CTA walks which slot, and in what order), for every tuning: one to three walker pairs
per CTA, lattices in shared memory, in global memory, or mixed.  Production mode: the batch must
reproduce each handle run alone bit for bit as long as no energy recomputation intervenes (the
recomputation's FP64 sum runs over a different number of threads), and run_to_convergence must
retire every job."""
import numpy as np
import pytest

import oracle
import paper_1411_4212_gb300 as rw
from rewl_pairs import assert_same_state

pytestmark = pytest.mark.gpu

# uneven lattices, window counts, walkers and seeds; two coupling shells throughout
JOBS = [
    dict(L=4, J=(1.0, 0.5), n_bins=200, n_windows=4, walkers_per_window=2, seed=1),
    dict(L=5, J=(1.0, 0.4), n_bins=150, n_windows=3, walkers_per_window=3, seed=2),
    dict(L=6, J=(1.0, 0.3), n_bins=240, n_windows=5, walkers_per_window=2, seed=3),
    dict(L=3, J=(1.0, 0.6), n_bins=80, n_windows=2, walkers_per_window=1, seed=4),
]
COMMON = dict(overlap=0.75, flatness=0.8, lnf_final=1e-3, exchange_interval=700, group_size=1)


def _traj_jobs(specs, recompute_every=0):
    # the energy recomputation only measures drift in trajectory mode: the oracle needs no cadence
    gpus = [rw.REWL(kind=rw.BCC, mode=rw.TRAJECTORY, recompute_every=recompute_every, **s, **COMMON)
            for s in specs]
    orcs = [oracle.OracleREWL(kind=oracle.BCC, init_max_moves=1 << 40, **s, **COMMON) for s in specs]
    for g in gpus:
        assert g.info()["pipelined"] == 1
    return gpus, orcs


# (pairs per CTA, largest lattice kept in shared memory, conflict-table cap for global lattices):
# a 256-entry cap makes sites of the L=5 and L=6 lattices share entries
@pytest.mark.parametrize("workers,smem_max_n,own_cap", [(1, 0, 0), (1, 0, 256), (2, 300, 0), (3, 1 << 30, 0)])
def test_batch_trajectory_matches_oracle(workers, smem_max_n, own_cap):
    gpus, orcs = _traj_jobs(JOBS)
    for o in orcs:
        o.init_walkers()
    with rw.Batch(gpus) as b:
        b.set_tuning(workers, smem_max_n, own_cap)
        info = b.info()
        assert info["workers_per_block"] == workers and info["n_items"] == sum(g.n_slots for g in gpus)
        assert info["owner_entries_max"] == (own_cap or 8192)
        n_smem = sum(1 for g in gpus if g.N <= smem_max_n)
        assert info["n_smem_lattice_jobs"] == n_smem
        b.run_intervals(5)
        assert b.info()["graphs_built"] >= 1
    for o in orcs:
        o.run_intervals(5)
    for g, o in zip(gpus, orcs):
        assert_same_state(g, o)
        lg, _ = g.merge()
        lo, _ = o.merge()
        assert np.array_equal(lg.view(np.int64), lo.view(np.int64))
        g.close()


def test_batch_trajectory_graph_cadence_with_recompute_every():
    """recompute_every = 3: the R-interval graph and the single-interval graphs interleave."""
    gpus, orcs = _traj_jobs(JOBS[:2], recompute_every=3)
    for o in orcs:
        o.init_walkers()
    with rw.Batch(gpus) as b:
        for n in (1, 4, 2, 3):
            b.run_intervals(n)
        assert b.info()["intervals_done"] == 10
    for o in orcs:
        o.run_intervals(10)
    for g, o in zip(gpus, orcs):
        assert_same_state(g, o)
        g.close()


def test_batch_production_equals_single_runs_before_recompute():
    specs = [dict(s) for s in JOBS[:3]]
    mk = lambda s: rw.REWL(kind=rw.BCC, mode=rw.PRODUCTION, recompute_every=1000, **s, **COMMON)
    singles = [mk(s) for s in specs]
    batched = [mk(s) for s in specs]
    for g in singles:
        g.init_walkers()
        g.run_intervals(4, stats=False)
    with rw.Batch(batched) as b:
        b.set_tuning(2, 300)
        b.run_intervals(4)
    for g1, g2 in zip(singles, batched):
        w1, w2 = g1.walkers(), g2.walkers()
        for k in ("H", "bin", "replica", "accepts", "steps", "stage"):
            assert np.array_equal(w1[k], w2[k]), k
        for k in ("lng", "E", "lnf"):
            assert np.array_equal(w1[k].view(np.int64), w2[k].view(np.int64)), k
        assert np.array_equal(g1.spins().view(np.int64), g2.spins().view(np.int64))
        g1.close()
        g2.close()


def test_batch_autotune_and_convergence():
    """Restricted energy range (bins narrower than the temperature there): converges in seconds."""
    jobs = [rw.REWL(kind=rw.BCC, mode=rw.PRODUCTION, L=4, J=(1.0, j2), e_min=-400.0, e_max=0.0, n_bins=120,
                    n_windows=3, walkers_per_window=2, overlap=0.75, flatness=0.8, lnf_final=1e-4, seed=s,
                    exchange_interval=2000, group_size=1)
            for s, j2 in enumerate((0.3, 0.45, 0.6), start=11)]
    with rw.Batch(jobs) as b:
        steps0 = [j.walkers()["steps"].copy() for j in jobs]
        t = b.autotune(trial_moves=500)
        assert 1 <= t["workers_per_block"] <= 3 and t["trial_ms"] > 0
        info = b.info()
        assert info["workers_per_block"] == t["workers_per_block"]
        # the timed trials are ordinary moves: every walker advanced by the same count
        adv = [j.walkers()["steps"] - s0 for j, s0 in zip(jobs, steps0)]
        assert len({int(a.min()) for a in adv} | {int(a.max()) for a in adv}) == 1
        converged, n_done = b.run_to_convergence(max_intervals=20000, check_every=16)
        assert converged and n_done == len(jobs)
        assert b.info()["n_active_jobs"] == 0
    for j in jobs:
        w = j.walkers()
        assert np.all(w["lnf"] < 1e-4)
        lng, _ = j.merge()
        assert np.all(np.isfinite(lng))
        j.close()


def test_batch_rejects_mixed_jobs():
    a = rw.REWL(kind=rw.BCC, mode=rw.TRAJECTORY, **JOBS[0], **COMMON)
    b = rw.REWL(kind=rw.BCC, mode=rw.PRODUCTION, **JOBS[1], **COMMON)
    c = rw.REWL(kind=rw.BCC, mode=rw.TRAJECTORY, L=4, J=(1.0, 0.5, 0.1), n_bins=100, n_windows=2,
                walkers_per_window=1, seed=5, **COMMON)
    for pair in ((a, b), (a, c), (a, a)):
        with pytest.raises(rw.RewlError) as e:
            rw.Batch(list(pair))
        assert e.value.status == rw.EINVAL
    with rw.Batch([a]) as bt:
        for bad in ((4, 0, 0), (2, 0, 300), (2, 0, 128), (2, 0, 16384)):
            with pytest.raises(rw.RewlError):
                bt.set_tuning(*bad)
        info = bt.info()   # the previous tuning stays
        assert info["workers_per_block"] == 2 and info["owner_entries_max"] == 8192
    for h in (a, b, c):
        h.close()


def test_batched_convergence_of_mixed_lattices_gives_every_job_its_result():
    """16 jobs of four lattice sizes (bcc L = 4, 5, 6, 8) with random three-shell couplings, each on its
    restricted range [0.6 E_gs, 0] with one bin per spin, converged to ln f = 1e-4 in one batch (the
    batch autotuned first; finished jobs leave the work list).  Every job must reach its ln f target
    (Sec. 4.2), and its merged ln g (Sec. 4.3) must be finite, mean zero and increasing with E: the
    range lies below the energy of infinite temperature, so 1/T = d ln g/dE > 0.  Its specific heat
    (Sec. 4.1, Eq. 3) must peak inside the temperature grid."""
    from paper_1411_4212_gb300 import warmstart, workloads
    sizes = (4, 5, 6, 8)
    jobs = [warmstart.restricted_job(L, workloads.random_couplings(300 + 4 * i + k), seed=40 + 4 * i + k,
                                     lnf_final=1e-4)
            for i, L in enumerate(sizes) for k in range(4)]
    with rw.Batch(jobs) as b:
        b.autotune(trial_moves=500)
        converged, n_done = b.run_to_convergence(max_intervals=100000, check_every=8)
        assert converged and n_done == len(jobs)
    T = np.linspace(0.8, 5.0, 2101)
    peaks = []
    for j in jobs:
        assert np.all(j.walkers()["lnf"] < 1e-4)
        lng, cen = j.merge()
        assert np.all(np.isfinite(lng)) and abs(lng.mean()) < 1e-9 * max(1.0, np.abs(lng).max())
        k = max(4, j.W // 8)                       # slope over k bins: the bin noise averages out
        slope = (lng[k:] - lng[:-k]) / (cen[k:] - cen[:-k])
        assert np.mean(slope > 0) > 0.98, (j.N, np.mean(slope > 0))
        _, Cv, _ = rw.thermo(lng, cen, j.N, T)
        tp = rw.peak_temperature(T, Cv)
        assert T[0] < tp < T[-1], tp
        peaks.append(tp)
        j.close()
    print("T_peak per job:", np.round(peaks, 3))


def test_production_walk_does_not_depend_on_the_conflict_table_size():
    """The conflict (owner) table maps a site to entry site mod size, so a smaller table flags more
    pairs of moves that share an entry without sharing a neighbourhood; the resolver drops those
    aliases before they become events.  The walk must not depend on the table size: a four-shell
    bcc L = 24 lattice (in global memory) run alone (2048 entries) and as a one-job batch with 256,
    1024 and 8192 entries reaches the same state bit for bit."""
    spec = dict(L=24, J=(1.0, 0.6, -0.05, -0.1), n_bins=2000, n_windows=8, walkers_per_window=2)
    states, recomputes = [], []
    for cap in (None, 256, 1024, 8192):
        g = rw.REWL(kind=rw.BCC, mode=rw.PRODUCTION, lnf_final=1e-8, seed=5, exchange_interval=5000,
                    recompute_every=1000, group_size=1, **spec)
        assert g.info()["pipelined"] == 1 and g.info()["lattice_in_shared"] == 0
        if cap is None:
            g.init_walkers()
            g.run_intervals(3, stats=False)
        else:
            with rw.Batch([g]) as b:
                b.set_tuning(1, 0, cap)
                assert b.info()["n_smem_lattice_jobs"] == 0
                b.run_intervals(3)
        w = g.walkers()
        st = {k: np.array(w[k]) for k in ("H", "bin", "replica", "accepts", "steps", "stage")}
        for k in ("lng", "E", "lnf"):
            st[k] = np.array(w[k]).view(np.int64)
        st["spins"] = g.spins().view(np.int64)
        states.append(st)
        recomputes.append(g.counters()["recomputes"])
        g.close()
    print("corrections (real conflicts only):", recomputes)
    assert len(set(recomputes)) == 1     # aliases are dropped, so only real conflicts are corrected
    for st in states[1:]:
        for k in st:
            assert np.array_equal(states[0][k], st[k]), k
