"""Checkpoint and resume (rewl_save_state / rewl_load_state).  A run stopped at an interval boundary,
saved, and resumed in a fresh handle must continue exactly as the uninterrupted run would have:
- in trajectory mode, bit for bit, and against the FP64 oracle;
- in production mode, bit for bit against the uninterrupted production run;
- for a partitioned run, one checkpoint per handle.
A corrupted buffer or the checkpoint of another run is rejected with REWL_EINVAL and leaves the
handle as it was."""
import numpy as np
import pytest

import paper_1411_4212_gb300 as rw
from paper_1411_4212_gb300.partition import PartitionedRun, window_ranges
from rewl_pairs import assert_same_state, make_pair

pytestmark = pytest.mark.gpu

TRAJ = dict(L=4, J=(1.0, 0.5), e_min=-400.0, e_max=0.0, n_bins=120, n_windows=4, walkers_per_window=2,
            lnf_final=1e-3, exchange_interval=5000, seed=3)
PROD = dict(L=16, J=(1.0, 0.5), n_bins=2000, n_windows=16, walkers_per_window=4, lnf_final=1e-8,
            exchange_interval=10000, seed=4)


def _snapshot(g):
    out = dict(g.walkers())
    out["spins"] = g.spins()
    out["ex"] = np.concatenate(g.exchange_counts())
    out["trips"] = np.concatenate([a.astype(np.int64) for a in g.round_trips()])
    out["counters"] = np.array(list(g.counters().values()))
    info = g.info()
    out["info"] = np.array([info["intervals_done"], info["exchange_index"]])
    out["merged"] = g.merge()[0]
    return out


def _equal(a, b):
    for k, v in a.items():
        w = b[k]
        same = np.array_equal(v.view(np.int64), w.view(np.int64)) if v.dtype == np.float64 else np.array_equal(v, w)
        assert same, f"{k} differs after the resume"


def test_trajectory_resume_is_bit_identical(tmp_path):
    path = tmp_path / "traj.ckpt"
    a, orc = make_pair(**TRAJ)
    a.init_walkers()
    orc.init_walkers()
    a.run_intervals(12)
    a.save_state(path)
    a.run_intervals(20)
    ref = _snapshot(a)
    b = rw.REWL(kind=rw.BCC, mode=rw.TRAJECTORY, group_size=1, **TRAJ)
    b.load_state(str(path))
    b.run_intervals(20)
    _equal(ref, _snapshot(b))
    orc.run_intervals(32)
    assert_same_state(b, orc)
    a.close()
    b.close()


def test_production_resume_is_bit_identical():
    a = rw.REWL(kind=rw.BCC, mode=rw.PRODUCTION, **PROD)
    a.run_intervals(5)
    ck = a.save_state()
    a.run_intervals(11)      # crosses an energy recomputation (every 8 intervals)
    ref = _snapshot(a)
    b = rw.REWL(kind=rw.BCC, mode=rw.PRODUCTION, **PROD)
    b.load_state(ck)
    b.run_intervals(11)
    _equal(ref, _snapshot(b))
    a.close()
    b.close()


def test_partitioned_run_resumes_from_one_checkpoint_per_handle():
    cfg = dict(TRAJ, n_windows=6, walkers_per_window=3, exchange_interval=2000, seed=9)
    ranges = window_ranges(6, 2)
    mk = lambda: [rw.REWL(kind=rw.BCC, mode=rw.TRAJECTORY, group_size=1, partition=r, **cfg) for r in ranges]
    run = PartitionedRun(mk())
    run.init_walkers()
    run.run_intervals(10)
    cks = [p.save_state() for p in run.parts]
    run.run_intervals(15)
    ref = run.gather()
    run2 = PartitionedRun(mk())
    for p, ck in zip(run2.parts, cks):
        p.load_state(ck)
    run2.run_intervals(15)
    got = run2.gather()
    for k, v in ref.items():
        assert np.array_equal(v.view(np.int64) if v.dtype == np.float64 else v,
                              got[k].view(np.int64) if v.dtype == np.float64 else got[k]), k
    assert run.cross_swaps > 0


def test_corrupted_or_foreign_checkpoint_is_rejected():
    a = rw.REWL(kind=rw.BCC, mode=rw.TRAJECTORY, group_size=1, **TRAJ)
    a.run_intervals(6)
    ck = a.save_state()
    b = rw.REWL(kind=rw.BCC, mode=rw.TRAJECTORY, group_size=1, **TRAJ)
    b.run_intervals(2)
    before = _snapshot(b)
    bad = ck.copy()
    bad[bad.size // 2] ^= 0x10
    for buf, what in ((bad, b"checksum"), (ck[:-8], b"size")):
        with pytest.raises(rw.RewlError) as e:
            b.load_state(buf)
        assert e.value.status == rw.EINVAL and what in rw.load_library().rewl_last_error(b._h)
    other = rw.REWL(kind=rw.BCC, mode=rw.TRAJECTORY, group_size=1, **dict(TRAJ, seed=4))
    with pytest.raises(rw.RewlError) as e:
        other.load_state(ck)
    assert e.value.status == rw.EINVAL and b"other arguments" in rw.load_library().rewl_last_error(other._h)
    _equal(before, _snapshot(b))
    b.load_state(ck)
    _equal(_snapshot(a), _snapshot(b))
    for g in (a, b, other):
        g.close()
