"""Window-partitioned REWL on one GPU: the run split over two or three handles by contiguous window ranges,
driven through the protocol layer (paper_1411_4212_gb300.partition).  Replica exchange crosses the
handles (Sec. 4.3, Eq. 5) by moving slot states, never configurations.  It must be the same run as one
handle holding every walker, slot for slot.  In trajectory mode it must also match the FP64 oracle bit
for bit: ln g, H, energies, bins, ln f, stages, counters, the configuration each slot holds, every
configuration's spins, exchange counts, round trips and the merged ln g."""
import numpy as np
import pytest

import oracle
import paper_1411_4212_gb300 as rw
from paper_1411_4212_gb300.partition import PartitionedRun, window_ranges
from rewl_pairs import TRAJ_KEYS_BITS, TRAJ_KEYS_EXACT, make_pair

pytestmark = pytest.mark.gpu

CFG = dict(L=4, J=(1.0, 0.5), e_min=-400.0, e_max=0.0, n_bins=120, n_windows=6, walkers_per_window=3,
           lnf_final=1e-3, exchange_interval=2000, seed=9)


def _same(a, b, what):
    for key in TRAJ_KEYS_EXACT:
        assert np.array_equal(a[key], b[key]), f"{what}: {key} differs at {np.nonzero(a[key] != b[key])}"
    for key in TRAJ_KEYS_BITS:
        bad = np.nonzero(a[key].view(np.int64) != b[key].view(np.int64))
        assert bad[0].size == 0, f"{what}: {key} differs at {bad}"


def _configs(parts, m):
    """Spins [R][3][N] and round trips by global configuration id."""
    sp, cnt, last = [], [], []
    for p in sorted(parts, key=lambda q: q.window_begin):
        sp.append(p.spins())
        c, l = p.round_trips()
        cnt.append(c)
        last.append(l)
    return np.concatenate(sp), np.concatenate(cnt), np.concatenate(last)


def _merged(run, ref):
    import torch
    g = run.gather()
    frag = torch.tensor(g["lng"].reshape(ref.h, ref.m, ref.W), dtype=torch.float64, device="cuda")
    out = torch.zeros(ref.B, dtype=torch.float64, device="cuda")
    starts = oracle.window_layout(ref.B, ref.h, 0.75)[1]
    rw.stitch_device(frag, starts, ref.B, out)
    return out.cpu().numpy()


@pytest.mark.parametrize("n_parts,group_size", [(2, 1), (3, 1), (2, 8)])
def test_trajectory_partition_matches_single_handle_and_oracle(n_parts, group_size):
    ranges = window_ranges(CFG["n_windows"], n_parts)
    parts = [rw.REWL(kind=rw.BCC, mode=rw.TRAJECTORY, group_size=group_size, partition=r, **CFG) for r in ranges]
    run = PartitionedRun(parts)
    run.init_walkers()
    single, orc = make_pair(group_size=group_size, **CFG)
    single.init_walkers()
    orc.init_walkers()
    for chunk in range(6):
        run.run_intervals(5)
        single.run_intervals(5)
        orc.run_intervals(5)
        g = run.gather()
        _same(g, single.walkers(), f"chunk {chunk}: partition vs single handle")
        _same(g, orc.walkers(), f"chunk {chunk}: partition vs oracle")
    assert run.cross_swaps > 0, "no exchange crossed the handles"
    sp, cnt, last = _configs(parts, CFG["walkers_per_window"])
    assert np.array_equal(sp.view(np.int64), orc.spins().view(np.int64))
    co, lo = orc.round_trips()
    assert np.array_equal(cnt, co) and np.array_equal(last, lo)
    att = sum(p.exchange_counts()[0] for p in parts)
    acc = sum(p.exchange_counts()[1] for p in parts)
    ao, bo = orc.exchange_counts()
    assert np.array_equal(att, ao) and np.array_equal(acc, bo)
    lo_merged, _ = orc.merge()
    assert np.array_equal(_merged(run, single).view(np.int64), lo_merged.view(np.int64))
    print(f"{n_parts} parts, G={group_size}: {run.cross_swaps} slot states moved between handles, "
          f"{int(acc.sum())} accepted exchanges of {int(att.sum())}, stages up to {g['stage'].max()}")
    for p in parts:
        p.close()
    single.close()


def test_production_partition_matches_single_handle():
    """Production mode (FP32 spins, fixed-point ln g): the partitioned run and the single handle reach
    the same state bit for bit on the pipelined walker, including the energy recomputation every 8
    intervals."""
    cfg = dict(CFG, n_windows=8, walkers_per_window=2, L=6, J=(1.0, 0.5, 0.2), e_min=-0.6 * 2 * 216 * 6.7,
               n_bins=432)
    ranges = window_ranges(cfg["n_windows"], 2)
    parts = [rw.REWL(kind=rw.BCC, mode=rw.PRODUCTION, group_size=1, partition=r, **cfg) for r in ranges]
    assert all(p.info()["pipelined"] == 1 for p in parts)
    run = PartitionedRun(parts)
    run.init_walkers()
    single = rw.REWL(kind=rw.BCC, mode=rw.PRODUCTION, group_size=1, **cfg)
    single.init_walkers()
    run.run_intervals(24)
    single.run_intervals(24)
    g, ws = run.gather(), single.walkers()
    for key, v in ws.items():
        assert np.array_equal(g[key], v), key
    sp, cnt, last = _configs(parts, cfg["walkers_per_window"])
    assert np.array_equal(sp, single.spins())
    assert run.cross_swaps > 0
    for p in parts:
        p.close()
    single.close()


def test_partition_rejects_whole_run_calls():
    p = rw.REWL(kind=rw.BCC, mode=rw.TRAJECTORY, group_size=1, partition=(0, 3), **CFG)
    for call in (lambda: p.run_intervals(1), p.run_stage, p.exchange, p.merge):
        with pytest.raises(rw.RewlError) as e:
            call()
        assert e.value.status == rw.ESTATE
    with pytest.raises(rw.RewlError):
        rw.Batch([p])
    p.init_walkers()
    buf = p.slot_export(0)
    with pytest.raises(rw.RewlError) as e:
        p.slot_import(1, buf)          # slot 0 is hosted here already
    assert e.value.status == rw.EINVAL
    p.close()
