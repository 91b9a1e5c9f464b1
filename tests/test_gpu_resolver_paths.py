"""The production walker resolves each batch of 32 trial moves by one of three paths: a warp scan, 8-move
branch-free blocks, or one move at a time.  They must take the same decisions.  Forcing one path for every
batch must leave the walk (Sec. 4.2, Eq. 4; trial move Sec. 4.4) in the same state, bit for bit, as the
per-batch choice.

The one-move-at-a-time path is the plain reading of the walk, and its statistics are checked against the
FP64 oracle in test_gpu_production.py.  This file pins the scan and the blocks to it, on the geometries
where the per-batch choice uses them."""
import math

import numpy as np
import pytest

import paper_1411_4212_gb300 as rw

pytestmark = pytest.mark.gpu

PATHS = {"auto": rw.RESOLVER_AUTO, "scan": rw.RESOLVER_SCAN, "blocks": rw.RESOLVER_BLOCKS,
         "sequential": rw.RESOLVER_SEQUENTIAL}

CASES = {
    # the benchmark geometry: [E_gs, 0] with bins of 22.5 J1; the high windows take the scan, the
    # low windows (mostly rejected exits) the blocks
    "bcc16_egs": (dict(L=16, J=(1.0, 0.5), n_bins=2000, n_windows=16, walkers_per_window=4, lnf_final=1e-8,
                       exchange_interval=10000), 4),
    # converging regime: bins about as wide as the temperature, most accepted moves change bin
    "bcc8_restricted": (dict(L=8, J=(1.0, 0.5, -0.05), e_min=-0.6 * 5.5 * 1024, e_max=0.0, n_bins=1024,
                             n_windows=16, walkers_per_window=2, lnf_final=1e-8, exchange_interval=4000), 12),
    # 128 spins: almost every move of a batch touches an earlier one (corrections everywhere)
    "bcc4_restricted": (dict(L=4, J=(1.0, 0.5), e_min=-400.0, e_max=0.0, n_bins=120, n_windows=4,
                             walkers_per_window=2, lnf_final=1e-4, exchange_interval=10000), 20),
    # the large four-shell lattice in global memory (the other kernel form)
    "bcc32_4shell": (dict(L=32, J=(1.0, 0.6, -0.05, -0.1), n_bins=8000, n_windows=64, walkers_per_window=8,
                          lnf_final=1e-8, exchange_interval=10000), 1),
}


def _run(cfg, intervals, resolver):
    g = rw.REWL(kind=rw.BCC, mode=rw.PRODUCTION, group_size=1, seed=7, resolver=resolver, **cfg)
    assert g.info()["pipelined"] == 1
    g.run_intervals(intervals)
    out = dict(walkers=g.walkers(), spins=g.spins(), counters=g.counters(), exchange=g.exchange_counts(),
               trips=g.round_trips(), lng=g.merge()[0])
    g.close()
    return out


def _same(a, b, what):
    for k, v in a["walkers"].items():
        assert np.array_equal(v, b["walkers"][k]), f"{what}: walkers[{k}] differs"
    assert np.array_equal(a["spins"], b["spins"]), f"{what}: spins differ"
    for k in ("moves", "accepts", "recomputes"):
        assert a["counters"][k] == b["counters"][k], f"{what}: {k} differs"
    for x, y in zip(a["exchange"] + a["trips"], b["exchange"] + b["trips"]):
        assert np.array_equal(x, y), f"{what}: exchange or round-trip counts differ"
    assert np.array_equal(a["lng"].view(np.int64), b["lng"].view(np.int64)), f"{what}: merged ln g differs"


@pytest.mark.parametrize("case", list(CASES))
def test_forced_paths_reach_the_same_state(case):
    cfg, intervals = CASES[case]
    res = {name: _run(cfg, intervals, r) for name, r in PATHS.items()}
    for name in ("scan", "blocks", "sequential"):
        c = res[name]["counters"]
        used = {"scan": c["batches_scan"], "blocks": c["batches_blocks"], "sequential": c["batches_sequential"]}
        assert used[name] > 0 and sum(used.values()) == used[name], (name, used)
        _same(res["auto"], res[name], f"{case}: auto vs forced {name}")
    c = res["auto"]["counters"]
    total = c["batches_scan"] + c["batches_blocks"] + c["batches_sequential"]
    assert total == math.ceil(cfg["exchange_interval"] / 32) * intervals * cfg["n_windows"] * cfg["walkers_per_window"]
    shares = {k: c["batches_" + k] / total for k in ("scan", "blocks", "sequential")}
    print(f"{case}: auto batches {total}, shares " + ", ".join(f"{k} {v:.3f}" for k, v in shares.items())
          + f"; accepts {c['accepts']}, corrections {c['recomputes']}")
    if case == "bcc16_egs":
        # the benchmark geometry is served by the scan and the blocks, not by the sequential path
        assert shares["scan"] >= 0.05 and shares["blocks"] >= 0.05, shares
    if case in ("bcc8_restricted", "bcc4_restricted"):
        # bins as wide as the temperature: most batches need the one-move-at-a-time path
        assert shares["sequential"] >= 0.5, shares

