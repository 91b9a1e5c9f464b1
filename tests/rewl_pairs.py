"""Matched GPU / oracle simulations for the parity tests (same configuration on both sides)."""
import numpy as np

import oracle
import paper_1411_4212_gb300 as rw

TRAJ_KEYS_EXACT = ("H", "bin", "replica", "accepts", "steps", "init_moves", "stage")
TRAJ_KEYS_BITS = ("lng", "E", "lnf")


def make_pair(kind="bcc", group_size=1, **cfg):
    k_rw = {"bcc": rw.BCC, "chain": rw.CHAIN, "table": rw.TABLE}[kind]
    k_or = {"bcc": oracle.BCC, "chain": oracle.CHAIN, "table": oracle.TABLE}[kind]
    gcfg = dict(cfg)
    ocfg = dict(cfg)
    if "lnf_initial" in gcfg and gcfg["lnf_initial"] == 1.0:
        gcfg["lnf_initial"] = 0.0
    if "init_max_moves" not in ocfg:
        ocfg["init_max_moves"] = 1 << 40
    gpu = rw.REWL(kind=k_rw, mode=rw.TRAJECTORY, group_size=group_size, **gcfg)
    orc = oracle.OracleREWL(kind=k_or, group_size=group_size, **ocfg)
    return gpu, orc


def assert_same_state(gpu, orc, spins=True):
    wg, wo = gpu.walkers(), orc.walkers()
    for key in TRAJ_KEYS_EXACT:
        assert np.array_equal(wg[key], wo[key]), f"{key} differs: {np.nonzero(wg[key] != wo[key])}"
    for key in TRAJ_KEYS_BITS:
        bad = np.nonzero(wg[key].view(np.int64) != wo[key].view(np.int64))
        assert bad[0].size == 0, f"{key} differs at {bad}"
    if spins:
        sg, so = gpu.spins(), orc.spins()
        assert np.array_equal(sg.view(np.int64), so.view(np.int64)), "spins differ"
    ag, bg = gpu.exchange_counts()
    ao, bo = orc.exchange_counts()
    assert np.array_equal(ag, ao) and np.array_equal(bg, bo), "exchange counters differ"
    cg, lg = gpu.round_trips()
    co, lo = orc.round_trips()
    assert np.array_equal(cg, co) and np.array_equal(lg, lo), "round trips differ"
