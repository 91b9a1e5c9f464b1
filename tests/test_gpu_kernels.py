"""Single-kernel parity on the GPU: neighbour geometry, the FP64 exp, Philox against cuRAND, the merge
kernels on synthetic fragments, thermodynamics, energy recomputation, bandwidth probe."""
import ctypes as C
import math
import os

import numpy as np
import pytest

import oracle
import paper_1411_4212_gb300 as rw

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("L,J", [(4, (1.0,)), (4, (1.0, 0.5)), (5, (1.0, 0.5, 0.25)), (7, (1.0, 0.6, -0.05, -0.1)),
                                 (9, (1.0, 0.6, -0.05, -0.1))])
def test_bcc_neighbour_table_bit_exact(L, J):
    g = rw.REWL(kind=rw.BCC, L=L, J=J, n_bins=50, n_windows=1, walkers_per_window=1, mode=rw.TRAJECTORY)
    o = oracle.OracleREWL(kind=oracle.BCC, L=L, J=J, n_bins=50, n_windows=1, walkers_per_window=1)
    ng, jg = g.neighbours()
    no, jo = o.neighbours()
    assert np.array_equal(ng, no) and np.array_equal(jg, jo)
    assert g.e_min == o.e_min and g.dE == o.dE
    assert g.info()["initial_energy"] == o.initial_energy()
    g.close()


def test_chain_neighbour_table():
    g = rw.REWL(kind=rw.CHAIN, L=7, J=(1.5,), n_bins=20, n_windows=1, walkers_per_window=1)
    o = oracle.OracleREWL(kind=oracle.CHAIN, L=7, J=(1.5,), n_bins=20, n_windows=1, walkers_per_window=1)
    ng, jg = g.neighbours()
    no, jo = o.neighbours()
    assert np.array_equal(ng, no) and np.array_equal(jg, jo)
    assert g.e_min == o.e_min and g.e_max == o.e_max
    g.close()


def test_device_exp_bit_identical_to_oracle():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(-708, 0, 200000), rng.uniform(-1, 0, 50000), -np.logspace(-15, 2.85, 3000),
                        [0.0, -708.0, -708.5, -750.0, -1e-310]])
    y = rw.device_exp(x)
    yo = np.array([oracle.exp(float(v)) for v in x])
    assert np.array_equal(y.view(np.int64), yo.view(np.int64))


def test_philox_matches_curand():
    lib = C.CDLL(os.path.join(HERE, "cuda", "libcurand_probe.so"))
    rng = np.random.default_rng(3)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [1, 0, 0, 0], [0xFFFFFFFF] * 4, [5, 6, 2, 7]]
    key[:4] = [[0, 0], [0, 0], [0xFFFFFFFF] * 2, [9, 1]]
    out = np.zeros((n, 4), dtype=np.uint32)
    rc = lib.curand_philox_probe(ctr.ctypes.data_as(C.c_void_p), key.ctypes.data_as(C.c_void_p), n,
                                 out.ctypes.data_as(C.c_void_p))
    assert rc == 0
    ours = np.array([oracle.philox4x32_10(c, k) for c, k in zip(ctr, key)])
    assert np.array_equal(ours, out)


def _stitch_cases():
    rng = np.random.default_rng(4)
    cases = []
    for B, h, m in [(200, 4, 2), (2000, 16, 4), (8000, 64, 8), (57, 3, 1), (40, 1, 3)]:
        W, st = oracle.window_layout(B, h, 0.75 if h > 1 else 0.0)
        base = np.cumsum(rng.normal(0.5, 0.2, B))
        frag = np.zeros((h, m, W))
        for k in range(h):
            for a in range(m):
                frag[k, a] = base[st[k]:st[k] + W] + rng.uniform(-100, 100) + rng.normal(0, 0.05, W)
        cases.append((frag, st, B))
    return cases


@pytest.mark.parametrize("case", range(5))
def test_stitch_kernel_bit_exact(case):
    import torch
    frag, st, B = _stitch_cases()[case]
    ref, bref, rc = oracle.merge_fragments(frag, st, B)
    tf = torch.tensor(frag, dtype=torch.float64, device="cuda")
    out = torch.zeros(B, dtype=torch.float64, device="cuda")
    bst = torch.zeros(max(len(st) - 1, 1), dtype=torch.int32, device="cuda")
    rw.stitch_device(tf, st, B, out, bst)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    assert np.array_equal(bst.cpu().numpy()[: len(st) - 1], bref)


def test_thermo_matches_oracle():
    B = 2000
    e = np.linspace(-45000, 0, B)
    lng = 8192 * np.log(4 * np.pi) * 0.5 * (1 - ((e + 20000) / 25000) ** 2) + 0.01 * np.sin(e / 100)
    T = np.linspace(0.2, 3.0, 2801)
    Ug, Cg, Zg = rw.thermo(lng, e, 8192, T)
    Uo, Co, Zo = oracle.thermo(lng, e, 8192, T)
    assert np.allclose(Ug, Uo, rtol=1e-10, atol=1e-8)
    assert np.allclose(Cg, Co, rtol=1e-8, atol=1e-12)
    assert np.allclose(Zg, Zo, rtol=1e-12)
    assert rw.peak_temperature(T, Cg) == pytest.approx(oracle.peak(T, Co), rel=1e-9)


def test_replica_energies_match_running_energy():
    g = rw.REWL(kind=rw.BCC, L=6, J=(1.0, 0.5, 0.2), n_bins=200, n_windows=4, walkers_per_window=2,
                mode=rw.TRAJECTORY, exchange_interval=2000)
    g.run_intervals(3)
    w = g.walkers()
    Er = g.replica_energies()
    assert np.allclose(Er[w["replica"]], w["E"], rtol=0, atol=1e-9)
    g.close()
    p = rw.REWL(kind=rw.BCC, L=6, J=(1.0, 0.5, 0.2), n_bins=200, n_windows=4, walkers_per_window=2,
                mode=rw.PRODUCTION, exchange_interval=2000)
    p.run_intervals(3)
    w = p.walkers()
    Er = p.replica_energies()
    # FP32 spins: the running energy tracks the configuration to ~1e-4 absolute per 1e4 moves
    assert np.allclose(Er[w["replica"]], w["E"], rtol=0, atol=5e-3)
    p.close()


def test_smem_bandwidth_probe_is_sane():
    bw, ms = rw.measure_smem_bandwidth()
    assert 5e12 < bw < 1e14 and ms > 0
