"""The window-partition protocol on CPU: two or three gloo ranks on 127.0.0.1 drive the round protocol of
paper_1411_4212_gb300.partition (bins by max all-reduce, ln g lookups by sum all-reduce, the decision,
slot states moved by all-reduce, the second look) across contiguous window ranges of a REWL run.  Each rank holds
a stand-in part that keeps its slot states and configurations in plain arrays.  The arithmetic of the
decision is Eq. 5 with the oracle's Philox and exp, as the library's exchange kernel does it.

After several rounds, every slot must hold the configuration that the FP64 oracle's own exchange rounds
(one process, every slot) give it, and the exchange counts must agree.  The library's GPU side of the
same protocol is tested in test_gpu_partition.py."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CFG = dict(L=4, J=(1.0, 0.5), e_min=-400.0, e_max=0.0, n_bins=120, n_windows=6, walkers_per_window=3,
           lnf_final=1e-3, exchange_interval=2000, seed=9)
WARM_INTERVALS, ROUNDS = 12, 16


def _oracle_state(n_windows):
    import oracle
    o = oracle.OracleREWL(kind=oracle.BCC, **dict(CFG, n_windows=n_windows))
    o.init_walkers()
    o.run_intervals(WARM_INTERVALS)
    return o


class OraclePart:
    """Stand-in for one handle of a partitioned run: hosts windows [k0, k1) of the run's state."""

    def __init__(self, o, k0, k1):
        import oracle
        self.oracle = oracle
        w = o.walkers()
        self.h, self.m, self.W = o.h, o.m, o.W
        self.n_global_slots = self.h * self.m
        self.window_begin = k0
        self.starts = o.starts
        self.key1 = (CFG["seed"] & 0xffffffff) ^ (CFG["seed"] >> 32)
        g = np.arange(k0 * self.m, k1 * self.m)
        self.gid = g.copy()                       # slot hosted at each position
        self.lng = {int(s): w["lng"][s].copy() for s in g}   # slot states (ln g of the slot's window)
        self.conf = w["replica"][g].copy()        # configuration at each position (stays here)
        self.E, self.bin = w["E"][g].copy(), w["bin"][g].copy()
        self.t = o.exchange_index()
        self.att = np.zeros(self.h - 1, dtype=np.int64)
        self.acc = np.zeros(self.h - 1, dtype=np.int64)

    def _pos(self, s):
        hit = np.nonzero(self.gid == s)[0]
        return int(hit[0]) if hit.size else -1

    def _pairs(self):
        t, m = self.t, self.m
        shift = (t // 2) % m
        for k in range(t & 1, self.h - 1, 2):
            for a in range(m):
                yield k, a, k * m + a, (k + 1) * m + (a + shift) % m

    def _in(self, s, b):
        st = self.starts[s // self.m]
        return 0 <= b - st < self.W

    def _lng(self, s, b):
        return self.lng[s][b - self.starts[s // self.m]]

    def _accept(self, k, a, iA, iB, jB, jA):
        D = ((iA - iB) + jB) - jA
        if D >= 0.0:
            return True
        x = self.oracle.philox4x32_10([self.t & 0xffffffff, self.t >> 32, 3, a], [k, self.key1 ^ 0x5eed5eed])
        return self.oracle.u53(x[0], x[1]) < self.oracle.exp(D)

    def partition_bins(self, bins):
        bins[self.gid] = self.bin

    def partition_lookups(self, bins_all, lk):
        for k, a, i, j in self._pairs():
            pi, pj = self._pos(i), self._pos(j)
            if (pi >= 0) == (pj >= 0):
                continue
            s, o = (i, j) if pi >= 0 else (j, i)
            for n, b in enumerate((bins_all[s], bins_all[o])):
                lk[2 * s + n] = np.float64(self._lng(s, b)).view(np.int64) if self._in(s, b) else 0

    def partition_exchange(self, bins_all, lk_all):
        sw = np.full(self.n_global_slots, -1, dtype=np.int32)
        f = lk_all.view(np.float64)
        for k, a, i, j in self._pairs():
            pi, pj = self._pos(i), self._pos(j)
            if pi < 0 and pj < 0:
                continue
            bA, bB = bins_all[i], bins_all[j]
            if pi >= 0:
                self.att[k] += 1
            if not (self._in(j, bA) and self._in(i, bB)):
                continue
            if pi >= 0 and pj >= 0:
                if self._accept(k, a, self._lng(i, bA), self._lng(i, bB), self._lng(j, bB), self._lng(j, bA)):
                    for arr in (self.conf, self.E, self.bin):
                        arr[pi], arr[pj] = arr[pj], arr[pi]
                    self.acc[k] += 1
            elif self._accept(k, a, f[2 * i], f[2 * i + 1], f[2 * j], f[2 * j + 1]):
                if pi >= 0:
                    sw[i] = j
                    self.acc[k] += 1
                else:
                    sw[j] = i
        self.t += 1
        return sw

    def partition_observe(self):
        pass

    def slot_state_words(self):
        return 1 + self.W

    def slot_export(self, s):
        return np.concatenate([[s], self.lng[s].view(np.int64)])

    def slot_import(self, s_out, buf):
        s_in = int(buf[0])
        p = self._pos(s_out)
        del self.lng[s_out]
        self.lng[s_in] = buf[1:].view(np.float64).copy()
        self.gid[p] = s_in

    def partition_slots(self):
        return self.gid.astype(np.int32)

    def walkers(self):
        return {"lng": np.array([self.lng[int(s)] for s in self.gid]), "E": self.E.copy(), "bin": self.bin.copy(),
                "replica": (self.conf - self.window_begin * self.m).astype(np.int32)}


def _rank(rank, world, n_windows, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1411_4212_gb300.partition import DistComm, PartitionedRun, window_ranges
    dist.init_process_group("gloo")
    k0, k1 = window_ranges(n_windows, world)[rank]
    part = OraclePart(_oracle_state(n_windows), k0, k1)
    run = PartitionedRun([part], DistComm())
    for _ in range(ROUNDS):
        run.exchange_round()
    g = run.gather()
    att = run.comm.sum_(part.att)
    acc = run.comm.sum_(part.acc)
    q.put((rank, {k: v for k, v in g.items()}, att, acc, run.cross_swaps))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("world,n_windows", [(2, 6), (3, 7)])
def test_gloo_ranks_exchange_like_one_process(world, n_windows):
    """Two ranks with three windows each, and three ranks with 3, 2 and 2 windows (uneven ranges)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, n_windows, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    o = _oracle_state(n_windows)
    a0, b0 = o.exchange_counts()
    for _ in range(ROUNDS):
        o.exchange()
    w = o.walkers()
    a1, b1 = o.exchange_counts()
    for rank, g, att, acc, moved in res:
        assert np.array_equal(g["replica"], w["replica"]), rank
        assert np.array_equal(g["E"].view(np.int64), w["E"].view(np.int64)), rank
        assert np.array_equal(g["bin"], w["bin"]), rank
        assert np.array_equal(g["lng"].view(np.int64), w["lng"].view(np.int64)), rank
        assert np.array_equal(att, a1 - a0) and np.array_equal(acc, b1 - b0), rank
    assert sum(r[4] for r in res) > 0, "no slot state crossed the ranks"
    assert int((b1 - b0).sum()) > 0
