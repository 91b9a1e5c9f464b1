"""Window-partitioned REWL: one run of h windows x m walkers split over several handles, one per GPU,
by contiguous window ranges.  Replica exchange crosses the handles (Sec. 4.3, Eq. 5).

The paper runs every walker as a process and exchanges replicas between processes of adjacent windows.
Here a handle (``REWL(..., partition=(k0, k1))``) hosts the walkers of windows [k0, k1).  A
configuration never leaves the GPU it starts on.  An accepted exchange between two handles moves the
two slot states instead (ln g and H of a window, ln f, Philox key and counter: a few KB, against
1 MB for a bcc L = 32 lattice).  The run is then the same Markov chain as one handle holding every
walker, slot for slot.

This module drives the round protocol that include/rewl.h states (bins, lookups, decision, slot-state
moves, second look at the extreme windows).  It only marshals arrays between the handles and a
communicator; every decision and every walk step runs in the library's kernels:

- ``LocalComm``: every part lives in this process (several handles on one or more GPUs);
- ``DistComm``: one part per torch.distributed rank.  It uses gloo on CPU tensors or NCCL on the rank's
  GPU, with one all-reduce of a few KB per step and one of the moving slot states per round.

A part is any object with the handle's partition methods (``partition_bins``, ``partition_lookups``,
``partition_exchange``, ``partition_observe``, ``slot_export``, ``slot_import``, ``walk``, ``flatness``,
``init_walkers``) and the attributes ``n_global_slots`` and ``window_begin``.
"""
import numpy as np

__all__ = ["window_ranges", "LocalComm", "DistComm", "PartitionedRun"]


def window_ranges(n_windows, n_parts):
    """Contiguous window ranges [(k0, k1), ...] of n_parts nearly equal sizes (the first ones larger)."""
    if not 1 <= n_parts <= n_windows:
        raise ValueError("need 1 <= n_parts <= n_windows")
    base, extra = divmod(n_windows, n_parts)
    out, k = [], 0
    for r in range(n_parts):
        n = base + (1 if r < extra else 0)
        out.append((k, k + n))
        k += n
    return out


class LocalComm:
    """Every part of the run in this process: the per-slot arrays are already combined (each part
    writes its own entries into the same array), and slot states are handed over directly."""

    rank, size = 0, 1

    def max_(self, a):
        return a

    def sum_(self, a):
        return a

    def route(self, outgoing, n_slots, words):
        return dict(outgoing)


class DistComm:
    """One part per torch.distributed rank.  Per-slot arrays are combined by all-reduce: entries of
    slots hosted elsewhere hold -1 (max) or 0 (sum).  The moving slot states travel in one all-reduce
    (sum) of an [h m][words] int64 buffer in which each rank fills the rows of the slots it sends."""

    def __init__(self, device=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.rank, self.size = dist.get_rank(), dist.get_world_size()
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
        self.device = device

    def _reduce(self, a, op):
        t = self.torch.from_numpy(np.ascontiguousarray(a).astype(np.int64)).to(self.device)
        self.dist.all_reduce(t, op=op)
        return t.cpu().numpy().astype(a.dtype)

    def max_(self, a):
        return self._reduce(a, self.dist.ReduceOp.MAX)

    def sum_(self, a):
        return self._reduce(a, self.dist.ReduceOp.SUM)

    def route(self, outgoing, n_slots, words):
        buf = np.zeros((n_slots, words), dtype=np.int64)
        sent = np.zeros(n_slots, dtype=np.int64)
        for g, state in outgoing.items():
            buf[g] = state
            sent[g] = 1
        buf = self.sum_(buf.reshape(-1)).reshape(n_slots, words)
        sent = self.sum_(sent)
        return {g: buf[g] for g in np.nonzero(sent)[0].tolist()}


class PartitionedRun:
    """The parts of one run that live in this process (all of them with LocalComm, this rank's with
    DistComm), driven interval by interval: Wang-Landau moves on every part, one replica-exchange
    round across the parts, the flatness test on every part (the order of rewl_run_intervals)."""

    def __init__(self, parts, comm=None):
        self.parts = list(parts)
        self.comm = comm if comm is not None else LocalComm()
        self.S = self.parts[0].n_global_slots
        self.words = None
        self.cross_swaps = 0

    def init_walkers(self):
        for p in self.parts:
            p.init_walkers()

    def exchange_round(self):
        S = self.S
        bins = np.full(S, -1, dtype=np.int32)
        for p in self.parts:
            p.partition_bins(bins)
        bins = self.comm.max_(bins)
        lk = np.zeros(2 * S, dtype=np.int64)
        for p in self.parts:
            p.partition_lookups(bins, lk)
        lk = self.comm.sum_(lk)
        moves = []
        for p in self.parts:
            sw = p.partition_exchange(bins, lk)
            moves += [(p, int(g), int(sw[g])) for g in np.nonzero(sw >= 0)[0]]
        out = {g: p.slot_export(g) for p, g, _ in moves}
        if self.words is None:
            self.words = int(self.parts[0].slot_state_words())
        states = self.comm.route(out, S, self.words)
        for p, g, o in moves:
            p.slot_import(g, states[o])
        self.cross_swaps += len(moves)
        for p in self.parts:
            p.partition_observe()

    def run_intervals(self, n):
        for _ in range(int(n)):
            for p in self.parts:
                p.walk()
            self.exchange_round()
            for p in self.parts:
                p.flatness()

    def gather(self):
        """Every global slot's state, combined over the parts and ranks: ln g, H, E, bin, ln f, stage,
        accepts, steps, init_moves by global slot, and replica = the global id of the configuration
        it holds (window_begin m + the configuration's index in its part)."""
        S = self.S
        acc, dtypes = None, None
        for p in self.parts:
            w = p.walkers()
            gid = p.partition_slots()
            if acc is None:
                acc = {k: np.zeros((S,) + v.shape[1:], dtype=np.int64) for k, v in w.items()}
                dtypes = {k: v.dtype for k, v in w.items()}
            for k, v in w.items():
                if k == "replica":
                    v = v + p.window_begin * p.m
                v = np.ascontiguousarray(v)
                bits = v.view(np.int64) if v.dtype == np.float64 else v.astype(np.int64)
                acc[k][gid] = bits
        out = {}
        for k, v in acc.items():
            v = self.comm.sum_(v.reshape(-1)).reshape(v.shape)
            out[k] = v.view(np.float64) if dtypes[k] == np.float64 else v.astype(dtypes[k])
        return out
