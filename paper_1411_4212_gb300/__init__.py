"""GB300 replica-exchange Wang-Landau (REWL) sampling for the classical Heisenberg model.

Thin ctypes binding over ``librewl.so`` (C ABI in ``include/rewl.h``): argument marshalling only.
Every step of the sampling runs in the library's CUDA kernels; there is no CPU fallback.  PyTorch,
when present, supplies the CUDA stream (``torch.cuda.current_stream()``) and device buffers for the
device-pointer entry points.

Method: Perera, Li, Eisenbach, Vogel, Landau, "Replica-exchange Wang-Landau sampling: pushing the
limits of Monte Carlo simulations in materials sciences" -- Heisenberg model on bcc (Sec. 3, Eq. 1),
Wang-Landau walk (Sec. 4.2, Eq. 4), windows and replica exchange (Sec. 4.3, Eq. 5), joining of the
ln g fragments (Sec. 4.3), thermodynamics from g(E) (Sec. 4.1, Eq. 2-3).
"""
import ctypes as C
import math
import os

import numpy as np

__all__ = ["REWL", "Batch", "Mlp", "RewlError", "load_library", "thermo", "peak_temperature", "stitch_device",
           "device_exp", "measure_smem_bandwidth", "BCC", "CHAIN", "TABLE", "PRODUCTION", "TRAJECTORY"]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librewl.so")

BCC, CHAIN, TABLE = 0, 1, 2
ITERATION_WALKER, ITERATION_WINDOW = 0, 1
PRODUCTION, TRAJECTORY = 0, 1
RESOLVER_AUTO, RESOLVER_SCAN, RESOLVER_BLOCKS, RESOLVER_SEQUENTIAL = 0, 1, 2, 3
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE = range(6)
_STATUS = {0: "REWL_OK", 1: "REWL_EINVAL", 2: "REWL_ENOMEM", 3: "REWL_ECUDA", 4: "REWL_ETIMEOUT",
           5: "REWL_ESTATE"}


class RewlError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Lattice(C.Structure):
    _fields_ = [("kind", C.c_int32), ("L", C.c_int32), ("n_sites", C.c_int32), ("z", C.c_int32),
                ("nbr", C.POINTER(C.c_int32)), ("J", C.POINTER(C.c_double))]


class Couplings(C.Structure):
    _fields_ = [("n_shells", C.c_int32), ("J", C.c_double * 4)]


class Windows(C.Structure):
    _fields_ = [("e_min", C.c_double), ("e_max", C.c_double), ("n_bins", C.c_int32),
                ("n_windows", C.c_int32)]


class Config(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("mode", C.c_int32), ("group_size", C.c_int32),
                ("exchange_interval", C.c_int64), ("max_moves_per_stage", C.c_int64),
                ("init_max_moves", C.c_int64), ("recompute_every", C.c_int32), ("iteration", C.c_int32),
                ("lnf_initial", C.c_double), ("timeout_s", C.c_double), ("cuda_stream", C.c_void_p),
                ("resolver", C.c_int32)]


class StageStats(C.Structure):
    _fields_ = [("moves", C.c_int64), ("accepts", C.c_int64), ("exchange_attempts", C.c_int64),
                ("exchange_accepts", C.c_int64), ("intervals", C.c_int32), ("n_halved", C.c_int32),
                ("n_done", C.c_int32), ("all_done", C.c_int32), ("min_lnf", C.c_double),
                ("max_lnf", C.c_double), ("max_energy_drift", C.c_double), ("elapsed_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(C.Structure):
    _fields_ = [("n_sites", C.c_int32), ("z", C.c_int32), ("n_slots", C.c_int32), ("n_replicas", C.c_int32),
                ("n_bins", C.c_int32), ("n_windows", C.c_int32), ("walkers_per_window", C.c_int32),
                ("window_bins", C.c_int32), ("group_size", C.c_int32), ("mode", C.c_int32),
                ("e_min", C.c_double), ("e_max", C.c_double), ("bin_width", C.c_double),
                ("initial_energy", C.c_double), ("exchange_index", C.c_int64), ("intervals_done", C.c_int64),
                ("shared_bytes_per_walker", C.c_size_t), ("lattice_in_shared", C.c_int32),
                ("pipelined", C.c_int32), ("conflict_entries", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class BatchTuning(C.Structure):
    _fields_ = [("workers_per_block", C.c_int32), ("smem_lattice_max_n", C.c_int32),
                ("owner_entries_max", C.c_int32)]


class BatchInfo(C.Structure):
    _fields_ = [("n_jobs", C.c_int32), ("n_items", C.c_int32), ("n_active_jobs", C.c_int32),
                ("workers_per_block", C.c_int32), ("smem_lattice_max_n", C.c_int32),
                ("owner_entries_max", C.c_int32), ("grid", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("n_smem_lattice_jobs", C.c_int32), ("arena_bytes", C.c_int64),
                ("intervals_done", C.c_int64), ("graphs_built", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Counters(C.Structure):
    _fields_ = [("moves", C.c_int64), ("accepts", C.c_int64), ("recomputes", C.c_int64),
                ("batches_scan", C.c_int64), ("batches_blocks", C.c_int64), ("batches_sequential", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_vp = C.c_void_p


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def load_library(path=LIB_PATH):
    """Load librewl.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(path)
    st = C.c_int
    sig = {
        "rewl_create": ([C.POINTER(Lattice), C.POINTER(Couplings), C.POINTER(Windows), C.c_int, C.c_double,
                         C.c_double, C.c_double, C.POINTER(Config), C.POINTER(_vp)], st),
        "rewl_init_walkers": ([_vp], st),
        "rewl_run_intervals": ([_vp, C.c_int, C.POINTER(StageStats)], st),
        "rewl_run_stage": ([_vp, C.POINTER(StageStats)], st),
        "rewl_exchange": ([_vp, C.POINTER(StageStats)], st),
        "rewl_walk": ([_vp], st),
        "rewl_autotune": ([_vp, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_double)], st),
        "rewl_flatness": ([_vp], st),
        "rewl_merge_lng": ([_vp, _vp, _vp], st),
        "rewl_merge_lng_device": ([_vp, _vp], st),
        "rewl_stitch_device": ([_vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp], st),
        "rewl_stitch_device_noalloc": ([_vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp], st),
        "rewl_thermo": ([_vp, _vp, C.c_int, C.c_double, _vp, C.c_int, _vp, _vp, _vp, _vp], st),
        "rewl_set_initial_lng": ([_vp, _vp, C.c_double], st),
        "rewl_peak_temperature": ([_vp, _vp, C.c_int, C.POINTER(C.c_double), _vp], st),
        "rewl_state_bytes": ([_vp, C.POINTER(C.c_int64)], st),
        "rewl_save_state": ([_vp, _vp, C.c_int64], st),
        "rewl_load_state": ([_vp, _vp, C.c_int64], st),
        "rewl_create_partition": ([C.POINTER(Lattice), C.POINTER(Couplings), C.POINTER(Windows), C.c_int, C.c_double,
                                   C.c_double, C.c_double, C.POINTER(Config), C.c_int, C.c_int, C.POINTER(_vp)], st),
        "rewl_partition_slots": ([_vp, _vp], st),
        "rewl_partition_bins": ([_vp, _vp], st),
        "rewl_partition_lookups": ([_vp, _vp, _vp], st),
        "rewl_partition_exchange": ([_vp, _vp, _vp, _vp], st),
        "rewl_partition_observe": ([_vp], st),
        "rewl_slot_state_bytes": ([_vp, C.POINTER(C.c_int64)], st),
        "rewl_slot_export": ([_vp, C.c_int32, _vp], st),
        "rewl_slot_import": ([_vp, C.c_int32, _vp], st),
        "rewl_get_info": ([_vp, C.POINTER(Info)], st),
        "rewl_get_walkers": ([_vp] + [_vp] * 10, st),
        "rewl_get_spins": ([_vp, _vp], st),
        "rewl_get_exchange_counts": ([_vp, _vp, _vp], st),
        "rewl_get_round_trips": ([_vp, _vp, _vp], st),
        "rewl_get_counters": ([_vp, C.POINTER(Counters)], st),
        "rewl_get_neighbours": ([_vp, _vp, _vp], st),
        "rewl_replica_energies": ([_vp, _vp], st),
        "rewl_last_error": ([_vp], C.c_char_p),
        "rewl_destroy": ([_vp], None),
        "rewl_device_exp": ([_vp, _vp, C.c_int], st),
        "rewl_measure_smem_bandwidth": ([_vp, _vp, _vp], st),
        "rewl_batch_create": ([C.POINTER(_vp), C.c_int, _vp, C.POINTER(_vp)], st),
        "rewl_batch_set_tuning": ([_vp, C.POINTER(BatchTuning)], st),
        "rewl_batch_autotune": ([_vp, C.c_int64, C.POINTER(BatchTuning), C.POINTER(C.c_double)], st),
        "rewl_batch_run_intervals": ([_vp, C.c_int], st),
        "rewl_batch_run_to_convergence": ([_vp, C.c_int64, C.c_int, C.POINTER(C.c_int)], st),
        "rewl_batch_get_info": ([_vp, C.POINTER(BatchInfo)], st),
        "rewl_batch_destroy": ([_vp], None),
        "rewl_mlp_param_count": ([], C.c_int64),
        "rewl_mlp_create": ([_vp, _vp, C.c_uint64, _vp, C.POINTER(_vp)], st),
        "rewl_mlp_set_params": ([_vp, _vp], st),
        "rewl_mlp_get_params": ([_vp, _vp, _vp], st),
        "rewl_mlp_forward": ([_vp, _vp, C.c_int64, _vp], st),
        "rewl_mlp_gradient": ([_vp, _vp, _vp, _vp, C.c_int, C.POINTER(C.c_double), _vp], st),
        "rewl_mlp_train": ([_vp, _vp, _vp, _vp, C.c_int, C.c_int, C.c_float, _vp], st),
        "rewl_mlp_features": ([_vp, _vp, _vp, _vp], st),
        "rewl_mlp_warm_start": ([_vp, _vp, C.c_double, _vp], st),
        "rewl_mlp_destroy": ([_vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(status, handle=None):
    if status != OK:
        msg = load_library().rewl_last_error(handle)
        raise RewlError(status, msg.decode() if msg else "")


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class REWL:
    """One REWL simulation: h windows x m walkers over [e_min, e_max) in n_bins bins.

    kind: BCC (L cells per side, couplings per shell J[0..3]), CHAIN (L spins, J[0]) or TABLE
    (nbr, Jt arrays [z][n_sites]).  mode: PRODUCTION (FP32 spins, fixed-point ln g / energy) or
    TRAJECTORY (FP64, bit-reproducible walk).  resolver: RESOLVER_AUTO, or one of RESOLVER_SCAN /
    _BLOCKS / _SEQUENTIAL forced for every batch of the production pipelined walker (the same
    decisions at a different cost).
    """

    def __init__(self, kind=BCC, L=4, J=(1.0, 0.5), nbr=None, Jt=None, e_min=math.nan, e_max=math.nan,
                 n_bins=200, n_windows=4, walkers_per_window=2, overlap=0.75, flatness=0.8,
                 lnf_final=1e-3, seed=1, mode=PRODUCTION, group_size=0, exchange_interval=10000,
                 max_moves_per_stage=0, init_max_moves=0, recompute_every=0, lnf_initial=0.0,
                 timeout_s=0.0, stream=None, iteration=0, resolver=RESOLVER_AUTO, partition=None):
        lib = load_library()
        lat = Lattice()
        lat.kind = kind
        lat.L = L
        self._keep = []
        if kind == TABLE:
            nbr = np.ascontiguousarray(nbr, dtype=np.int32)
            Jt = np.ascontiguousarray(Jt, dtype=np.float64)
            lat.z, lat.n_sites = nbr.shape
            lat.nbr = nbr.ctypes.data_as(C.POINTER(C.c_int32))
            lat.J = Jt.ctypes.data_as(C.POINTER(C.c_double))
            self._keep += [nbr, Jt]
        cp = Couplings()
        J = list(J)
        cp.n_shells = len(J)
        for i in range(4):
            cp.J[i] = J[i] if i < len(J) else 0.0
        win = Windows()
        win.e_min, win.e_max, win.n_bins, win.n_windows = e_min, e_max, n_bins, n_windows
        cfg = Config()
        cfg.seed = seed
        cfg.mode = mode
        cfg.group_size = group_size
        cfg.exchange_interval = exchange_interval
        cfg.max_moves_per_stage = max_moves_per_stage
        cfg.init_max_moves = init_max_moves
        cfg.recompute_every = recompute_every
        cfg.iteration = iteration
        cfg.lnf_initial = lnf_initial
        cfg.timeout_s = timeout_s
        cfg.cuda_stream = _stream_ptr(stream)
        cfg.resolver = resolver
        h = _vp()
        if partition is None:
            _check(lib.rewl_create(C.byref(lat), C.byref(cp), C.byref(win), walkers_per_window, overlap, flatness,
                                   lnf_final, C.byref(cfg), C.byref(h)))
            self.window_begin = 0
        else:
            k0, k1 = partition
            _check(lib.rewl_create_partition(C.byref(lat), C.byref(cp), C.byref(win), walkers_per_window, overlap,
                                             flatness, lnf_final, C.byref(cfg), int(k0), int(k1), C.byref(h)))
            self.window_begin = int(k0)
        self.partition = partition
        self._h = h
        self._lib = lib
        info = self.info()
        self.N, self.z = info["n_sites"], info["z"]
        self.n_slots, self.B, self.h = info["n_slots"], info["n_bins"], info["n_windows"]
        self.m, self.W = info["walkers_per_window"], info["window_bins"]
        self.e_min, self.e_max, self.dE = info["e_min"], info["e_max"], info["bin_width"]
        self.exchange_interval = exchange_interval
        self.lnf_final = lnf_final
        self.mode = mode

    # -- lifecycle -------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.rewl_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- sampling --------------------------------------------------------------------------
    def init_walkers(self):
        _check(self._lib.rewl_init_walkers(self._h), self._h)

    def run_intervals(self, n, stats=True):
        s = StageStats() if stats else None
        _check(self._lib.rewl_run_intervals(self._h, int(n), C.byref(s) if s is not None else None), self._h)
        return s.as_dict() if s is not None else None

    def run_stage(self):
        s = StageStats()
        st = self._lib.rewl_run_stage(self._h, C.byref(s))
        if st not in (OK, ETIMEOUT):
            _check(st, self._h)
        d = s.as_dict()
        d["capped"] = st == ETIMEOUT
        return d

    def exchange(self):
        s = StageStats()
        _check(self._lib.rewl_exchange(self._h, C.byref(s)), self._h)
        return s.as_dict()

    def autotune(self, trial_moves=2000):
        """Conflict-table size of a pipelined walker with the lattice in global memory, chosen by
        timing; the trial moves are ordinary moves.  Returns {"conflict_entries", "trial_ms"}."""
        e, ms = C.c_int32(), C.c_double()
        _check(self._lib.rewl_autotune(self._h, int(trial_moves), C.byref(e), C.byref(ms)), self._h)
        return {"conflict_entries": e.value, "trial_ms": ms.value}

    def walk(self):
        """Enqueue one interval of trial moves (walker kernel only); does not block."""
        _check(self._lib.rewl_walk(self._h), self._h)

    def exchange_async(self):
        """Enqueue one replica-exchange round; does not block."""
        _check(self._lib.rewl_exchange(self._h, None), self._h)

    def flatness(self):
        """Enqueue the flatness test and ln f update; does not block."""
        _check(self._lib.rewl_flatness(self._h), self._h)

    def merge(self):
        out = np.zeros(self.B)
        cen = np.zeros(self.B)
        _check(self._lib.rewl_merge_lng(self._h, _ptr(out), _ptr(cen)), self._h)
        return out, cen

    def merge_device(self, out):
        """Merged ln g into a device buffer (e.g. a torch.float64 CUDA tensor of n_bins)."""
        _check(self._lib.rewl_merge_lng_device(self._h, C.c_void_p(out.data_ptr())), self._h)
        return out

    def set_initial_lng(self, lng, lnf0):
        lng = np.ascontiguousarray(lng, dtype=np.float64)
        assert lng.size == self.B
        _check(self._lib.rewl_set_initial_lng(self._h, _ptr(lng), float(lnf0)), self._h)

    def run_to_convergence(self, max_stages=1000, log=None):
        """Stages (rewl_run_stage) until every walker has ln f < lnf_final.  Stops at the first stage
        that a cap (max_moves_per_stage, timeout_s) ended: that stage's dict has capped = True.
        log: a writable text file that receives one JSON line per stage (stage_report of the stage)."""
        import json
        stages = []
        for _ in range(max_stages):
            st = self.run_stage()
            stages.append(st)
            if log is not None:
                log.write(json.dumps(self.stage_report(st)) + "\n")
                log.flush()
            if st["all_done"] or st["capped"]:
                break
        return stages

    def stage_report(self, stage=None):
        """The run's state as plain numbers (the quantities the paper reports, Sec. 5): moves/s of the stage
        when its stats are given, accept rate, replica-exchange acceptance per window pair, round trips
        per configuration, ln f per walker and each walker's flatness ratio min H / mean H."""
        w = self.walkers()
        att, acc = self.exchange_counts()
        trips, _ = self.round_trips()
        c = self.counters()
        H = w["H"].astype(np.float64)
        mean = H.mean(axis=1)
        rep = {"moves": int(c["moves"]), "accept_rate": c["accepts"] / max(1, c["moves"]),
               "exchange_acceptance": [float(a) / max(1, int(t)) for a, t in zip(acc, att)],
               "round_trips": [int(v) for v in trips], "lnf": [float(v) for v in w["lnf"]],
               "stage": [int(v) for v in w["stage"]],
               "flatness_ratio": [float(m) for m in np.where(mean > 0, H.min(axis=1) / np.maximum(mean, 1e-300), 0.0)]}
        if stage is not None:
            rep["stage_moves_per_s"] = stage["moves"] / max(stage["elapsed_ms"] * 1e-3, 1e-12)
            rep["stage_intervals"] = stage["intervals"]
            rep["capped"] = bool(stage.get("capped", False))
        return rep

    # -- state -----------------------------------------------------------------------------
    def info(self):
        i = Info()
        _check(self._lib.rewl_get_info(self._h, C.byref(i)), self._h)
        return i.as_dict()

    def walkers(self):
        S, W = self.n_slots, self.W
        out = dict(lng=np.zeros((S, W)), H=np.zeros((S, W), dtype=np.uint32), E=np.zeros(S),
                   bin=np.zeros(S, dtype=np.int32), lnf=np.zeros(S), replica=np.zeros(S, dtype=np.int32),
                   stage=np.zeros(S, dtype=np.int32), accepts=np.zeros(S, dtype=np.int64),
                   steps=np.zeros(S, dtype=np.int64), init_moves=np.zeros(S, dtype=np.int64))
        _check(self._lib.rewl_get_walkers(self._h, *[_ptr(out[k]) for k in
                                                     ("lng", "H", "E", "bin", "lnf", "replica", "stage",
                                                      "accepts", "steps", "init_moves")]), self._h)
        return out

    def spins(self):
        sp = np.zeros((self.n_slots, 3, self.N))
        _check(self._lib.rewl_get_spins(self._h, _ptr(sp)), self._h)
        return sp

    def exchange_counts(self):
        n = max(self.h - 1, 1)
        a = np.zeros(n, dtype=np.int64)
        b = np.zeros(n, dtype=np.int64)
        _check(self._lib.rewl_get_exchange_counts(self._h, _ptr(a), _ptr(b)), self._h)
        return a[: self.h - 1], b[: self.h - 1]

    def round_trips(self):
        """(round trips completed [S], extreme window seen last [S]: -1 none, 0 lowest, 1 highest)
        per configuration."""
        c = np.zeros(self.n_slots, dtype=np.int64)
        last = np.zeros(self.n_slots, dtype=np.int32)
        _check(self._lib.rewl_get_round_trips(self._h, _ptr(c), _ptr(last)), self._h)
        return c, last

    def counters(self):
        c = Counters()
        _check(self._lib.rewl_get_counters(self._h, C.byref(c)), self._h)
        return c.as_dict()

    def neighbours(self):
        nbr = np.zeros((self.z, self.N), dtype=np.int32)
        J = np.zeros((self.z, self.N))
        _check(self._lib.rewl_get_neighbours(self._h, _ptr(nbr), _ptr(J)), self._h)
        return nbr, J

    def replica_energies(self):
        E = np.zeros(self.n_slots)
        _check(self._lib.rewl_replica_energies(self._h, _ptr(E)), self._h)
        return E

    def centres(self):
        return self.e_min + (np.arange(self.B) + 0.5) * self.dE

    # -- checkpoints -------------------------------------------------------------------------
    def save_state(self, path=None):
        """The handle's checkpoint as a uint8 array (written to `path` as well when given)."""
        n = C.c_int64()
        _check(self._lib.rewl_state_bytes(self._h, C.byref(n)), self._h)
        buf = np.empty(n.value, dtype=np.uint8)
        _check(self._lib.rewl_save_state(self._h, _ptr(buf), buf.size), self._h)
        if path is not None:
            buf.tofile(path)
        return buf

    def load_state(self, src):
        """Resume from a checkpoint (a save_state array, or the path of a file it was written to)."""
        buf = np.fromfile(src, dtype=np.uint8) if isinstance(src, (str, os.PathLike)) else \
            np.ascontiguousarray(src, dtype=np.uint8)
        _check(self._lib.rewl_load_state(self._h, _ptr(buf), buf.size), self._h)

    # -- partitioned runs (see partition.py for the round protocol) -------------------------
    @property
    def n_global_slots(self):
        return self.h * self.m

    def partition_slots(self):
        g = np.zeros(self.n_slots, dtype=np.int32)
        _check(self._lib.rewl_partition_slots(self._h, _ptr(g)), self._h)
        return g

    def partition_bins(self, bins):
        """Write the bins of the hosted slots' configurations into bins (int32 [h m]) in place."""
        assert bins.dtype == np.int32 and bins.flags.c_contiguous and bins.size == self.n_global_slots
        _check(self._lib.rewl_partition_bins(self._h, _ptr(bins)), self._h)

    def partition_lookups(self, bins_all, lk):
        """Write the hosted slots' ln g lookups of the coming round into lk (int64 [2 h m]) in place."""
        bins_all = np.ascontiguousarray(bins_all, dtype=np.int32)
        assert lk.dtype == np.int64 and lk.flags.c_contiguous and lk.size == 2 * self.n_global_slots
        _check(self._lib.rewl_partition_lookups(self._h, _ptr(bins_all), _ptr(lk)), self._h)

    def partition_exchange(self, bins_all, lk_all):
        """The exchange round; returns swap_with (int32 [h m])."""
        bins_all = np.ascontiguousarray(bins_all, dtype=np.int32)
        lk_all = np.ascontiguousarray(lk_all, dtype=np.int64)
        sw = np.zeros(self.n_global_slots, dtype=np.int32)
        _check(self._lib.rewl_partition_exchange(self._h, _ptr(bins_all), _ptr(lk_all), _ptr(sw)), self._h)
        return sw

    def partition_observe(self):
        _check(self._lib.rewl_partition_observe(self._h), self._h)

    def slot_state_words(self):
        n = C.c_int64()
        _check(self._lib.rewl_slot_state_bytes(self._h, C.byref(n)), self._h)
        return n.value // 8

    def slot_export(self, g):
        buf = np.zeros(self.slot_state_words(), dtype=np.int64)
        _check(self._lib.rewl_slot_export(self._h, int(g), _ptr(buf)), self._h)
        return buf

    def slot_import(self, g_out, buf):
        buf = np.ascontiguousarray(buf, dtype=np.int64)
        assert buf.size == self.slot_state_words()
        _check(self._lib.rewl_slot_import(self._h, int(g_out), _ptr(buf)), self._h)


class Batch:
    """Many REWL jobs (REWL objects, bcc, same mode / shell count / exchange interval) run together:
    one persistent walker launch over every walker slot, replayed from a CUDA graph.  The jobs must
    outlive the batch; their results are read from the REWL objects as usual."""

    def __init__(self, jobs, stream=None):
        lib = load_library()
        self._lib = lib
        self.jobs = list(jobs)
        arr = (_vp * len(self.jobs))(*[j._h for j in self.jobs])
        b = _vp()
        _check(lib.rewl_batch_create(arr, len(self.jobs), _stream_ptr(stream), C.byref(b)))
        self._b = b

    def close(self):
        if getattr(self, "_b", None):
            self._lib.rewl_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_tuning(self, workers_per_block, smem_lattice_max_n, owner_entries_max=0):
        t = BatchTuning(int(workers_per_block), int(smem_lattice_max_n), int(owner_entries_max))
        _check(self._lib.rewl_batch_set_tuning(self._b, C.byref(t)))

    def autotune(self, trial_moves=2000):
        t = BatchTuning()
        ms = C.c_double()
        _check(self._lib.rewl_batch_autotune(self._b, int(trial_moves), C.byref(t), C.byref(ms)))
        return {"workers_per_block": t.workers_per_block, "smem_lattice_max_n": t.smem_lattice_max_n,
                "owner_entries_max": t.owner_entries_max, "trial_ms": ms.value}

    def run_intervals(self, n):
        _check(self._lib.rewl_batch_run_intervals(self._b, int(n)))

    def run_to_convergence(self, max_intervals, check_every=8):
        """Returns (converged, n_done_jobs)."""
        nd = C.c_int()
        st = self._lib.rewl_batch_run_to_convergence(self._b, int(max_intervals), int(check_every), C.byref(nd))
        if st not in (OK, ETIMEOUT):
            _check(st)
        return st == OK, nd.value

    def info(self):
        i = BatchInfo()
        _check(self._lib.rewl_batch_get_info(self._b, C.byref(i)))
        return i.as_dict()


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


class Mlp:
    """Learned warm start: MLP (E/N, 1/L, J1..J4) -> ln g/N, trained and evaluated by the library's
    kernels.  shift/scale: the fixed input normalisation x' = (x - shift) * scale (6 values each)."""

    N_IN = 6

    def __init__(self, shift, scale, seed=0, stream=None):
        lib = load_library()
        self._lib = lib
        self.n_params = int(lib.rewl_mlp_param_count())
        sh, sc = _f32(shift), _f32(scale)
        m = _vp()
        _check(lib.rewl_mlp_create(_ptr(sh), _ptr(sc), int(seed), _stream_ptr(stream), C.byref(m)))
        self._m = m

    def close(self):
        if getattr(self, "_m", None):
            self._lib.rewl_mlp_destroy(self._m)
            self._m = None

    def __del__(self):
        self.close()

    def set_params(self, p):
        p = _f32(p)
        assert p.size == self.n_params
        _check(self._lib.rewl_mlp_set_params(self._m, _ptr(p)))

    def params(self, bf16=False):
        """FP32 master parameters, or (bf16=True) the BF16 weights the kernels use, widened to FP32."""
        if bf16:
            raw = np.zeros(self.n_params, dtype=np.uint16)
            _check(self._lib.rewl_mlp_get_params(self._m, None, _ptr(raw)))
            return (raw.astype(np.uint32) << 16).view(np.float32)
        p = np.zeros(self.n_params, dtype=np.float32)
        _check(self._lib.rewl_mlp_get_params(self._m, _ptr(p), None))
        return p

    def forward(self, x):
        x = _f32(x, (-1, self.N_IN))
        y = np.zeros(x.shape[0], dtype=np.float32)
        _check(self._lib.rewl_mlp_forward(self._m, _ptr(x), x.shape[0], _ptr(y)))
        return y

    def gradient(self, x, target, run_offsets):
        x = _f32(x, (-1, self.N_IN))
        t = _f32(target)
        seg = np.ascontiguousarray(run_offsets, dtype=np.int32)
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = C.c_double()
        _check(self._lib.rewl_mlp_gradient(self._m, _ptr(x), _ptr(t), _ptr(seg), seg.size - 1, C.byref(loss), _ptr(g)))
        return loss.value, g

    def train(self, x, target, run_offsets, steps, lr):
        x = _f32(x, (-1, self.N_IN))
        t = _f32(target)
        seg = np.ascontiguousarray(run_offsets, dtype=np.int32)
        hist = np.zeros(int(steps), dtype=np.float32)
        _check(self._lib.rewl_mlp_train(self._m, _ptr(x), _ptr(t), _ptr(seg), seg.size - 1, int(steps), float(lr),
                                        _ptr(hist)))
        return hist

    def warm_start(self, job, lnf0):
        """Install the predicted ln g in every walker of `job` (a REWL) with ln f = lnf0."""
        lng = np.zeros(job.B)
        _check(self._lib.rewl_mlp_warm_start(self._m, job._h, float(lnf0), _ptr(lng)))
        return lng


def mlp_features(job, lng=None):
    """(x [n_bins][6], ln g/N [n_bins] or None) of a bcc REWL job's bins."""
    lib = load_library()
    x = np.zeros((job.B, Mlp.N_IN), dtype=np.float32)
    t = np.zeros(job.B, dtype=np.float32) if lng is not None else None
    lp = None if lng is None else np.ascontiguousarray(lng, dtype=np.float64)
    _check(lib.rewl_mlp_features(job._h, _ptr(lp), _ptr(x), _ptr(t)))
    return x, t


def thermo(lng, centres, n_spins, T, stream=None):
    """(U(T), C(T)/N, ln Z(T)) from ln g at bin centres (k_B = 1), computed on the GPU."""
    lib = load_library()
    lng = np.ascontiguousarray(lng, dtype=np.float64)
    centres = np.ascontiguousarray(centres, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    U, Cv, lnZ = np.zeros(T.size), np.zeros(T.size), np.zeros(T.size)
    _check(lib.rewl_thermo(_ptr(lng), _ptr(centres), lng.size, float(n_spins), _ptr(T), T.size, _ptr(U),
                           _ptr(Cv), _ptr(lnZ), _stream_ptr(stream)))
    return U, Cv, lnZ


def peak_temperature(T, Cv, stream=None):
    """Temperature of the maximum of C(T): grid argmax refined by a 3-point parabola (library kernel)."""
    lib = load_library()
    T = np.ascontiguousarray(T, dtype=np.float64)
    Cv = np.ascontiguousarray(Cv, dtype=np.float64)
    out = C.c_double()
    _check(lib.rewl_peak_temperature(_ptr(T), _ptr(Cv), T.size, C.byref(out), _stream_ptr(stream)))
    return out.value


def stitch_device(frag, starts, n_bins, out, bstar=None, stream=None):
    """Join fragments frag [h][m][W] (float64 CUDA tensor) into out [n_bins] (float64 CUDA tensor)."""
    lib = load_library()
    h, m, W = frag.shape
    st = np.ascontiguousarray(starts, dtype=np.int32)
    _check(lib.rewl_stitch_device(C.c_void_p(frag.data_ptr()), _ptr(st), h, m, W, int(n_bins),
                                  C.c_void_p(out.data_ptr()), None if bstar is None else C.c_void_p(bstar.data_ptr()),
                                  _stream_ptr(stream)))
    return out


def stitch_device_noalloc(frag, starts, n_bins, out, bstar=None, stream=None):
    """Same as stitch_device, for callers that must not allocate device memory: the scratch is a
    fixed 4 MiB device array inside the library (shared by all calls; see include/rewl.h)."""
    lib = load_library()
    h, m, W = frag.shape
    st = np.ascontiguousarray(starts, dtype=np.int32)
    _check(lib.rewl_stitch_device_noalloc(C.c_void_p(frag.data_ptr()), _ptr(st), h, m, W, int(n_bins),
                                          C.c_void_p(out.data_ptr()),
                                          None if bstar is None else C.c_void_p(bstar.data_ptr()),
                                          _stream_ptr(stream)))
    return out


def device_exp(x):
    lib = load_library()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    _check(lib.rewl_device_exp(_ptr(x), _ptr(y), x.size))
    return y


def measure_smem_bandwidth(stream=None):
    lib = load_library()
    bw = C.c_double()
    ms = C.c_double()
    _check(lib.rewl_measure_smem_bandwidth(C.byref(bw), C.byref(ms), _stream_ptr(stream)))
    return bw.value, ms.value
