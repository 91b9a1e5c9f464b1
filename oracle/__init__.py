"""FP64 single-threaded REWL oracle (ctypes wrapper over ``rewl_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference leg.  The library under ``paper_1411_4212_gb300`` never imports it and
shares no code with it.
"""
import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None


class _Params(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("L", C.c_int32), ("n_shells", C.c_int32),
        ("J", C.c_double * 4),
        ("n_sites", C.c_int32), ("z", C.c_int32),
        ("nbr", C.POINTER(C.c_int32)), ("Jt", C.POINTER(C.c_double)),
        ("e_min", C.c_double), ("e_max", C.c_double),
        ("n_bins", C.c_int32), ("n_windows", C.c_int32), ("walkers_per_window", C.c_int32),
        ("overlap", C.c_double), ("flatness", C.c_double), ("lnf_final", C.c_double),
        ("lnf_initial", C.c_double),
        ("seed", C.c_uint64), ("exchange_interval", C.c_int64), ("group_size", C.c_int32),
        ("init_max_moves", C.c_int64), ("iteration", C.c_int32),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        up = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
        lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
        L.ro_philox4x32_10.argtypes = [up, up, up]
        L.ro_u53.argtypes = [C.c_uint32, C.c_uint32]
        L.ro_u53.restype = C.c_double
        L.ro_exp.argtypes = [C.c_double]
        L.ro_exp.restype = C.c_double
        L.ro_bcc_offsets.argtypes = [C.c_int, ip, ip, ip, ip]
        L.ro_bcc_ground_state.argtypes = [C.c_int, C.c_int, dp]
        L.ro_bcc_ground_state.restype = C.c_double
        L.ro_window_layout.argtypes = [C.c_int, C.c_int, C.c_double, ip]
        L.ro_sum32.argtypes = [dp, C.c_int]
        L.ro_sum32.restype = C.c_double
        L.ro_create.argtypes = [C.POINTER(_Params), C.POINTER(C.c_void_p), C.c_char_p, C.c_int]
        L.ro_destroy.argtypes = [C.c_void_p]
        L.ro_init_walkers.argtypes = [C.c_void_p]
        L.ro_run_intervals.argtypes = [C.c_void_p, C.c_int]
        L.ro_run_moves_only.argtypes = [C.c_void_p, C.c_int64]
        L.ro_exchange.argtypes = [C.c_void_p]
        L.ro_flatness.argtypes = [C.c_void_p]
        i32p = C.POINTER(C.c_int32)
        L.ro_sizes.argtypes = [C.c_void_p] + [i32p] * 7
        L.ro_energy_grid.argtypes = [C.c_void_p] + [C.POINTER(C.c_double)] * 3
        L.ro_window_starts.argtypes = [C.c_void_p, ip]
        L.ro_neighbours.argtypes = [C.c_void_p, ip, dp]
        L.ro_initial_energy.argtypes = [C.c_void_p]
        L.ro_initial_energy.restype = C.c_double
        L.ro_get_walkers.argtypes = [C.c_void_p, dp, up, dp, ip, dp, ip, lp, ip, lp, lp]
        L.ro_get_spins.argtypes = [C.c_void_p, dp]
        L.ro_get_exchange_counts.argtypes = [C.c_void_p, lp, lp]
        L.ro_get_round_trips.argtypes = [C.c_void_p, lp, ip]
        L.ro_max_drift.argtypes = [C.c_void_p]
        L.ro_max_drift.restype = C.c_double
        L.ro_exchange_index.argtypes = [C.c_void_p]
        L.ro_exchange_index.restype = C.c_int64
        L.ro_set_lng.argtypes = [C.c_void_p, dp, C.c_double]
        L.ro_draw_direction.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32, dp]
        L.ro_draw_site.argtypes = [C.c_void_p, C.c_uint32, C.c_uint64, C.c_uint32,
                                   C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        L.ro_set_slot.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double]
        L.ro_replica_energy.argtypes = [C.c_void_p, C.c_int]
        L.ro_replica_energy.restype = C.c_double
        L.ro_merge.argtypes = [C.c_void_p, dp, dp]
        L.ro_merge_fragments.argtypes = [dp, ip, C.c_int, C.c_int, C.c_int, C.c_int, dp, ip]
        L.ro_thermo.argtypes = [dp, dp, C.c_int, C.c_double, dp, C.c_int, dp, dp, dp]
        L.ro_peak.argtypes = [dp, dp, C.c_int]
        L.ro_peak.restype = C.c_double
        _lib = L
    return _lib


# ---------------------------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().ro_philox4x32_10(c, k, out)
    return out


def draw_direction(slot, key1, t, purpose=1):
    S = np.zeros(3)
    lib().ro_draw_direction(int(slot), int(key1), int(t), int(purpose), S)
    return S


def u53(a, b):
    return lib().ro_u53(int(a), int(b))


def exp(x):
    return lib().ro_exp(float(x))


def bcc_offsets(n_shells):
    d = [np.zeros(64, dtype=np.int32) for _ in range(4)]
    z = lib().ro_bcc_offsets(n_shells, *d)
    if z < 0:
        raise ValueError("n_shells must be 1..4")
    return np.stack([d[0][:z], d[1][:z], d[2][:z]], axis=1), d[3][:z].copy()


def bcc_ground_state(L, J):
    J = np.zeros(4) if J is None else np.asarray(list(J) + [0.0] * (4 - len(J)), dtype=np.float64)
    n_shells = int(np.max(np.nonzero(J)[0]) + 1) if np.any(J) else 1
    return lib().ro_bcc_ground_state(L, n_shells, np.ascontiguousarray(J))


def bcc_ground_state_shells(L, n_shells, J):
    J = np.asarray(list(J) + [0.0] * (4 - len(J)), dtype=np.float64)
    return lib().ro_bcc_ground_state(L, n_shells, np.ascontiguousarray(J))


def window_layout(n_bins, n_windows, overlap):
    starts = np.zeros(max(n_windows, 1), dtype=np.int32)
    W = lib().ro_window_layout(n_bins, n_windows, overlap, starts)
    if W < 0:
        raise ValueError("invalid window layout")
    return W, starts[:n_windows].copy()


def sum32(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().ro_sum32(x, x.size)


def merge_fragments(frag, starts, B):
    frag = np.ascontiguousarray(frag, dtype=np.float64)
    h, m, W = frag.shape
    starts = np.ascontiguousarray(starts, dtype=np.int32)
    out = np.zeros(B, dtype=np.float64)
    bstar = np.zeros(max(h - 1, 1), dtype=np.int32)
    rc = lib().ro_merge_fragments(frag.reshape(-1), starts, h, m, W, B, out, bstar)
    return out, bstar[: h - 1].copy(), rc


def thermo(lng, centres, n_spins, T):
    lng = np.ascontiguousarray(lng, dtype=np.float64)
    centres = np.ascontiguousarray(centres, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    U = np.zeros(T.size)
    Cv = np.zeros(T.size)
    lnZ = np.zeros(T.size)
    lib().ro_thermo(lng, centres, lng.size, float(n_spins), T, T.size, U, Cv, lnZ)
    return U, Cv, lnZ


def peak(T, Cv):
    T = np.ascontiguousarray(T, dtype=np.float64)
    Cv = np.ascontiguousarray(Cv, dtype=np.float64)
    return lib().ro_peak(T, Cv, T.size)


# ---------------------------------------------------------------------------------------------
# simulation
# ---------------------------------------------------------------------------------------------
BCC, CHAIN, TABLE = 0, 1, 2


class OracleREWL:
    """One REWL simulation (all windows and walkers) held by the C oracle."""

    def __init__(self, kind=BCC, L=4, J=(1.0, 0.5), n_shells=None, nbr=None, Jt=None,
                 e_min=math.nan, e_max=math.nan, n_bins=200, n_windows=4, walkers_per_window=2,
                 overlap=0.75, flatness=0.8, lnf_final=1e-3, lnf_initial=1.0, seed=1,
                 exchange_interval=10000, group_size=1, init_max_moves=1 << 40, iteration=0):
        p = _Params()
        p.kind = kind
        p.L = L
        J = list(J)
        if n_shells is None:
            n_shells = len(J)
        p.n_shells = n_shells
        for i in range(4):
            p.J[i] = J[i] if i < len(J) else 0.0
        self._keep = []
        if kind == TABLE:
            nbr = np.ascontiguousarray(nbr, dtype=np.int32)
            Jt = np.ascontiguousarray(Jt, dtype=np.float64)
            p.z, p.n_sites = nbr.shape
            p.nbr = nbr.ctypes.data_as(C.POINTER(C.c_int32))
            p.Jt = Jt.ctypes.data_as(C.POINTER(C.c_double))
            self._keep += [nbr, Jt]
        p.e_min = e_min
        p.e_max = e_max
        p.n_bins = n_bins
        p.n_windows = n_windows
        p.walkers_per_window = walkers_per_window
        p.overlap = overlap
        p.flatness = flatness
        p.lnf_final = lnf_final
        p.lnf_initial = lnf_initial
        p.seed = seed
        p.exchange_interval = exchange_interval
        p.group_size = group_size
        p.iteration = iteration
        p.init_max_moves = init_max_moves
        h = C.c_void_p()
        err = C.create_string_buffer(256)
        rc = lib().ro_create(C.byref(p), C.byref(h), err, 256)
        if rc != 0:
            raise ValueError(err.value.decode())
        self._h = h
        vals = [C.c_int32() for _ in range(7)]
        lib().ro_sizes(h, *[C.byref(v) for v in vals])
        self.N, self.z, self.n_slots, self.W, self.B, self.h, self.m = [v.value for v in vals]
        g = [C.c_double() for _ in range(3)]
        lib().ro_energy_grid(h, *[C.byref(v) for v in g])
        self.e_min, self.e_max, self.dE = [v.value for v in g]
        self.starts = np.zeros(self.h, dtype=np.int32)
        lib().ro_window_starts(h, self.starts)
        self.exchange_interval = exchange_interval

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ro_destroy(self._h)
            self._h = None

    def init_walkers(self):
        if lib().ro_init_walkers(self._h) != 0:
            raise RuntimeError("initial drive did not reach every window")

    def run_intervals(self, n):
        lib().ro_run_intervals(self._h, int(n))

    def run_moves_only(self, moves_per_walker):
        lib().ro_run_moves_only(self._h, int(moves_per_walker))

    def exchange(self):
        lib().ro_exchange(self._h)

    def flatness(self):
        return lib().ro_flatness(self._h)

    def neighbours(self):
        nbr = np.zeros((self.z, self.N), dtype=np.int32)
        J = np.zeros((self.z, self.N), dtype=np.float64)
        lib().ro_neighbours(self._h, nbr, J)
        return nbr, J

    def initial_energy(self):
        return lib().ro_initial_energy(self._h)

    def walkers(self):
        S, W = self.n_slots, self.W
        out = dict(lng=np.zeros((S, W)), H=np.zeros((S, W), dtype=np.uint32), E=np.zeros(S),
                   bin=np.zeros(S, dtype=np.int32), lnf=np.zeros(S), replica=np.zeros(S, dtype=np.int32),
                   accepts=np.zeros(S, dtype=np.int64), stage=np.zeros(S, dtype=np.int32),
                   steps=np.zeros(S, dtype=np.int64), init_moves=np.zeros(S, dtype=np.int64))
        lib().ro_get_walkers(self._h, out["lng"], out["H"], out["E"], out["bin"], out["lnf"],
                             out["replica"], out["accepts"], out["stage"], out["steps"], out["init_moves"])
        return out

    def spins(self):
        sp = np.zeros((self.n_slots, 3, self.N))
        lib().ro_get_spins(self._h, sp)
        return sp

    def exchange_counts(self):
        n = max(self.h - 1, 1)
        a = np.zeros(n, dtype=np.int64)
        b = np.zeros(n, dtype=np.int64)
        lib().ro_get_exchange_counts(self._h, a, b)
        return a[: self.h - 1], b[: self.h - 1]

    def round_trips(self):
        """(round trips completed [S], extreme window seen last [S]: -1 none, 0 lowest, 1 highest)
        per replica."""
        c = np.zeros(self.n_slots, dtype=np.int64)
        last = np.zeros(self.n_slots, dtype=np.int32)
        lib().ro_get_round_trips(self._h, c, last)
        return c, last

    def max_drift(self):
        return lib().ro_max_drift(self._h)

    def exchange_index(self):
        return lib().ro_exchange_index(self._h)

    def replica_energy(self, r):
        return lib().ro_replica_energy(self._h, int(r))

    def draw_site(self, slot, t, purpose=0):
        site = C.c_int32()
        u = C.c_double()
        lib().ro_draw_site(self._h, slot, t, purpose, C.byref(site), C.byref(u))
        return site.value, u.value

    def set_slot(self, slot, lng=None, H=None, E=math.nan):
        lp = None if lng is None else np.ascontiguousarray(lng, dtype=np.float64)
        hp = None if H is None else np.ascontiguousarray(H, dtype=np.uint32)
        lib().ro_set_slot(self._h, int(slot), None if lp is None else lp.ctypes.data,
                          None if hp is None else hp.ctypes.data, float(E))

    def set_lng(self, lng0, lnf0):
        lib().ro_set_lng(self._h, np.ascontiguousarray(lng0, dtype=np.float64), float(lnf0))

    def merge(self):
        out = np.zeros(self.B)
        cen = np.zeros(self.B)
        lib().ro_merge(self._h, out, cen)
        return out, cen

    def centres(self):
        return self.e_min + (np.arange(self.B) + 0.5) * self.dE

    def all_done(self, lnf_final):
        return bool(np.all(self.walkers()["lnf"] < lnf_final))
