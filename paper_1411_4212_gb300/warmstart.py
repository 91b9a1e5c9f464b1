"""Learned warm start, end to end, on the library's public API: REWL runs that converge produce
ln g curves over random coupling sets; the MLP is trained on them by the library's kernels; a
held-out job starts from the predicted ln g at a small ln f0 and plain Wang-Landau finishes it.
This module only sequences library calls (every sampling, training and inference step runs on
the GPU); the numbers it compares are the jobs' own outputs.

Runs use a restricted energy range [0.6 E_gs, 0] with one bin per spin, so that the bin width stays
near the microcanonical temperature at the lower edge and every run converges in seconds (over
[E_gs, 0] with N/4 bins the lowest window does not converge at any speed: the bins there are far
wider than the temperature).
"""
import numpy as np

from . import REWL, Batch, Mlp, BCC, PRODUCTION, mlp_features
from . import workloads

WINDOWS = {4: 4, 5: 6, 6: 8, 7: 12, 8: 16}
WINDOW_BINS = 216   # window width of the L = 8 layout, kept for larger lattices


def windows_for(L, overlap=0.75):
    """Window count of the restricted range at bcc L: the table above up to L = 8, beyond it as many
    windows as keep each about WINDOW_BINS wide (h from W = B / (1 + (h - 1)(1 - overlap)))."""
    if L in WINDOWS:
        return WINDOWS[L]
    N = 2 * L ** 3
    return max(2, int(round(1 + (N / WINDOW_BINS - 1) / (1 - overlap))))
# input normalisation x' = (x - SHIFT) * SCALE of (E/N, 1/L, J1, J2, J3, J4)
SHIFT = np.array([-1.9, 0.19, 1.0, 0.4, 0.0, 0.0], dtype=np.float32)
SCALE = np.array([1 / 1.1, 20.0, 1.0, 5.0, 10.0, 1.0], dtype=np.float32)
LNF0_WARM = 2.0 ** -7


def ground_state(L, J):
    """E_gs of the couplings (Luttinger-Tisza, computed by the library at creation)."""
    p = REWL(kind=BCC, L=L, J=J, n_bins=16, n_windows=1, walkers_per_window=1, group_size=1)
    e = p.info()["e_min"]
    p.close()
    return e


def restricted_job(L, J, seed, lnf_final, walkers=2, exchange_interval=4000, stream=None):
    N = 2 * L ** 3
    return REWL(kind=BCC, mode=PRODUCTION, L=L, J=J, e_min=0.6 * ground_state(L, J), e_max=0.0, n_bins=N,
                n_windows=windows_for(L), walkers_per_window=walkers, overlap=0.75, flatness=0.8, lnf_final=lnf_final,
                seed=seed, exchange_interval=exchange_interval, group_size=1, stream=stream)


def converge(jobs, max_intervals=400000, check_every=8, autotune=True):
    """Run jobs together until all converge; returns True if they did."""
    with Batch(jobs) as b:
        if autotune and len(jobs) > 1:
            b.autotune(trial_moves=200)
        ok, _ = b.run_to_convergence(max_intervals=max_intervals, check_every=check_every)
    return ok


def corpus(sizes=(4, 5, 6), per_size=64, lnf_final=1e-4, seed0=0, shells=3, max_samples=None):
    """Converged ln g curves over random couplings: (x [M][6], ln g/N [M], run offsets [R+1], meta).
    shells = 4 draws a fourth coupling too (workloads.random_couplings4).  max_samples keeps every
    k-th bin of a run so that it contributes at most that many samples (the curves are smooth on the
    scale of a few bins)."""
    draw = workloads.random_couplings4 if shells == 4 else workloads.random_couplings
    jobs, meta = [], []
    k = seed0
    for L in sizes:
        for _ in range(per_size):
            J = draw(k)
            jobs.append(restricted_job(L, J, seed=5000 + k, lnf_final=lnf_final))
            meta.append((L, J))
            k += 1
    ok = converge(jobs)
    xs, ts = [], []
    for j in jobs:
        lng, _ = j.merge()
        x, t = mlp_features(j, lng)
        if max_samples is not None and len(t) > max_samples:
            step = -(-len(t) // max_samples)
            x, t = x[::step], t[::step]
        xs.append(x)
        ts.append(t)
        j.close()
    off = np.cumsum([0] + [len(t) for t in ts]).astype(np.int32)
    return np.concatenate(xs), np.concatenate(ts), off, dict(converged=ok, runs=meta)


def train(x, t, off, steps=2000, lr=2e-3, seed=0, stream=None):
    net = Mlp(SHIFT, SCALE, seed=seed, stream=stream)
    hist = net.train(x, t, off, steps=steps, lr=lr)
    return net, hist


def centred_rms(a, b):
    d = np.asarray(a) - np.asarray(b)
    return float(np.sqrt(np.mean((d - d.mean()) ** 2)))


def warm_vs_cold(net, L, couplings, lnf_final=1e-5, replicas=2, lnf0=LNF0_WARM, seed0=900, separate=False,
                 autotune=False, n_ref=0, lnf_ref=None):
    """For every coupling set: `replicas` cold starts (ln g = 0, ln f0 = 1) and `replicas` warm starts
    (network ln g, ln f0).  Returns (converged, per-set records, wall seconds).  Records hold the moves
    per walker to converge and the centred rms of each converged ln g against the first cold
    replica; a job's walkers all walk until the whole job has converged, so its moves per walker are
    the job's time to converge.  separate=False converges all jobs in one batch (wall = None);
    separate=True converges the cold jobs, then the warm jobs (network inference included), in two
    timed batches: wall = (cold seconds, warm seconds).  autotune=True lets each batch's autotuner
    pick its launch shape first (its trial moves are ordinary moves of the jobs).  n_ref > 0 judges every
    cold and warm run against an independent reference instead: the mean of n_ref further cold runs
    converged to lnf_ref (run first, in a batch of their own); cold_rms then has all replicas."""
    import time
    cold, warm, pred, refs = [], [], [], []
    s = seed0
    for J in couplings:
        cold.append([restricted_job(L, J, seed=s + r, lnf_final=lnf_final) for r in range(replicas)])
        warm.append([restricted_job(L, J, seed=s + 100 + r, lnf_final=lnf_final) for r in range(replicas)])
        refs.append([restricted_job(L, J, seed=s + 200 + r, lnf_final=lnf_ref) for r in range(n_ref)])
        s += 1000
    ref_curves = []
    if n_ref > 0:
        flat_ref = [j for group in refs for j in group]
        converge(flat_ref, autotune=autotune)
        for group in refs:
            ref_curves.append(reference_curve([j.merge()[0] for j in group]))
            for j in group:
                j.close()
    for group in cold + warm:
        for j in group:
            j.init_walkers()

    def start_warm():
        for ws in warm:
            for w in ws:
                p = net.warm_start(w, lnf0)
            pred.append(p)

    flat_cold = [j for group in cold for j in group]
    flat_warm = [j for group in warm for j in group]
    if separate:
        t0 = time.perf_counter()
        ok = converge(flat_cold, autotune=autotune)
        t1 = time.perf_counter()
        start_warm()
        ok = converge(flat_warm, autotune=autotune) and ok
        t2 = time.perf_counter()
        wall = (t1 - t0, t2 - t1)
    else:
        start_warm()
        ok = converge(flat_cold + flat_warm, autotune=autotune)
        wall = None
    out = []
    for i, (J, cs, ws, p) in enumerate(zip(couplings, cold, warm, pred)):
        ref = ref_curves[i] if n_ref > 0 else cs[0].merge()[0]
        rec = dict(J=J, cold_moves=[], warm_moves=[], cold_rms=[], warm_rms=[],
                   prediction_rms=centred_rms(p, ref))
        for j in cs:
            rec["cold_moves"].append(float(j.walkers()["steps"].mean()))
        for j in (cs if n_ref > 0 else cs[1:]):
            rec["cold_rms"].append(centred_rms(j.merge()[0], ref))
        for j in ws:
            rec["warm_moves"].append(float(j.walkers()["steps"].mean()))
            rec["warm_rms"].append(centred_rms(j.merge()[0], ref))
        out.append(rec)
        for j in cs + ws:
            j.close()
    return ok, out, wall


def target_job(spec, seed, lnf_final, stream=None):
    """The bcc L = 32 four-shell run on its range around the specific-heat peak (workloads.TARGET_L32):
    bins of spec["bin_width"], windows of about spec["window_bins"] bins."""
    L = spec["L"]
    N = 2 * L ** 3
    lo, hi = spec["e_per_spin"]
    B = int(round((hi - lo) * N / spec["bin_width"]))
    h = max(2, int(round(1 + (B / spec["window_bins"] - 1) / (1 - spec["overlap"]))))
    return REWL(kind=BCC, mode=PRODUCTION, L=L, J=spec["J"], e_min=lo * N, e_max=hi * N, n_bins=B, n_windows=h,
                walkers_per_window=spec["walkers_per_window"], overlap=spec["overlap"], flatness=spec["flatness"],
                lnf_final=lnf_final, seed=seed, exchange_interval=spec["exchange_interval"], group_size=1,
                stream=stream)


def converge_alone(job, check_every=16, max_intervals=2_000_000, autotune=True):
    """Converge one (initialised) job on the GPU by itself (a batch of one: graph replays, the job
    leaves when every walker has ln f < ln f_final), its launch shape autotuned first (ordinary moves,
    counted); returns (converged, wall seconds, trial moves per walker)."""
    import time
    t0 = time.perf_counter()
    with Batch([job]) as b:
        if autotune:
            b.autotune(trial_moves=2000)
        ok, _ = b.run_to_convergence(max_intervals=max_intervals, check_every=check_every)
    wall = time.perf_counter() - t0
    return ok, wall, float(job.walkers()["steps"].mean())


def reference_curve(curves):
    """Mean of centred ln g curves (an estimate of ln g with the runs' noise averaged down)."""
    c = np.array([np.asarray(x) - np.mean(x) for x in curves])
    return c.mean(0)


def paired_excess(a, b):
    """Mean and standard error of a - b over paired samples."""
    d = np.asarray(a, dtype=float) - np.asarray(b, dtype=float)
    se = float(d.std(ddof=1) / np.sqrt(len(d))) if len(d) > 1 else float("inf")
    return float(d.mean()), se


def first_iteration_job(L, J, seed, window_bins=64, overlap=0.75, exchange_interval=4000, serial=False):
    """The first Wang-Landau iteration (ln f 1 -> 1/2) as a job that converges at ln f < 0.9: the
    restricted range with one bin per spin, windows of about `window_bins` bins at `overlap`, their
    number growing with the lattice (the paper's weak-scaling set-up, Sec. 5, Fig. 3), one walker per
    window; serial=True puts one walker over the whole range instead."""
    N = 2 * L ** 3
    h = 1 if serial else max(2, int(round(1 + (N / window_bins - 1) / (1 - overlap))))
    return REWL(kind=BCC, mode=PRODUCTION, L=L, J=J, e_min=0.6 * ground_state(L, J), e_max=0.0, n_bins=N,
                n_windows=h, walkers_per_window=1, overlap=overlap if h > 1 else 0.0, flatness=0.8,
                lnf_final=0.9, seed=seed, exchange_interval=exchange_interval, group_size=1)
