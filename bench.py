"""Benchmark: spin-move attempts/s of replica-exchange Wang-Landau on one GB300.

Default workload (the paper's method on the large configuration): classical Heisenberg model on bcc
L=32 (65536 spins, periodic), four coupling shells J=(1, 0.6, -0.05, -0.1) (8+6+12+24 = 50
neighbours), energy range [E_gs, 0] in 8000 bins, 64 windows x 8 walkers at 75 % overlap, flatness
0.8, ln f 1 -> 1e-8, exchange every 1e4 moves; production mode (FP32 spins and dE, 64-bit
fixed-point ln g and energy).  Synthetic: the state is the sampler's own, started from the aligned
configuration and driven into the windows (untimed).  --workload cfg2 runs bcc L=16 with two shells,
16 windows x 4 walkers and 2000 bins instead.

One step = `intervals` exchange intervals, each = walker kernel (1e4 trial moves per walker,
energy recomputation every 8th) + replica-exchange kernel + flatness kernel, then the merge kernels
(all steps of the hot path).  The L2 cache is flushed (256 MB write) between timed steps; the bcc L=32
lattices alone hold 537 MB.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]

With N > 1 (torchrun) every rank runs an independent replica of the workload with its own seed
(weak scaling, no data-path collective); rank 0 prints the aggregate.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LARGE = dict(L=32, J=(1.0, 0.6, -0.05, -0.1), n_bins=8000, n_windows=64, walkers_per_window=8, overlap=0.75,
             flatness=0.8, lnf_final=1e-8, exchange_interval=10000)
LARGE_NAME = ("REWL bcc L=32 (65536 spins) J=(1,0.6,-0.05,-0.1) (50 neighbours), [E_gs,0] 8000 bins, "
              "64 windows x 8 walkers, 75% overlap, exchange every 1e4 moves")
CFG2 = dict(L=16, J=(1.0, 0.5), n_bins=2000, n_windows=16, walkers_per_window=4, overlap=0.75,
            flatness=0.8, lnf_final=1e-8, exchange_interval=10000)
CFG2_NAME = ("REWL bcc L=16 (8192 spins) J1=1 J2=0.5, [E_gs,0] 2000 bins, 16 windows x 4 walkers, "
             "75% overlap, exchange every 1e4 moves")
# workload -> (configuration, name, walkers per window of the bounded CPU sample)
WORKLOADS = {"large": (LARGE, LARGE_NAME, 1), "cfg2": (CFG2, CFG2_NAME, 4)}
METRIC = "spin-move attempts/s"
UNIT = "moves/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--intervals", type=int, default=20, help="exchange intervals per step")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--warm-l", type=int, default=12,
                   help="warmstart: bcc L of the held-out evaluation jobs (windows about 216 bins wide)")
    p.add_argument("--jobs-per-size", type=int, default=16,
                   help="batch64: jobs per lattice size (16 gives the 64-job workload; smaller for profiling)")
    p.add_argument("--workload", default="large",
                   choices=["large", "cfg2", "batch64", "warmstart", "weak-scaling", "target"],
                   help="large: one job, bcc L=32 with four shells, 64 windows x 8 walkers (the headline "
                        "line); cfg2: one job, bcc L=16 with two shells, 16 windows x 4 walkers; batch64: 64 "
                        "jobs of bcc L=8..20 in one persistent launch; warmstart: learned warm start versus "
                        "plain REWL; weak-scaling: moves to finish the first WL iteration versus L; target: "
                        "bcc L=32 four-shell couplings converged, warm start against plain")
    p.add_argument("--ws-sizes", default="4,6,8,10,16,20,30,40,50",
                   help="weak-scaling: bcc L of the windowed jobs (the paper's Fig. 3 covers L = 10..50)")
    p.add_argument("--target-lnf", type=float, default=1e-6, help="target: ln f_final of the plain and warm runs")
    p.add_argument("--target-replicas", type=int, default=2, help="target: plain and warm runs each")
    p.add_argument("--target-refs", type=int, default=1, help="target: reference runs (ln f_final / 10)")
    p.add_argument("--target-seed-offset", type=int, default=0,
                   help="target: first seed of the plain and warm runs past 8000 / 9000 (new runs against the "
                        "same reference)")
    p.add_argument("--corpus-per-size", type=int, default=64, help="target: corpus runs per lattice size")
    p.add_argument("--mlp-cache", default=None,
                   help="target: .npz of the trained network; read when it exists (no corpus, no training), "
                        "else written after training")
    return p.parse_args()


# ------------------------------------------------------------------------------------------------
# distributed plumbing (barrier + max over ranks)
# ------------------------------------------------------------------------------------------------
def dist_init(n):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def replica_seed(rank):
    """Every rank runs its own replica of the workload (weak scaling, no data-path collective)."""
    return 1 + rank


def aggregate_rate(units_per_rank, world, max_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (max_ms * 1e-3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def all_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def wait_first(self, timeout=10.0):
        """Block until nvidia-smi has printed its first sample, so the timed region is covered."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.02)
        self.lines.clear()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands on the host cores
# ------------------------------------------------------------------------------------------------
def cpu_sample(workload):
    """The bounded CPU sample of a workload: its lattice, couplings, bins and window layout, with
    `sample_m` walkers per window instead of all of them (moves/s per walker do not depend on m)."""
    cfg, name, sample_m = WORKLOADS[workload]
    return dict(cfg, walkers_per_window=sample_m), name


def oracle_interval(s, cfg):
    """One exchange interval of the oracle as it stands, the steps of the hot path: Wang-Landau moves of
    every walker, one replica-exchange round, the flatness test.  (The oracle's own interval also
    recomputes every walker's energy from scratch as a drift check, which changes no state; at z = 50
    it costs three times the moves, so it is left out here.)"""
    s.run_moves_only(cfg["exchange_interval"])
    s.exchange()
    s.flatness()
    return s.n_slots * cfg["exchange_interval"]


def _oracle_replica(workload, seed):
    import oracle
    cfg, _ = cpu_sample(workload)
    s = oracle.OracleREWL(kind=oracle.BCC, seed=seed, **cfg)
    s.init_walkers()
    return s, cfg


def _oracle_rate_worker(args):
    seconds, seed, workload = args
    s, cfg = _oracle_replica(workload, seed)
    moves = n = 0
    t0 = time.perf_counter()
    while n < 1 or time.perf_counter() - t0 < seconds:
        moves += oracle_interval(s, cfg)
        n += 1
    dt = time.perf_counter() - t0
    return moves / dt, moves, dt, n


def host_cores():
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    return max(1, min(cores, 64))


def cpu_baseline(seconds, workload):
    """The single-threaded oracle as it stands, one independent replica of the bounded sample (own seed)
    per host core, in spawned processes; the value is the replicas' aggregate rate."""
    import multiprocessing as mp
    cores = host_cores()
    cfg, _ = cpu_sample(workload)
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_rate_worker, [(seconds, 1 + i, workload) for i in range(cores)])
    rate = sum(r[0] for r in res)
    moves = sum(r[1] for r in res)
    n = sum(r[3] for r in res)
    dt = max(r[2] for r in res)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_value": res[0][0],
            "sample": f"{cores} independent replicas, one per core, of the same lattice, couplings, bins and "
                      f"{cfg['n_windows']} windows with {cfg['walkers_per_window']} walker(s) per window; {n} exchange "
                      f"intervals in all ({moves} trial moves with the exchange rounds and flatness tests) in "
                      f"{dt:.1f} s, FP64"}


# ------------------------------------------------------------------------------------------------
# reference arm: the oracle timed as it stands, step by step
# ------------------------------------------------------------------------------------------------
def _reference_worker(args):
    steps, warmup, seed, workload = args
    s, cfg = _oracle_replica(workload, seed)
    for _ in range(warmup):
        oracle_interval(s, cfg)
    moves = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        moves += oracle_interval(s, cfg)
    return moves, time.perf_counter() - t0


def run_reference(args):
    """The FP64 oracle as it stands, one independent replica of the bounded sample per host core
    (spawned processes); a step is one exchange interval of every replica."""
    import multiprocessing as mp
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm covers the single-job workloads "
                                                              f"({', '.join(WORKLOADS)}), not {args.workload}"}))
        return 0
    cores = host_cores()
    cfg, name = cpu_sample(args.workload)
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_reference_worker, [(args.steps, args.warmup, 1 + i, args.workload) for i in range(cores)])
    moves = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    value = moves / dt
    sample = (f"{args.steps} exchange intervals of {cores} independent replicas, one per host core, each with the "
              f"lattice, couplings, bins and {cfg['n_windows']} windows of the workload and {cfg['walkers_per_window']} "
              f"walker(s) per window ({moves} moves in all)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name,
                   "step": f"one exchange interval (moves, exchange round, flatness test) of each of {cores} FP64 "
                           "oracle replicas, one per host core"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
# DRAM traffic of the walker kernel, taken from the committed ncu summary of the same kernel (the
# summary under profiles/ whose `kernel` field names it).  The summary records a hash of the
# kernel's sources (code only, without comments); once the code changes the figure no longer applies
# and the traffic is reported as null.
PROFILES = os.path.join(ROOT, "profiles")
KERNEL_SOURCES = ["walker_pipe.cu", "walker_common.cuh", "device_common.cuh", "rewl_types.h"]


def _code_only(text):
    """C++ source without comments and with whitespace runs collapsed: what the compiler sees."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"' or c == "'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash():
    """Hash of the walker kernel's sources, comments and layout excluded."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1411_4212_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()


def profile_fields(path):
    fields = {}
    for line in open(path):
        if line.startswith("- ") and ": " in line:
            k, v = line[2:].split(": ", 1)
            fields[k.strip()] = v.strip().strip("`")
    return fields


def profiled_traffic(kernel, moves_per_launch):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch, scaled from the profiled launch."""
    if not os.path.isdir(PROFILES):
        return None
    for name in sorted(os.listdir(PROFILES)):
        if not name.endswith(".md"):
            continue
        fields = profile_fields(os.path.join(PROFILES, name))
        if fields.get("kernel") != kernel:
            continue
        try:
            if fields["source_sha256"] != kernel_source_hash():
                return None
            return float(fields["dram_bytes_per_launch"]) * moves_per_launch / float(fields["moves_per_launch"])
        except (KeyError, ValueError):
            return None
    return None


def hbm_peak():
    """Measured HBM copy bandwidth of this machine's GPUs (bytes/s) and where it comes from."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]) * 1e9, "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"
    except (OSError, KeyError, ValueError):
        return 6.8e12, "fallback 6.8 TB/s (no measured peak file)"


def run_batch64(args):
    """64 independent jobs (16 per bcc L in 8, 12, 16, 20; random three-shell couplings; N/4 bins over
    [E_gs, 0]; 8..32 windows x 4 walkers) in one persistent walker launch per interval, replayed
    from a CUDA graph after the autotuner picked walkers per block and lattice placement."""
    import torch
    import paper_1411_4212_gb300 as rw
    from paper_1411_4212_gb300 import workloads

    rank, world, local = dist_init(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    I = args.intervals
    specs = workloads.batch64_jobs(jobs_per_size=args.jobs_per_size)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        jobs = [rw.REWL(kind=rw.BCC, mode=rw.PRODUCTION, group_size=1, stream=stream,
                        **dict(s, seed=s["seed"] + 100000 * (replica_seed(rank) - 1))) for s in specs]
        batch = rw.Batch(jobs, stream=stream)
    setup_s = time.perf_counter() - t0
    tune = batch.autotune(trial_moves=2000)
    S = sum(j.n_slots for j in jobs)
    moves_per_step = S * specs[0]["exchange_interval"] * I
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    batch.run_intervals(max(3, args.warmup))
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first()
    barrier(world)
    step_ms = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.run_intervals(I)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    total_ms = all_max(sum(step_ms), world)
    value = aggregate_rate(moves_per_step * args.steps, world, total_ms)
    info = batch.info()

    # end to end through the public API with host buffers: every job's ln g in (a warm start at
    # ln f = 1), the batch's intervals, every job's merged ln g out
    lng_in = [np.zeros(j.B) for j in jobs]
    h2d = sum(j.n_slots * j.W * 8 + 2 * j.n_slots * 8 for j in jobs)
    d2h = sum(j.B * 8 for j in jobs)
    e2e_ms = []
    for k in range(max(2, args.steps)):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j, lng in zip(jobs, lng_in):
            j.set_initial_lng(lng, 1.0)
        batch.run_intervals(I)
        for j in jobs:
            j.merge()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total = all_max(sum(e2e_ms), world)
    e2e_value = moves_per_step * len(e2e_ms) * world / (e2e_total * 1e-3)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32 spins/dE + int64 fixed-point ln g/energy",
            "data": "synthetic",
            "config": {"workload": f"{len(specs)} REWL jobs, bcc L in {{8,12,16,20}} x {args.jobs_per_size}, "
                                   "J1=1 J2~U[0.2,0.6] J3~U[-0.1,0.1], "
                                   "N/4 bins over [E_gs,0], 8/16/24/32 windows x 4 walkers, exchange every 1e4 moves",
                       "walker_slots": S, "intervals_per_step": I, "moves_per_step": moves_per_step * world,
                       "l2": "flushed between steps (256 MB write)", "graph": True,
                       "tuning": tune, "batch": info, "setup_s": setup_s},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * I * 3,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    batch.close()
    for j in jobs:
        j.close()
    return 0


def run_warmstart(args):
    """Time to converged ln g with and without the learned warm start.  Corpus: 192 converged REWL
    runs (bcc L = 4, 5, 6 x 64 random three-shell coupling sets, ln f -> 1e-4) on the restricted
    range [0.6 E_gs, 0] with one bin per spin; the network is trained on them by the library's
    kernels; evaluation: 4 held-out coupling sets at bcc L = --warm-l (default 12: 3456 spins, 61
    windows x 2 walkers, ln f -> 1e-5), 2 cold and 2 warm replicas each, cold and warm converged in
    separate timed batches, each autotuned first."""
    import numpy as np
    import torch
    from paper_1411_4212_gb300 import warmstart, workloads
    rank, world, local = dist_init(args.gpus)
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    x, t, off, meta = warmstart.corpus(sizes=(4, 5, 6), per_size=64, lnf_final=1e-4)
    t1 = time.perf_counter()
    net, hist = warmstart.train(x, t, off, steps=4000, lr=2e-3)
    t2 = time.perf_counter()
    held = [workloads.random_couplings(20_000 + i) for i in range(4)]
    L = args.warm_l
    ok, res, wall = warmstart.warm_vs_cold(net, L, held, lnf_final=1e-5, replicas=2, separate=True, autotune=True)
    probe = warmstart.restricted_job(L, held[0], seed=1, lnf_final=1e-5)
    h, W = probe.h, probe.W
    probe.close()
    cold = float(np.mean([m for r in res for m in r["cold_moves"]]))
    warm = float(np.mean([m for r in res for m in r["warm_moves"]]))
    # Monte Carlo time: trial moves per walker until a job has converged, averaged over the jobs.
    # The wall time of each group is that of its slowest job (all run in one batch), so it is
    # reported beside it but is not the comparison.
    line = {
        "metric": "Monte Carlo time (moves per walker) to converged ln g, warm start / plain", "value": warm / cold,
        "unit": "ratio", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
        "config": {"workload": f"warm start: corpus 192 runs bcc L=4,5,6 (ln f->1e-4), evaluation 4 held-out "
                               f"coupling sets at bcc L={L}, {h} windows x 2 walkers ({W} bins each), ln f->1e-5, "
                               "range [0.6 E_gs, 0], one bin per spin, ln f0 = 2^-7 (warm) vs 1 (plain)",
                   "converged": bool(ok and meta["converged"])},
        "wall_s": {"plain": wall[0], "warm": wall[1], "ratio": wall[1] / wall[0], "corpus": t1 - t0,
                   "training": t2 - t1, "note": "each group's slowest job of 8"},
        "moves_per_walker": {"plain": cold, "warm": warm, "ratio": warm / cold},
        "rms": {"prediction": float(np.mean([r["prediction_rms"] for r in res])),
                "plain_vs_plain": float(np.mean([v for r in res for v in r["cold_rms"]])),
                "warm_vs_plain": float(np.mean([v for r in res for v in r["warm_rms"]]))},
        "training": {"samples": int(len(t)), "runs": int(len(off) - 1), "steps": 4000,
                     "loss_first": float(hist[0]), "loss_last": float(hist[-1])},
    }
    print(json.dumps(line), flush=True)
    net.close()
    return 0


def run_target(args):
    """The bcc L = 32 four-shell couplings converged to ln f_final, plain against the learned warm start,
    on the range around the specific-heat peak (workloads.TARGET_L32: E/N in [-2.50, -2.10], bins of
    1.6 J1, windows of about 216 bins x 2 walkers).  Corpus: converged runs of four-shell couplings at
    bcc L = 8, 12, 16, 20 (--corpus-per-size each, restricted range [0.6 E_gs, 0], one bin per spin,
    ln f -> 1e-4), the network trained on them by the library's kernels.  Each target run converges alone
    on the GPU.  Accuracy: centred rms of ln g against the mean of --target-refs further plain runs
    converged to ln f_final / 10, and the C(T) peak of every run."""
    import numpy as np
    import torch
    import paper_1411_4212_gb300 as rw
    from paper_1411_4212_gb300 import warmstart, workloads
    rank, world, local = dist_init(args.gpus)
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    spec = workloads.TARGET_L32
    lnf = args.target_lnf
    t0 = time.perf_counter()
    if args.mlp_cache and os.path.exists(args.mlp_cache):
        # a network trained by an earlier run of this leg (same corpus recipe)
        z = np.load(args.mlp_cache)
        net = rw.Mlp(warmstart.SHIFT, warmstart.SCALE)
        net.set_params(z["params"])
        t, off, hist, meta = z["targets"], z["offsets"], z["loss"], {"converged": bool(z["converged"])}
        t1 = t2 = time.perf_counter()
    else:
        x, t, off, meta = warmstart.corpus(sizes=(8, 12, 16, 20), per_size=args.corpus_per_size, lnf_final=1e-4,
                                           shells=4, max_samples=2048)
        t1 = time.perf_counter()
        net, hist = warmstart.train(x, t, off, steps=4000, lr=2e-3)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if args.mlp_cache:
            np.savez(args.mlp_cache, params=net.params(), targets=t, offsets=off, loss=hist,
                     converged=meta["converged"], corpus_s=t1 - t0, training_s=t2 - t1)
        print(json.dumps({"corpus_runs": int(len(off) - 1), "samples": int(len(t)), "corpus_s": t1 - t0,
                          "training_s": t2 - t1, "loss_first": float(hist[0]), "loss_last": float(hist[-1])}),
              file=sys.stderr, flush=True)
    T = np.linspace(1.2, 2.2, 2001)
    runs = []

    def one(kind, seed, lnf_final):
        job = warmstart.target_job(spec, seed=seed, lnf_final=lnf_final)
        job.init_walkers()
        pred = None
        tw = time.perf_counter()        # the warm run's time includes the network's inference
        if kind == "warm":
            pred = net.warm_start(job, warmstart.LNF0_WARM)
        ok, _, moves = warmstart.converge_alone(job)
        wall = time.perf_counter() - tw
        lng, cen = job.merge()
        _, Cv, _ = rw.thermo(lng, cen, job.N, T)
        rec = {"kind": kind, "seed": seed, "lnf_final": lnf_final, "converged": bool(ok), "wall_s": wall,
               "moves_per_walker": moves, "T_peak": rw.peak_temperature(T, Cv), "C_max": float(Cv.max()),
               "windows": job.h, "walkers": job.n_slots, "bins": job.B}
        print(json.dumps(rec), file=sys.stderr, flush=True)
        job.close()
        return rec, lng, pred

    refs = []
    for r in range(args.target_refs):
        rec, lng, _ = one("reference", 7000 + r, lnf / 10)
        runs.append(rec)
        refs.append(lng)
    ref = warmstart.reference_curve(refs)
    for r in range(args.target_replicas):
        for kind, s0 in (("plain", 8000 + args.target_seed_offset), ("warm", 9000 + args.target_seed_offset)):
            rec, lng, pred = one(kind, s0 + r, lnf)
            rec["rms_vs_reference"] = warmstart.centred_rms(lng, ref)
            if pred is not None:
                rec["prediction_rms_vs_reference"] = warmstart.centred_rms(pred, ref)
            runs.append(rec)
    plain = [r for r in runs if r["kind"] == "plain"]
    warm = [r for r in runs if r["kind"] == "warm"]
    mean = lambda rs, k: float(np.mean([r[k] for r in rs]))
    line = {
        "metric": "time to converged ln g(E), learned warm start / plain REWL (bcc L=32, 4 shells)",
        "value": mean(warm, "wall_s") / mean(plain, "wall_s"), "unit": "ratio", "higher_is_better": False,
        "n_gpus": 1, "data": "synthetic",
        "config": {"workload": f"bcc L=32 J=(1,0.6,-0.05,-0.1), E/N in [-2.50,-2.10], {runs[-1]['bins']} bins "
                               f"of 1.6 J1, {runs[-1]['windows']} windows x 2 walkers, ln f 1 -> {lnf:g} (plain) or "
                               f"2^-7 -> {lnf:g} (warm); corpus {len(off) - 1} runs bcc L=8..20, four shells",
                   "corpus_converged": bool(meta["converged"])},
        "moves_per_walker": {"plain": mean(plain, "moves_per_walker"), "warm": mean(warm, "moves_per_walker"),
                             "ratio": mean(warm, "moves_per_walker") / mean(plain, "moves_per_walker")},
        "wall_s": {"plain": mean(plain, "wall_s"), "warm": mean(warm, "wall_s"), "corpus": t1 - t0,
                   "training": t2 - t1},
        "rms_vs_reference": {"plain": mean(plain, "rms_vs_reference"), "warm": mean(warm, "rms_vs_reference")},
        "T_peak": {k: [r["T_peak"] for r in runs if r["kind"] == k] for k in ("reference", "plain", "warm")},
        "training": {"samples": int(len(t)), "runs": int(len(off) - 1), "loss_first": float(hist[0]),
                     "loss_last": float(hist[-1])},
        "runs": runs,
    }
    print(json.dumps(line), flush=True)
    net.close()
    return 0


def run_weak_scaling(args):
    """Trial moves per walker to finish the first Wang-Landau iteration versus lattice size (the
    paper's weak-scaling measure, Sec. 5, Fig. 3, over its L = 10..50 and smaller): windows of 64 bins
    at 75 % overlap, one walker each, their number growing with N (5 windows at bcc L = 4, 15622 at
    L = 50, 250 000 spins), against one serial walker over the same range (L <= 8).  Range
    [0.6 E_gs, 0] with one bin per spin, J = (1, 0.5).  All jobs run in one batch; each leaves the work
    list when its walkers have halved ln f once."""
    import numpy as np
    import torch
    import paper_1411_4212_gb300 as rw
    from paper_1411_4212_gb300 import warmstart
    rank, world, local = dist_init(args.gpus)
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    J = (1.0, 0.5)
    sizes = tuple(int(v) for v in args.ws_sizes.split(","))
    serial_sizes = tuple(L for L in (4, 6, 8) if L <= max(sizes))
    t0 = time.perf_counter()
    jobs = [warmstart.first_iteration_job(L, J, seed=100 + L) for L in sizes]
    jobs += [warmstart.first_iteration_job(L, J, seed=200 + L, serial=True) for L in serial_sizes]
    for j in jobs:
        j.init_walkers()
    torch.cuda.synchronize()
    t_init = time.perf_counter() - t0
    t0 = time.perf_counter()
    with rw.Batch(jobs) as b:
        ok, done = b.run_to_convergence(max_intervals=20000, check_every=4)
    wall = time.perf_counter() - t0
    rows = []
    for j, L in zip(jobs, list(sizes) + list(serial_sizes)):
        w = j.walkers()
        rows.append({"L": L, "N": 2 * L ** 3, "windows": j.h, "bins_per_window": j.W,
                     "moves_per_walker": float(w["steps"].mean()), "first_iteration_done": bool(np.all(w["stage"] >= 1)),
                     "serial": j.h == 1, "lattice_bytes": j.n_slots * 2 * L ** 3 * 8})
        j.close()
    rewl = [r for r in rows if not r["serial"]]
    line = {
        "metric": "trial moves per walker to finish the first WL iteration, largest / smallest lattice",
        "value": rewl[-1]["moves_per_walker"] / rewl[0]["moves_per_walker"], "unit": "ratio",
        "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
        "config": {"workload": f"weak scaling: bcc L={','.join(map(str, sizes))}, J=(1,0.5), range [0.6 E_gs, 0], "
                               "one bin per spin, windows of ~64 bins at 75% overlap (h grows with N), 1 walker per "
                               "window; serial: one walker over the whole range", "all_done": bool(ok),
                   "init_s": t_init, "wall_s": wall},
        "rows": rows,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch64(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "weak-scaling":
        return run_weak_scaling(args)
    if args.workload == "target":
        return run_target(args)
    import torch
    import paper_1411_4212_gb300 as rw

    rank, world, local = dist_init(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    I = args.intervals

    workload, workload_name, _ = WORKLOADS[args.workload]
    sim = rw.REWL(kind=rw.BCC, mode=rw.PRODUCTION, seed=replica_seed(rank), stream=stream, **workload)
    sim.init_walkers()
    # the conflict-table size is timed before the warm-up (ordinary moves)
    tune = sim.autotune(trial_moves=2000)
    S, B = sim.n_slots, sim.B
    moves_per_step = S * workload["exchange_interval"] * I
    out = torch.zeros(B, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(walk_events=None):
        for i in range(I):
            if walk_events is not None:
                walk_events[i][0].record(stream)
            sim.walk()
            if walk_events is not None:
                walk_events[i][1].record(stream)
            sim.exchange_async()
            sim.flatness()
        sim.merge_device(out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    c0 = sim.counters()

    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first()
    step_ms, walk_ms = [], []
    barrier(world)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(I)]
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        step(ev)
        s1.record(stream)
        s1.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        walk_ms.extend(a.elapsed_time(b) for a, b in ev)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    c1 = sim.counters()

    total_ms = all_max(sum(step_ms), world)
    value = aggregate_rate(moves_per_step * args.steps, world, total_ms)
    acc_rate = (c1["accepts"] - c0["accepts"]) / max(1, c1["moves"] - c0["moves"])
    rec_rate = (c1["recomputes"] - c0["recomputes"]) / max(1, c1["moves"] - c0["moves"])

    # roofline of the walker kernel: lattices in shared memory against the shared-memory bandwidth
    # of this GPU (neighbour spins, ln g and H, records); lattices in global memory against HBM
    # (the lattice bytes alone).  Algorithmic bytes per move as the hot path's scope defines them: a
    # spin is its three FP32 components, 12 B (the library stores it in an 8-byte code, so the
    # kernel itself moves less than this)
    z = sim.z
    walk_avg_ms = statistics.mean(walk_ms)
    walker_share = sum(walk_ms) / sum(step_ms)
    pipelined = bool(sim.info()["pipelined"])
    in_smem = "true" if sim.info()["lattice_in_shared"] else "false"
    if in_smem == "true":
        bound = "smem"
        bytes_per_move = 12 * z + 12 + 2 * 8 + 8 + 4 + 12 * acc_rate
        peak, _ = rw.measure_smem_bandwidth(stream)
        peak_source = "measured live: conflict-free 16-byte shared-memory loads on every SM"
    else:
        bound = "hbm"
        bytes_per_move = 12 * z + 12 + 12 * acc_rate
        peak, peak_source = hbm_peak()
    achieved = bytes_per_move * S * workload["exchange_interval"] / (walk_avg_ms * 1e-3)
    nsh = len(workload["J"])
    if not pipelined:
        kernel = f"walker_kernel<false,{in_smem}>"
    elif in_smem == "true":
        kernel = f"walker_pipe_kernel<false,{nsh}>"
    else:
        kernel = f"walker_pipe_global_kernel<false,{nsh}>"
    traffic = profiled_traffic(kernel, S * workload["exchange_interval"])

    # end to end through the public API with host buffers: ln g in (warm start), merged ln g out
    lng_in = np.zeros(B)
    lng_out = np.zeros(B)
    h2d = S * sim.W * 8 + 2 * S * 8
    d2h = B * 8
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(max(2, args.steps)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.set_initial_lng(lng_in, 1.0)
        sim.run_intervals(I, stats=False)
        lng_out[:], _ = sim.merge()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total = all_max(sum(e2e_ms), world)
    e2e_value = moves_per_step * len(e2e_ms) * world / (e2e_total * 1e-3)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and args.gpus == 1:
        cpu = cpu_baseline(args.cpu_seconds, args.workload)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32 spins/dE + int64 fixed-point ln g/energy",
            "data": "synthetic",
            "config": {"workload": workload_name, "intervals_per_step": I,
                       "moves_per_step": moves_per_step * world, "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"{world} independent replica(s), one per GPU",
                       "group_size": sim.info()["group_size"], "accept_rate": acc_rate,
                       "recompute_rate": rec_rate, "conflict_entries": sim.info()["conflict_entries"],
                       "autotune": tune},
            "roofline": {"bound": bound, "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": kernel, "bytes_per_move": bytes_per_move,
                         "walker_ms_per_launch": walk_avg_ms, "walker_share_of_step": walker_share,
                         "cycles_per_move_per_walker": walk_avg_ms * 1e-3 * (clk.get("sm_mhz") or 0) * 1e6
                                                       / workload["exchange_interval"],
                         "sms_used": min(S, torch.cuda.get_device_properties(dev).multi_processor_count),
                         "peak_source": peak_source},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * (3 * I + 2),
            "clocks": clk,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
