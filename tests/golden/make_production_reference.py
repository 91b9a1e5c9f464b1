"""Write production_reference_bcc4.json: the FP64 oracle's converged ln g(E) and specific-heat peak over
many seeds, the reference of the production-mode statistics test (tests/test_gpu_production.py).

Only the oracle runs here (oracle/, plain FP64 C).  Configuration: bcc L = 4 (128 spins), J = (1, 0.5),
restricted range [-400, 0) in 120 bins (bins about as wide as the temperature at the specific-heat peak),
4 windows x 2 walkers at 75 % overlap, flatness 0.8, exchange every 1e4 moves, ln f 1 -> 1e-5 by halving
(Sec. 4.2-4.3).  Per seed it stores the merged ln g (mean zero, Sec. 4.3) and the peak of
C(T) = (<E^2> - <E>^2) / (N T^2) (Sec. 4.1, Eq. 2-3) on T in [1.5, 4] (2501 points, parabola-refined).
The file holds the mean and standard deviation per bin and every seed's peak temperature.

    python tests/golden/make_production_reference.py [--seeds 256] [--procs N]
"""
import argparse
import json
import math
import os
import sys
import time
from multiprocessing import get_context

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

CFG = dict(L=4, J=[1.0, 0.5], e_min=-400.0, e_max=0.0, n_bins=120, n_windows=4, walkers_per_window=2,
           overlap=0.75, flatness=0.8, lnf_final=1e-5, exchange_interval=10000)
T_GRID = dict(start=1.5, stop=4.0, num=2501)
SEED0 = 100000
OUT = os.path.join(HERE, "production_reference_bcc4.json")


def one(seed):
    import oracle
    s = oracle.OracleREWL(kind=oracle.BCC, seed=seed, **dict(CFG, J=tuple(CFG["J"])))
    s.init_walkers()
    while not s.all_done(CFG["lnf_final"]):
        s.run_intervals(10)
    lng, cen = s.merge()
    T = np.linspace(**T_GRID)
    _, Cv, _ = oracle.thermo(lng, cen, s.N, T)
    return lng, oracle.peak(T, Cv)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--seeds", type=int, default=256)
    p.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = p.parse_args()
    t0 = time.time()
    seeds = [SEED0 + i for i in range(a.seeds)]
    with get_context("spawn").Pool(a.procs) as pool:
        res = pool.map(one, seeds)
    lng = np.array([r[0] for r in res])
    tp = np.array([r[1] for r in res])
    out = {
        "what": "FP64 oracle, converged merged ln g (mean zero) and C(T) peak temperature per seed",
        "config": CFG, "lattice": "bcc", "T_grid": T_GRID, "seeds": [seeds[0], seeds[-1]], "n_seeds": len(seeds),
        "lng_mean": [float(v) for v in lng.mean(0)],
        "lng_sd": [float(v) for v in lng.std(0, ddof=1)],
        "tpeak": [float(v) for v in tp],
        "summary": {"per_seed_rms_spread": float(math.sqrt(np.mean(lng.var(0, ddof=1)))),
                    "tpeak_mean": float(tp.mean()), "tpeak_sd": float(tp.std(ddof=1)),
                    "cpu_seconds_wall": time.time() - t0, "procs": a.procs},
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out["summary"]))


if __name__ == "__main__":
    main()
