"""Seeded synthetic workloads: lattice sizes, coupling sets and window layouts of the benchmark
configurations.  Only parameters are generated here (no sampling arithmetic); the GPU path, the
benchmark and the tests share them.

The paper's own runs use bcc Fe with first-principles couplings (Sec. 5), which are not available;
these stand-ins keep its structure (bcc, up to four ferromagnetic/antiferromagnetic shells, many
overlapping windows) with dimensionless couplings in units of J1.
"""
import numpy as np

# bcc L=16, two shells: the single-job benchmark workload
SINGLE_L16 = dict(L=16, J=(1.0, 0.5), n_bins=2000, n_windows=16, walkers_per_window=4, overlap=0.75,
                  flatness=0.8, lnf_final=1e-8, exchange_interval=10000)

# bcc L=32, four shells (8 + 6 + 12 + 24 = 50 neighbours)
LARGE_L32 = dict(L=32, J=(1.0, 0.6, -0.05, -0.1), n_bins=8000, n_windows=64, walkers_per_window=8,
                 overlap=0.75, flatness=0.8, lnf_final=1e-8, exchange_interval=10000)

BATCH_SIZES = (8, 12, 16, 20)
BATCH_WINDOWS = {8: 8, 12: 16, 16: 24, 20: 32}


def random_couplings(seed):
    """J1 = 1, J2 ~ U[0.2, 0.6], J3 ~ U[-0.1, 0.1], drawn by a Philox generator keyed by `seed`."""
    g = np.random.Generator(np.random.Philox(key=int(seed)))
    j2 = g.uniform(0.2, 0.6)
    j3 = g.uniform(-0.1, 0.1)
    return (1.0, float(j2), float(j3))


def random_couplings4(seed):
    """Four shells: J1 = 1, J2 ~ U[0.2, 0.6], J3 ~ U[-0.1, 0.1] as random_couplings, and J4 ~ U[-0.1, 0.1]
    (the fourth shell of the bcc L = 32 workload's couplings lies inside these ranges)."""
    g = np.random.Generator(np.random.Philox(key=int(seed)))
    j2 = g.uniform(0.2, 0.6)
    j3 = g.uniform(-0.1, 0.1)
    j4 = g.uniform(-0.1, 0.1)
    return (1.0, float(j2), float(j3), float(j4))


# The bcc L = 32 four-shell couplings on a range around the specific-heat peak: E/N in [-2.50, -2.10]
# (the peak's energy per spin extrapolates to about -2.31 from oracle runs at L = 4, 5, 6), bins of
# 1.6 J1 (about the peak temperature), windows of about 216 bins at 75 % overlap, 2 walkers each.
TARGET_L32 = dict(L=32, J=(1.0, 0.6, -0.05, -0.1), e_per_spin=(-2.50, -2.10), bin_width=1.6, window_bins=216,
                  walkers_per_window=2, overlap=0.75, flatness=0.8, exchange_interval=4000)


def batch64_jobs(jobs_per_size=16, lnf_final=1e-6, exchange_interval=10000):
    """64 independent jobs, 16 per bcc L in {8, 12, 16, 20}: random three-shell couplings (job j keyed by
    seed j), n_bins = N/4 over [E_gs, 0], 8/16/24/32 windows x 4 walkers at 75 % overlap."""
    jobs = []
    j = 0
    for L in BATCH_SIZES:
        N = 2 * L ** 3
        for _ in range(jobs_per_size):
            jobs.append(dict(L=L, J=random_couplings(j), n_bins=N // 4, n_windows=BATCH_WINDOWS[L],
                             walkers_per_window=4, overlap=0.75, flatness=0.8, lnf_final=lnf_final,
                             exchange_interval=exchange_interval, seed=1000 + j))
            j += 1
    return jobs
