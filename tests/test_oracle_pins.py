"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks one part of the oracle against something other than the oracle itself:
closed forms, exact rational arithmetic, brute force over a tiny lattice, library routines for
special cases, invariants, and the few numbers the paper prints (``tests/golden``).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------------
# helpers written from the geometry, independent of the oracle's tables
# ---------------------------------------------------------------------------------------------
def bcc_positions(L):
    """Half-unit coordinates of every site, site index 2 (x + L (y + L z)) + s."""
    N = 2 * L ** 3
    pos = np.zeros((N, 3), dtype=np.int64)
    for z in range(L):
        for y in range(L):
            for x in range(L):
                for s in range(2):
                    i = 2 * (x + L * (y + L * z)) + s
                    pos[i] = (2 * x + s, 2 * y + s, 2 * z + s)
    return pos


def min_image_r2(pos, L):
    """Squared minimum-image distances (quarter lattice-constant units) between all sites."""
    d = pos[None, :, :] - pos[:, None, :]
    d = (d + L) % (2 * L) - L
    return (d ** 2).sum(-1)


SHELL_R2 = {3: 0, 4: 1, 8: 2, 11: 3}   # r^2 = 3/4, 1, 2, 11/4 a^2 in quarter units


def brute_energy_bcc(spins, L, J):
    """E = -sum_{i<j} J(r_ij) S_i.S_j over all pairs, J by geometric shell."""
    pos = bcc_positions(L)
    r2 = min_image_r2(pos, L)
    Jm = np.zeros_like(r2, dtype=np.float64)
    for r, sh in SHELL_R2.items():
        if sh < len(J):
            Jm[r2 == r] = J[sh]
    S = spins.T  # [N, 3]
    dots = S @ S.T
    iu = np.triu_indices(len(S), 1)
    return -np.sum(Jm[iu] * dots[iu])


def ih_cdf(y, n):
    """Exact Irwin-Hall CDF of a sum of n U[0,1], at rational y."""
    y = Fraction(y)
    if y <= 0:
        return Fraction(0)
    if y >= n:
        return Fraction(1)
    s = Fraction(0)
    for k in range(int(math.floor(y)) + 1):
        s += (-1) ** k * math.comb(n, k) * (y - k) ** n
    return s / math.factorial(n)


def chain_exact_lng(n_spins, J, e_min, e_max, B):
    """ln of the exact bin masses of g(E) for the open chain: E = -J sum_b c_b, with the n = N-1
    bond cosines c_b i.i.d. uniform on [-1, 1], i.e. E = J (2y - n), y ~ Irwin-Hall(n)."""
    n = n_spins - 1
    e_min, e_max = Fraction(e_min), Fraction(e_max)
    dE = (e_max - e_min) / B
    out = []
    for b in range(B):
        e1 = e_min + b * dE
        e2 = e1 + dE
        y1 = (e1 / Fraction(J) + n) / 2
        y2 = (e2 / Fraction(J) + n) / 2
        out.append(math.log(float(ih_cdf(y2, n) - ih_cdf(y1, n))))
    return np.array(out)


def ulp_diff(a, b):
    ia = np.float64(a).view(np.int64)
    ib = np.float64(b).view(np.int64)
    return abs(int(ia) - int(ib))


# ---------------------------------------------------------------------------------------------
# random numbers
# ---------------------------------------------------------------------------------------------
def test_u53_closed_forms():
    assert o.u53(0, 0) == 0.0
    assert o.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert o.u53(0x80000000, 0) == 0.5
    assert o.u53(0, 0x40) == 2.0 ** -53


def test_philox_uniform_and_avalanche():
    words = []
    for i in range(20000):
        words.append(o.philox4x32_10([i, 0, 0, 0], [7, 11]))
    w = np.concatenate(words)
    counts = np.bincount((w >> 24).astype(np.int64), minlength=256)
    exp_c = w.size / 256
    chi2 = ((counts - exp_c) ** 2 / exp_c).sum()
    from scipy.stats import chi2 as chi2d
    assert chi2d.sf(chi2, 255) > 1e-4
    # one flipped counter bit changes about half of the 128 output bits
    base = o.philox4x32_10([123, 456, 789, 1011], [5, 6])
    flips = []
    for word in range(4):
        for bit in range(32):
            c = [123, 456, 789, 1011]
            c[word] ^= 1 << bit
            out = o.philox4x32_10(c, [5, 6])
            flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(out, base)))
    assert 0.45 < np.mean(flips) / 128 < 0.55


def test_direction_is_uniform_on_sphere():
    from scipy.stats import kstest
    S = np.array([o.draw_direction(3, 99, t, 1) for t in range(20000)])
    norms = np.linalg.norm(S, axis=1)
    assert np.max(np.abs(norms - 1.0)) < 1e-14
    # Archimedes: S_z uniform on [-1, 1]; azimuth uniform on [0, 2 pi)
    assert kstest(S[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-3
    phi = np.arctan2(S[:, 1], S[:, 0]) % (2 * np.pi)
    assert kstest(phi, "uniform", args=(0, 2 * np.pi)).pvalue > 1e-3
    assert abs(np.mean(S[:, 0])) < 0.03 and abs(np.mean(S[:, 1])) < 0.03


def test_site_draw_uniform():
    s = o.OracleREWL(L=4)
    sites = np.array([s.draw_site(0, t)[0] for t in range(40000)])
    assert sites.min() >= 0 and sites.max() < s.N
    counts = np.bincount(sites, minlength=s.N)
    exp_c = sites.size / s.N
    from scipy.stats import chi2 as chi2d
    assert chi2d.sf(((counts - exp_c) ** 2 / exp_c).sum(), s.N - 1) > 1e-4


# ---------------------------------------------------------------------------------------------
# exp
# ---------------------------------------------------------------------------------------------
def test_exp_within_2ulp_of_libm():
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(-708.0, 0.0, 100000), rng.uniform(-1.0, 0.0, 50000),
                         -np.logspace(-12, 2.8, 2000), [0.0, -1e-300, -0.5, -1.0, -700.0]])
    worst = 0
    for x in xs:
        worst = max(worst, ulp_diff(o.exp(float(x)), math.exp(float(x))))
    assert worst <= 2
    assert o.exp(0.0) == 1.0
    assert o.exp(-709.0) == 0.0


# ---------------------------------------------------------------------------------------------
# lattice and energy (Sec. 3, Eq. 1)
# ---------------------------------------------------------------------------------------------
def test_bcc_shells_from_geometry():
    L = 5
    pos = bcc_positions(L)
    r2 = min_image_r2(pos, L)
    s = o.OracleREWL(kind=o.BCC, L=L, J=(1.0, 0.5, 0.25, 0.125), n_bins=50, n_windows=1,
                     walkers_per_window=1)
    nbr, J = s.neighbours()
    assert s.z == 50
    _, shell = o.bcc_offsets(4)
    assert list(np.bincount(shell)) == [8, 6, 12, 24]
    for i in [0, 1, 17, 2 * L ** 3 - 1]:
        for r, sh in SHELL_R2.items():
            geo = set(np.nonzero(r2[i] == r)[0].tolist())
            tab = set(nbr[shell == sh, i].tolist())
            assert geo == tab and len(geo) == [8, 6, 12, 24][sh]
            assert np.all(J[shell == sh, i] == [1.0, 0.5, 0.25, 0.125][sh])
    # symmetry: j in nbr(i) <=> i in nbr(j), each pair twice in the table
    pairs = {(int(nbr[j, i]), i) for j in range(s.z) for i in range(s.N)}
    assert all((b, a) in pairs for (a, b) in pairs)
    assert all(len(set(nbr[:, i])) == s.z and i not in set(nbr[:, i]) for i in range(s.N))


def test_chain_table():
    s = o.OracleREWL(kind=o.CHAIN, L=6, J=(1.5,), n_bins=20, n_windows=1, walkers_per_window=1)
    nbr, J = s.neighbours()
    assert nbr.shape == (2, 6)
    assert list(nbr[0]) == [0, 0, 1, 2, 3, 4] and list(J[0]) == [0, 1.5, 1.5, 1.5, 1.5, 1.5]
    assert list(nbr[1]) == [1, 2, 3, 4, 5, 5] and list(J[1]) == [1.5, 1.5, 1.5, 1.5, 1.5, 0]
    assert s.e_min == -7.5 and s.e_max == 7.5


def test_ground_state_closed_forms():
    # ferromagnet: E_gs = -(N/2) sum_n z_n J_n
    for L, J in [(4, (1.0, 0.5)), (6, (1.0, 0.6, -0.05, -0.1)), (5, (1.0, 0.2, 0.1))]:
        N = 2 * L ** 3
        z = [8, 6, 12, 24]
        assert o.bcc_ground_state_shells(L, len(J), J) == pytest.approx(
            -0.5 * N * sum(zz * jj for zz, jj in zip(z, J)), rel=1e-14)
    # nearest-neighbour antiferromagnet on the bipartite bcc lattice: Neel state, -(N/2) 8 |J1|
    assert o.bcc_ground_state_shells(4, 1, [-1.0]) == pytest.approx(-0.5 * 128 * 8, rel=1e-14)
    # config-5 couplings: the aligned state is the ground state (E_gs = -4.3 N)
    assert o.bcc_ground_state_shells(8, 4, [1.0, 0.6, -0.05, -0.1]) == pytest.approx(-4.3 * 1024, rel=1e-12)


def test_ground_state_equals_best_spiral_by_brute_force():
    """Frustrated couplings: LT value = lowest energy of any commensurate single-q spiral,
    energies by brute-force pair sums over the geometry."""
    L, J = 3, (1.0, -2.0)
    pos = bcc_positions(L)
    best = math.inf
    for n1 in range(2 * L):
        for n2 in range(2 * L):
            for n3 in range(2 * L):
                ph = np.pi * (pos @ np.array([n1, n2, n3])) / L
                spins = np.stack([np.cos(ph), np.sin(ph), np.zeros_like(ph)])
                best = min(best, brute_energy_bcc(spins, L, J))
    assert o.bcc_ground_state_shells(L, 2, J) == pytest.approx(best, rel=1e-12)
    assert best > -0.5 * 54 * (8 * 1.0 + 6 * 2.0) - 1e-9  # above the naive bound


def test_running_energy_matches_brute_force_pairs():
    """dE of every accepted move (sign, field, indices) keeps the running energy equal to the
    pair-sum energy of the configuration."""
    J = (1.0, 0.5)
    s = o.OracleREWL(L=4, J=J, n_bins=200, n_windows=4, walkers_per_window=2, exchange_interval=3000)
    assert s.initial_energy() == -704.0
    s.init_walkers()
    s.run_intervals(3)
    w = s.walkers()
    sp = s.spins()
    for slot in range(s.n_slots):
        e_brute = brute_energy_bcc(sp[w["replica"][slot]], 4, J)
        assert w["E"][slot] == pytest.approx(e_brute, abs=1e-9)
        assert s.replica_energy(w["replica"][slot]) == pytest.approx(e_brute, abs=1e-9)
    assert s.max_drift() < 1e-9
    assert sorted(w["replica"]) == list(range(s.n_slots))


# ---------------------------------------------------------------------------------------------
# windows (Sec. 4.3, Sec. 4.4, Sec. 5)
# ---------------------------------------------------------------------------------------------
def test_window_size_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "paper_windows.json")))
    for key in ("L10", "L40"):
        c = g[key]
        span = c["e_max_eV"] - c["e_min_eV"]
        B = int(round(span / 0.01))                      # 0.01 eV bins
        W, starts = o.window_layout(B, c["n_windows"], c["overlap"])
        assert abs(W * 0.01 - c["window_size_eV"]) < 0.02
        assert starts[0] == 0 and starts[-1] + W == B
        # the paper's window count is the one that gives its window size
        others = [h for h in range(c["n_windows"] - 3, c["n_windows"] + 4)
                  if abs(o.window_layout(B, h, c["overlap"])[0] * 0.01 - c["window_size_eV"]) < 0.02]
        assert others == [c["n_windows"]]
    # energy range proportional to N (Sec. 4.4 vs Sec. 5)
    assert g["L10"]["e_min_eV"] / g["L10"]["n_spins"] == g["L40"]["e_min_eV"] / g["L40"]["n_spins"]


def test_window_overlaps():
    for B, h in [(200, 4), (2000, 16), (8000, 64), (6912, 32)]:
        W, st = o.window_layout(B, h, 0.75)
        ov = [(st[k] + W - st[k + 1]) / W for k in range(h - 1)]
        assert min(ov) > 0.72 and max(ov) < 0.78
        assert st[0] == 0 and st[-1] + W == B and np.all(np.diff(st) > 0)


# ---------------------------------------------------------------------------------------------
# Wang-Landau + exchange + merge, whole pipeline, against the exact chain g(E) (Sec. 4.2, 4.3)
# ---------------------------------------------------------------------------------------------
def run_to_end(s, lnf_final, chunk=10):
    s.init_walkers()
    while not s.all_done(lnf_final):
        s.run_intervals(chunk)


def test_chain_density_of_states_full_range():
    """Open chain of 5 spins, full range: WL ln g equals the exact Irwin-Hall bin masses."""
    Ns, B = 5, 32
    devs = []
    for seed in range(1, 5):
        s = o.OracleREWL(kind=o.CHAIN, L=Ns, J=(1.0,), n_bins=B, n_windows=1, walkers_per_window=1,
                         flatness=0.8, lnf_final=1e-6, seed=seed, exchange_interval=2000)
        run_to_end(s, 1e-6)
        lng, cen = s.merge()
        ex = chain_exact_lng(Ns, 1.0, s.e_min, s.e_max, B)
        devs.append(lng - (ex - ex.mean()))
        # beta = 0 moments from ln g: <E> = 0, <E^2> = (N-1) J^2 / 3; bin masses placed at the
        # bin centres add dE^2 / 12 (Sheppard's correction)
        p = np.exp(lng - lng.max())
        p /= p.sum()
        assert abs(np.sum(p * cen)) < 0.03
        assert np.sum(p * cen ** 2) == pytest.approx((Ns - 1) / 3.0 + s.dE ** 2 / 12, rel=0.02)
    devs = np.array(devs)
    assert np.sqrt(np.mean(devs.mean(0) ** 2)) < 0.03
    assert np.max(np.abs(devs.mean(0))) < 0.12


def test_chain_density_of_states_windows_exchange_merge():
    """Open chain of 8 spins over 3 windows x 2 walkers: exchange and stitching keep it exact."""
    Ns, B = 8, 56
    s = o.OracleREWL(kind=o.CHAIN, L=Ns, J=(1.0,), n_bins=B, n_windows=3, walkers_per_window=2,
                     overlap=0.75, flatness=0.8, lnf_final=1e-5, seed=3, exchange_interval=2000)
    run_to_end(s, 1e-5)
    lng, _ = s.merge()
    ex = chain_exact_lng(Ns, 1.0, s.e_min, s.e_max, B)
    dev = lng - (ex - ex.mean())
    assert np.sqrt(np.mean(dev ** 2)) < 0.06
    att, acc = s.exchange_counts()
    assert np.all(acc > 0) and np.all(acc <= att)


def test_bcc_nn_symmetry_and_moments():
    """Nearest-neighbour bcc is bipartite: g(E) = g(-E) on [E_gs, -E_gs]; beta = 0 moments
    <E> = 0, <E^2> = sum_pairs J^2 / 3 = (8 N / 2) / 3."""
    L = 2
    N = 16
    B = 32
    s = o.OracleREWL(kind=o.BCC, L=L, J=(1.0,), e_min=-64.0, e_max=64.0, n_bins=B, n_windows=1,
                     walkers_per_window=1, lnf_final=1e-5, seed=2, exchange_interval=5000)
    run_to_end(s, 1e-5)
    lng, cen = s.merge()
    # the two extreme bins are the hardest to sample; compare the rest
    inner = slice(1, B - 1)
    assert np.sqrt(np.mean((lng[inner] - lng[::-1][inner]) ** 2)) < 0.1
    p = np.exp(lng - lng.max())
    p /= p.sum()
    assert abs(np.sum(p * cen)) < 0.1
    # Sheppard's correction for bin masses at bin centres: + dE^2 / 12
    assert np.sum(p * cen ** 2) == pytest.approx(N * 8 / 2 / 3.0 + s.dE ** 2 / 12, rel=0.02)


# ---------------------------------------------------------------------------------------------
# thermodynamics (Sec. 4.1, Eq. 2-3) on the exact chain g(E)
# ---------------------------------------------------------------------------------------------
def test_thermo_chain_closed_form():
    """C = (N-1) (1 - x^2 / sinh^2 x), x = J/T, from Z = (4 pi)^N (sinh x / x)^(N-1)."""
    Ns, B = 10, 1800
    e_min, e_max = -9.0, 9.0
    lng = chain_exact_lng(Ns, 1.0, e_min, e_max, B)
    cen = e_min + (np.arange(B) + 0.5) * (e_max - e_min) / B
    T = np.array([0.5, 1.0, 2.0])
    U, Cps, _ = o.thermo(lng, cen, Ns, T)
    x = 1.0 / T
    c_bond = 1.0 - x ** 2 / np.sinh(x) ** 2
    assert np.allclose(Cps * Ns / (Ns - 1), c_bond, rtol=2e-3)
    assert c_bond[0] == pytest.approx(0.69591, abs=1e-5) and c_bond[1] == pytest.approx(0.27594, abs=1e-5)
    # U = -(N-1) J (coth x - 1/x) (Langevin function)
    assert np.allclose(U, -(Ns - 1) * (1 / np.tanh(x) - 1 / x), rtol=2e-3)


def test_peak_refinement_on_parabola():
    T = np.linspace(0.2, 3.0, 2801)
    C = 5.0 - (T - 1.2345) ** 2
    assert o.peak(T, C) == pytest.approx(1.2345, abs=1e-9)


# ---------------------------------------------------------------------------------------------
# merge (Sec. 4.3)
# ---------------------------------------------------------------------------------------------
def test_merge_recovers_offsets_exactly():
    B, h, m = 200, 5, 3
    W, st = o.window_layout(B, h, 0.75)
    f = 0.001 * (np.arange(B) - 100.0) ** 2 + 0.3 * np.arange(B)
    rng = np.random.default_rng(1)
    frag = np.zeros((h, m, W))
    for k in range(h):
        for a in range(m):
            frag[k, a] = f[st[k]:st[k] + W] + rng.uniform(-50, 50)
    out, bstar, rc = o.merge_fragments(frag, st, B)
    assert rc == 0
    assert np.max(np.abs(out - (f - f.mean()))) < 1e-9


def test_merge_joins_where_slopes_coincide():
    B, h, m = 100, 2, 1
    W, st = o.window_layout(B, h, 0.75)
    f = np.sin(np.arange(B) / 9.0) * 3.0
    b0 = st[1] + (st[0] + W - st[1]) // 2
    frag = np.zeros((h, m, W))
    frag[0, 0] = f[:W] + 7.0
    bb = np.arange(st[1], st[1] + W)
    frag[1, 0] = f[st[1]:] - 4.0 + 0.01 * (bb - b0) ** 2
    out, bstar, rc = o.merge_fragments(frag, st, B)
    assert list(bstar) == [b0]
    assert out[b0] - out[b0 - 1] == pytest.approx(f[b0] - f[b0 - 1], abs=1e-12)
    assert out[b0 - 1] - out[b0 - 2] == pytest.approx(f[b0 - 1] - f[b0 - 2], abs=1e-12)


def test_merge_ties_go_to_lowest_bin():
    B, h, m = 40, 2, 2
    W, st = o.window_layout(B, h, 0.75)
    f = np.arange(B, dtype=np.float64)          # exact slopes everywhere
    frag = np.zeros((h, m, W))
    for k in range(h):
        for a in range(m):
            frag[k, a] = f[st[k]:st[k] + W] + 8.0 * (k + a)
    _, bstar, _ = o.merge_fragments(frag, st, B)
    assert list(bstar) == [st[1] + 1]


def test_sum32_is_a_sum():
    rng = np.random.default_rng(3)
    for n in [1, 31, 32, 33, 1000, 8000]:
        x = rng.integers(-1000, 1000, n).astype(np.float64)   # exact in any order
        assert o.sum32(x) == x.sum()


# ---------------------------------------------------------------------------------------------
# flatness, exchange, init, frozen walkers, accounting (Sec. 4.2, 4.3)
# ---------------------------------------------------------------------------------------------
def test_flatness_rule():
    s = o.OracleREWL(kind=o.CHAIN, L=5, J=(1.0,), n_bins=5, n_windows=1, walkers_per_window=1,
                     flatness=0.8, lnf_final=1e-3)
    s.set_slot(0, H=[10, 10, 10, 10, 7])           # 7 < 0.8 * 9.4
    assert s.flatness() == 0 and s.walkers()["lnf"][0] == 1.0
    s.set_slot(0, H=[10, 10, 10, 10, 8])           # 8 >= 0.8 * 9.6
    assert s.flatness() == 1
    w = s.walkers()
    assert w["lnf"][0] == 0.5 and w["stage"][0] == 1 and np.all(w["H"][0] == 0)
    s2 = o.OracleREWL(kind=o.CHAIN, L=5, J=(1.0,), n_bins=2, n_windows=1, walkers_per_window=1,
                      flatness=0.5, lnf_final=1e-3)
    s2.set_slot(0, H=[1, 3])                       # min == p * mean exactly: flat
    assert s2.flatness() == 1
    s2.set_slot(0, H=[0, 0])                       # empty histogram is not flat
    assert s2.flatness() == 0


def test_exchange_acceptance_probability():
    """Eq. 5: swap accepted with min[1, g_i(E_A) g_j(E_B) / (g_i(E_B) g_j(E_A))]."""
    s = o.OracleREWL(kind=o.CHAIN, L=9, J=(1.0,), n_bins=40, n_windows=2, walkers_per_window=1,
                     overlap=0.75, seed=4)
    W, st = s.W, s.starts
    bA, bB = st[1] + 2, st[1] + 5              # both in the overlap
    EA, EB = s.e_min + (bA + 0.5) * s.dE, s.e_min + (bB + 0.5) * s.dE
    li = np.zeros(W)
    lj = np.zeros(W)
    li[bA - st[0]], li[bB - st[0]] = 0.4, 1.0     # ln g_i(E_A) - ln g_i(E_B) = -0.6
    lj[bB - st[1]], lj[bA - st[1]] = 2.0, 2.6     # ln g_j(E_B) - ln g_j(E_A) = -0.6
    s.set_slot(0, lng=li)
    s.set_slot(1, lng=lj)
    n, acc = 3000, 0
    for t in range(2 * n):
        s.set_slot(0, E=EA)
        s.set_slot(1, E=EB)
        before = s.walkers()["replica"].copy()
        s.exchange()
        acc += int(np.any(s.walkers()["replica"] != before))
    p = math.exp(-1.2)
    assert abs(acc / n - p) < 5 * math.sqrt(p * (1 - p) / n)
    # reversed roles: ratio > 1, always accepted
    s.set_slot(0, lng=-li)
    s.set_slot(1, lng=-lj)
    for t in range(20):
        s.set_slot(0, E=EA)
        s.set_slot(1, E=EB)
        before = s.walkers()["replica"].copy()
        s.exchange()
        if s.exchange_index() % 2 == 1:
            assert np.any(s.walkers()["replica"] != before)
    # E_A outside window 1: never exchanged
    s.set_slot(0, E=s.e_min + 0.5 * s.dE)
    s.set_slot(1, E=EB)
    att0, acc0 = s.exchange_counts()
    for t in range(10):
        s.exchange()
    att1, acc1 = s.exchange_counts()
    assert acc1[0] == acc0[0] and att1[0] > att0[0]


def test_init_reaches_every_window():
    s = o.OracleREWL(L=4, J=(1.0, 0.5), n_bins=200, n_windows=4, walkers_per_window=2)
    s.init_walkers()
    w = s.walkers()
    for slot in range(s.n_slots):
        k = slot // s.m
        assert s.starts[k] <= w["bin"][slot] < s.starts[k] + s.W
    assert np.all(w["lnf"] == 1.0) and np.all(w["H"] == 0) and np.all(w["lng"] == 0)


def test_frozen_walkers_do_not_update():
    s = o.OracleREWL(L=4, J=(1.0, 0.5), n_bins=200, n_windows=2, walkers_per_window=1,
                     lnf_initial=1e-4, lnf_final=1e-3, exchange_interval=2000)
    s.init_walkers()
    s.run_intervals(2)
    w = s.walkers()
    assert np.all(w["lng"] == 0) and np.all(w["H"] == 0) and np.all(w["accepts"] > 0)


def test_accounting_before_first_reduction():
    s = o.OracleREWL(L=4, J=(1.0, 0.5), n_bins=200, n_windows=4, walkers_per_window=2,
                     exchange_interval=500, flatness=0.999)
    s.init_walkers()
    s.run_intervals(4)
    w = s.walkers()
    assert np.all(w["stage"] == 0)
    assert np.all(w["H"].sum(1) == 2000) and np.all(w["steps"] == 2000)
    assert np.all(w["lng"].sum(1) == 2000.0)       # ln f = 1 added once per move


def test_round_trips_two_windows_equal_accepted_exchanges():
    """Two windows, one walker each: every accepted swap brings one configuration from the highest
    window to the lowest, and both were seen at their extremes before, so the round trips of all
    configurations add up to the accepted exchanges (Sec. 5, Fig. 1)."""
    sim = o.OracleREWL(kind=o.BCC, L=4, J=(1.0, 0.5), e_min=-400.0, e_max=0.0, n_bins=60, n_windows=2,
                       walkers_per_window=1, overlap=0.75, seed=3, exchange_interval=200)
    sim.init_walkers()
    sim.run_intervals(150)
    counts, last = sim.round_trips()
    _, acc = sim.exchange_counts()
    assert acc[0] > 10 and counts.sum() == acc[0]
    assert sorted(last.tolist()) == [0, 1]


def test_round_trips_match_a_recount_from_the_replica_paths():
    """Recount from the windows each configuration occupies after every exchange round (one
    exchange round per interval), independently of the oracle's own counter."""
    h, m = 4, 2
    sim = o.OracleREWL(kind=o.BCC, L=4, J=(1.0, 0.5), e_min=-400.0, e_max=0.0, n_bins=60, n_windows=h,
                       walkers_per_window=m, overlap=0.75, seed=5, exchange_interval=200)
    sim.init_walkers()
    S = h * m
    paths = [np.arange(S)]                      # slot -> configuration before the first round
    for _ in range(250):
        sim.run_intervals(1)
        paths.append(sim.walkers()["replica"].copy())
    counts = np.zeros(S, dtype=np.int64)
    last = np.full(S, -1)
    for perm in paths:
        window = np.empty(S, dtype=int)
        window[perm] = np.arange(S) // m        # window of every configuration
        for r in range(S):
            if window[r] == 0:
                counts[r] += last[r] == 1
                last[r] = 0
            elif window[r] == h - 1:
                last[r] = 1
    c, l = sim.round_trips()
    assert counts.sum() > 5
    assert np.array_equal(c, counts) and np.array_equal(l, last)


def _restricted(**kw):
    cfg = dict(kind=o.BCC, L=4, J=(1.0, 0.5), e_min=-400.0, e_max=0.0, n_bins=60, n_windows=3, overlap=0.75,
               exchange_interval=300, lnf_final=1e-3)
    cfg.update(kw)
    return o.OracleREWL(**cfg)


def test_window_iteration_with_one_walker_is_the_walker_iteration():
    a = _restricted(walkers_per_window=1, seed=7, iteration=0)
    b = _restricted(walkers_per_window=1, seed=7, iteration=1)
    for sim in (a, b):
        sim.init_walkers()
        sim.run_intervals(800)
    wa, wb = a.walkers(), b.walkers()
    assert wa["stage"].min() >= 3
    for k in wa:
        assert np.array_equal(wa[k], wb[k]), k


def test_window_iteration_moves_the_walkers_of_a_window_together():
    """After an interval in which a window moved on, its walkers hold one ln g (the average); at all
    times they share ln f and the stage count."""
    h, m = 3, 3
    sim = _restricted(walkers_per_window=m, seed=9, iteration=1)
    sim.init_walkers()
    prev = sim.walkers()["stage"].copy()
    moved = 0
    for _ in range(900):
        sim.run_intervals(1)
        w = sim.walkers()
        st = w["stage"].reshape(h, m)
        lnf = w["lnf"].reshape(h, m)
        assert np.all(st == st[:, :1]) and np.all(lnf == lnf[:, :1])
        lng = w["lng"].reshape(h, m, -1)
        for k in np.nonzero(st[:, 0] > prev.reshape(h, m)[:, 0])[0]:
            assert all(np.array_equal(lng[k, 0], lng[k, a]) for a in range(1, m))
            moved += 1
        prev = w["stage"].copy()
    assert moved >= 3


def test_iteration_mode_is_validated():
    with pytest.raises(ValueError):
        _restricted(walkers_per_window=2, seed=1, iteration=2)
