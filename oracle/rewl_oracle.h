/*
 * rewl_oracle.h -- plain, slow, single-threaded FP64 replica-exchange Wang-Landau (REWL)
 * for the classical Heisenberg model (Perera, Li, Eisenbach, Vogel, Landau, "Replica-exchange
 * Wang-Landau sampling: pushing the limits of Monte Carlo simulations in materials sciences").
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library against a reading of
 * the paper that can be verified by eye.  Only the test suite, the smoke entry point and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table or constant
 * generator with the CUDA library, and the library never calls it.
 *
 * What it computes (paper section in brackets):
 *   - Heisenberg energy  H = -sum_{i<j} J_ij S_i.S_j, |S_i| = 1                       [Sec. 3, Eq. 1]
 *   - bcc lattice, N = 2 L^3, neighbour shells 1..4                                   [Sec. 3]
 *   - Wang-Landau walk: acceptance min[1, g(E_A)/g(E_B)], ln g += ln f, H += 1 at the
 *     resulting state, flatness H(E) >= p <H>, ln f -> ln f / 2                         [Sec. 4.2, Eq. 4]
 *   - trial move: a random spin gets a uniformly random new direction                  [Sec. 4.4]
 *   - h overlapping energy windows, m walkers per window, replica exchange between
 *     adjacent windows with acceptance min[1, g_i(E_A) g_j(E_B) / (g_i(E_B) g_j(E_A))]  [Sec. 4.3, Eq. 5]
 *   - joining of ln g fragments where d ln g / dE best coincide                         [Sec. 4.3]
 *   - Z, <E>, C_V = (<E^2> - <E>^2) / (k_B T^2) from g(E)                               [Sec. 4.1, Eq. 2-3]
 *
 * Randomness comes from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random
 * numbers: as easy as 1, 2, 3"), keyed by (walker slot, seed) with counter (step, purpose,
 * attempt), so that any implementation that follows the same trajectory specification draws
 * the same numbers.  All arithmetic is FP64 with no fused multiply-add; the build compiles this
 * file with -ffp-contract=off.
 */
#ifndef REWL_ORACLE_H
#define REWL_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ro_sim ro_sim;

enum { RO_BCC = 0, RO_CHAIN = 1, RO_TABLE = 2 };

typedef struct {
  int32_t kind;            /* RO_BCC, RO_CHAIN or RO_TABLE */
  int32_t L;               /* bcc: cubic cells per side; chain: number of spins */
  int32_t n_shells;        /* bcc: number of coupling shells, 1..4 */
  double J[4];             /* bcc: J per shell; chain: J[0] */
  int32_t n_sites, z;      /* table: sites and neighbour slots per site */
  const int32_t* nbr;      /* table: [z][n_sites] neighbour index (copied) */
  const double* Jt;        /* table: [z][n_sites] coupling (copied) */
  double e_min, e_max;     /* NaN, NaN -> default range (bcc: [E_gs, 0]; chain: full range) */
  int32_t n_bins, n_windows, walkers_per_window;
  double overlap, flatness, lnf_final, lnf_initial;
  uint64_t seed;
  int64_t exchange_interval;   /* moves per walker between exchanges */
  int32_t group_size;          /* G: lanes per neighbour sum; fixes the summation order */
  int64_t init_max_moves;      /* cap on the moves that drive a walker into its window */
  int32_t iteration;           /* 0: every walker halves ln f on its own flat histogram (Sec. 4.3,
                                  literal); 1: a window halves when all its walkers are flat, after
                                  averaging their ln g */
} ro_params;

/* --- building blocks (exposed so that tests can pin them one by one) --- */
void ro_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double ro_u53(uint32_t a, uint32_t b);
double ro_exp(double x);
/* canonical bcc offsets in half lattice units, shell by shell; returns z (or -1) */
int ro_bcc_offsets(int n_shells, int32_t* dx, int32_t* dy, int32_t* dz, int32_t* shell);
/* Luttinger-Tisza ground-state energy of the bcc lattice by brute force over allowed q */
double ro_bcc_ground_state(int L, int n_shells, const double* J);
/* window layout: returns W and fills starts[h]; -1 on invalid input */
int ro_window_layout(int n_bins, int n_windows, double overlap, int32_t* starts);
/* the canonical 32-lane reduction order: lane l sums x[l], x[l+32], ... ; xor butterfly 16..1 */
double ro_sum32(const double* x, int n);

/* --- the simulation --- */
int ro_create(const ro_params* p, ro_sim** out, char* err, int errlen);
void ro_destroy(ro_sim* s);
int ro_init_walkers(ro_sim* s);                 /* 0 ok, <0 error (window not reached) */
int ro_run_intervals(ro_sim* s, int n);         /* moves, energy check, exchange, flatness */
int ro_run_moves_only(ro_sim* s, int64_t moves_per_walker);  /* WL moves only (timing leg) */
int ro_exchange(ro_sim* s);                     /* one replica-exchange round */
int ro_flatness(ro_sim* s);                     /* flatness check; returns walkers that halved */

/* sizes */
void ro_sizes(const ro_sim* s, int32_t* N, int32_t* z, int32_t* n_slots, int32_t* W, int32_t* B,
              int32_t* h, int32_t* m);
void ro_energy_grid(const ro_sim* s, double* e_min, double* e_max, double* dE);
void ro_window_starts(const ro_sim* s, int32_t* starts);
void ro_neighbours(const ro_sim* s, int32_t* nbr /*[z][N]*/, double* J /*[z][N]*/);
double ro_initial_energy(const ro_sim* s);

/* state getters (all arrays caller-owned) */
void ro_get_walkers(const ro_sim* s, double* lng /*[S][W]*/, uint32_t* H /*[S][W]*/,
                    double* E /*[S]*/, int32_t* bin /*[S]*/, double* lnf /*[S]*/,
                    int32_t* replica /*[S]*/, int64_t* accepts /*[S]*/, int32_t* stage /*[S]*/,
                    int64_t* steps /*[S]*/, int64_t* init_moves /*[S]*/);
void ro_get_spins(const ro_sim* s, double* spins /*[R][3][N]*/);
void ro_get_exchange_counts(const ro_sim* s, int64_t* attempts /*[h-1]*/, int64_t* accepts);
/* Round trips per replica [S] and the extreme window each replica was found in last (-1 none,
   0 lowest, 1 highest); either pointer may be NULL. */
void ro_get_round_trips(const ro_sim* s, int64_t* counts, int32_t* last);
double ro_max_drift(const ro_sim* s);
int64_t ro_exchange_index(const ro_sim* s);
/* overwrite every walker's ln g with lng0[b] (global bins) and set ln f */
void ro_set_lng(ro_sim* s, const double* lng0 /*[B]*/, double lnf0);
/* test hooks: the trial-move draws of one slot, and direct setting of one slot's state */
void ro_draw_direction(uint32_t slot, uint32_t key1, uint64_t t, uint32_t purpose, double S[3]);
void ro_draw_site(const ro_sim* s, uint32_t slot, uint64_t t, uint32_t purpose, int32_t* site, double* u);
void ro_set_slot(ro_sim* s, int slot, const double* lng /*[W] or NULL*/, const uint32_t* H /*[W] or NULL*/,
                 double E /*NaN = keep*/);
/* full recomputation of the energy of one replica, in the canonical site/slot order */
double ro_replica_energy(const ro_sim* s, int replica);

/* merge of the window fragments into one ln g over all B bins (mean zero) */
int ro_merge(const ro_sim* s, double* lng_out /*[B]*/, double* centres /*[B] or NULL*/);
/* merge of given fragments frag[h][m][W] (same rule), for tests on synthetic fragments */
int ro_merge_fragments(const double* frag, const int32_t* starts, int h, int m, int W, int B,
                       double* lng_out, int32_t* bstar_out /*[h-1] or NULL*/);

/* thermodynamics from ln g at bin centres E[b] (k_B = 1) */
void ro_thermo(const double* lng, const double* E, int B, double n_spins, const double* T, int nT,
               double* U /*[nT]*/, double* C /*[nT] specific heat per spin*/, double* lnZ /*[nT]*/);
/* grid argmax of C refined by a 3-point parabola */
double ro_peak(const double* T, const double* C, int nT);

#ifdef __cplusplus
}
#endif
#endif
