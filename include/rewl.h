/*
 * rewl.h -- C ABI of the GB300 replica-exchange Wang-Landau (REWL) library.
 *
 * Method: Perera, Li, Eisenbach, Vogel, Landau, "Replica-exchange Wang-Landau sampling: pushing the
 * limits of Monte Carlo simulations in materials sciences".  The library samples the density of
 * states g(E) of the classical Heisenberg model H = -sum_{i<j} J_ij S_i.S_j, |S_i| = 1 (Sec. 3,
 * Eq. 1) with many Wang-Landau walkers (Sec. 4.2, Eq. 4) in overlapping energy windows, replica
 * exchange between adjacent windows (Sec. 4.3, Eq. 5) and joining of the ln g fragments where
 * their slopes coincide (Sec. 4.3).  Thermodynamics follow from g(E) (Sec. 4.1, Eq. 2-3).
 *
 * Conventions (every entry point):
 *   - A call returns rewl_status; REWL_OK is 0.  rewl_last_error() describes the latest failure
 *     of a handle (or of handle-less calls when passed NULL).
 *   - Inputs are copied at the call; the caller keeps ownership of its arrays.  Outputs go into
 *     caller-allocated buffers whose sizes are stated per argument.
 *   - Pointers documented as "host" must be host memory; "device" pointers must be device memory
 *     of the current CUDA device.  Work is ordered on the handle's CUDA stream (rewl_config
 *     .cuda_stream, NULL = legacy default stream); calls that return data to host memory
 *     synchronise that stream before returning.
 *   - Invalid arguments return REWL_EINVAL and leave the handle unchanged.  A CUDA failure
 *     returns REWL_ECUDA; a handle that saw REWL_ECUDA must only be destroyed.
 */
#ifndef REWL_H
#define REWL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rewl_handle rewl_handle; /* opaque, owned by the library */

typedef enum {
  REWL_OK = 0,
  REWL_EINVAL = 1,   /* invalid argument or combination of arguments */
  REWL_ENOMEM = 2,   /* host or device allocation failed */
  REWL_ECUDA = 3,    /* a CUDA call failed */
  REWL_ETIMEOUT = 4, /* a bounded device or host wait gave up (stage move cap, initial drive cap) */
  REWL_ESTATE = 5    /* call not valid in the handle's current state */
} rewl_status;

enum {
  REWL_LATTICE_BCC = 0,   /* periodic bcc, N = 2 L^3, neighbour shells 1..4 (Sec. 3) */
  REWL_LATTICE_CHAIN = 1, /* open 1D chain of L spins, nearest neighbours only */
  REWL_LATTICE_TABLE = 2  /* explicit neighbour table */
};

enum {
  REWL_ITERATION_WALKER = 0, /* each walker proceeds to its next iteration on its own (default) */
  REWL_ITERATION_WINDOW = 1  /* the walkers of a window proceed together, ln g averaged */
};

enum {
  REWL_MODE_PRODUCTION = 0, /* FP32 spins and dE; ln g and energy in 64-bit fixed point */
  REWL_MODE_TRAJECTORY = 1  /* everything FP64; reproduces the FP64 reference walk bit for bit */
};

/* Lattice.  bcc: site index 2 (x + L (y + L z)) + s for cubic cell (x, y, z), sublattice s (s = 1
 * is the body centre).  Shell n (n = 1..4) holds the 8, 6, 12, 24 sites at squared distance 3/4,
 * 1, 2, 11/4 (cubic lattice constant a = 1); periodic wrap needs every offset component < L/2.
 * chain: site i couples to i-1 and i+1 with J[0]; the two ends have one neighbour.
 * table: nbr[j * n_sites + i] is the j-th neighbour of site i (0 <= nbr < n_sites), J the
 * coupling of that bond ([z][n_sites] both, row-major, copied); a coupling of 0 marks an unused slot;
 * z <= 64. */
typedef struct {
  int32_t kind;
  int32_t L;
  int32_t n_sites, z;     /* table only */
  const int32_t* nbr;     /* table only, host */
  const double* J;        /* table only, host */
} rewl_lattice;

/* Couplings J_n of shell n for bcc (J > 0 ferromagnetic, H = -sum J S.S); J[0] for the chain. */
typedef struct {
  int32_t n_shells;
  double J[4];
} rewl_couplings;

/* Energy range [e_min, e_max) split into n_bins bins of width (e_max - e_min) / n_bins, covered by
 * n_windows windows (Sec. 3 restricted range; Sec. 4.3 windows).  e_min = e_max = NaN selects the
 * default range: bcc [E_gs, 0] with E_gs the Luttinger-Tisza ground-state energy; chain the full
 * range [-(L-1)|J|, (L-1)|J|].  Table lattices need an explicit range. */
typedef struct {
  double e_min, e_max;
  int32_t n_bins, n_windows;
} rewl_windows;

typedef struct {
  uint64_t seed;                 /* Philox key material */
  int32_t mode;                  /* REWL_MODE_PRODUCTION or REWL_MODE_TRAJECTORY */
  int32_t group_size;            /* lanes per trial move (1,2,4,8,16,32) = summation order of the
                                    local field; 0 = choose from N and z */
  int64_t exchange_interval;     /* trial moves per walker between replica exchanges (> 0) */
  int64_t max_moves_per_stage;   /* cap for rewl_run_stage (moves per walker); 0 = no cap */
  int64_t init_max_moves;        /* cap for the initial drive into the windows; 0 = 2^40 */
  int32_t recompute_every;       /* full energy recomputation every this many intervals; 0 =
                                    default (production 8: replaces the running energy;
                                    trajectory 1: drift diagnostic only) */
  int32_t iteration;             /* REWL_ITERATION_WALKER (0): every walker halves ln f on its own
                                    flat histogram (Sec. 4.3, as written); REWL_ITERATION_WINDOW (1):
                                    a window moves on when all its walkers are flat, after their
                                    ln g are averaged bin by bin */
  double lnf_initial;            /* initial ln f; 0 = 1 (f0 = e, Sec. 4.2) */
  double timeout_s;              /* wall-clock cap for rewl_run_stage (0 = none) */
  void* cuda_stream;             /* cudaStream_t used for every launch (NULL = default stream) */
  int32_t resolver;              /* production mode, warp-specialised walker: how each batch of 32
                                    trial moves is resolved in order.  REWL_RESOLVER_AUTO (0) picks
                                    per batch from the previous batch's event counts; the others
                                    force one path for every batch.  All paths take the same
                                    decisions (same state, bit for bit); only their cost differs */
} rewl_config;

enum {
  REWL_RESOLVER_AUTO = 0,       /* per batch: the cheapest of the three for the last batch's events */
  REWL_RESOLVER_SCAN = 1,       /* one 64-bit warp prefix scan of the energy increments, one ballot
                                   round per event (bin change, correction) */
  REWL_RESOLVER_BLOCKS = 2,     /* branch-free blocks of 8 moves; events leave the block */
  REWL_RESOLVER_SEQUENTIAL = 3  /* one move at a time */
};

typedef struct {
  int64_t moves;               /* trial moves attempted in the call (all walkers) */
  int64_t accepts;             /* accepted trial moves in the call */
  int64_t exchange_attempts;   /* replica-exchange attempts in the call */
  int64_t exchange_accepts;
  int32_t intervals;           /* exchange intervals run */
  int32_t n_halved;            /* ln f reductions in the call (all walkers) */
  int32_t n_done;              /* walkers with ln f < lnf_final after the call */
  int32_t all_done;            /* 1 when every walker has ln f < lnf_final */
  double min_lnf, max_lnf;
  double max_energy_drift;     /* largest |running E - recomputed E| seen so far */
  double elapsed_ms;           /* wall time of the call */
} rewl_stage_stats;

typedef struct {
  int32_t n_sites, z, n_slots, n_replicas;
  int32_t n_bins, n_windows, walkers_per_window, window_bins;
  int32_t group_size, mode;
  double e_min, e_max, bin_width;
  double initial_energy;       /* energy of the aligned starting state */
  int64_t exchange_index;      /* replica-exchange rounds done */
  int64_t intervals_done;
  size_t shared_bytes_per_walker;
  int32_t lattice_in_shared;   /* 1 when each walker's spins live in shared memory */
  int32_t pipelined;           /* 1 when the Wang-Landau moves run on the warp-specialised walker */
  int32_t conflict_entries;    /* pipelined walker: entries of its per-walker conflict table (sites
                                  map to entry site mod entries); 0 otherwise */
} rewl_info;

typedef struct {
  int64_t moves;
  int64_t accepts;
  int64_t recomputes;          /* trial moves whose dE was re-evaluated or corrected after an accepted
                                  move still in flight (the walker's batch or the one before) touched
                                  its neighbourhood.  The production walker over a lattice in global
                                  memory counts real conflicts only; with the lattice in shared
                                  memory, moves sharing a conflict-table entry count too (the table
                                  has an entry per site up to 8192 sites) */
  int64_t batches_scan;        /* production, warp-specialised walker: batches of 32 moves resolved */
  int64_t batches_blocks;      /*   by the warp scan, by 8-move blocks and one move at a time */
  int64_t batches_sequential;  /*   (all 0 for the other walkers and in trajectory mode) */
} rewl_counters;

/* Create a simulation: lattice and couplings (Sec. 3), windows (Sec. 4.3), m walkers per window,
 * overlap o in [0, 1), flatness p in (0, 1) (Sec. 4.2), ln f_final > 0.  Builds the neighbour
 * geometry, the window layout W = ceil(B / (1 + (h-1)(1-o))), start_k = round(k (B-W)/(h-1)),
 * allocates device state and puts every replica in the aligned (+z) state.  Rejects: bad
 * lattice (L too small for the shells, table index out of range), NaN couplings, empty or NaN
 * energy range, h > B, W < 2, fewer than 2 overlap bins between adjacent windows, p or o out of
 * range, lnf_final <= 0, exchange_interval < 1.  *out is NULL on failure. */
rewl_status rewl_create(const rewl_lattice* lattice, const rewl_couplings* couplings,
                        const rewl_windows* windows, int walkers_per_window, double overlap,
                        double flatness, double lnf_final, const rewl_config* config,
                        rewl_handle** out);

/* Drive every walker from the aligned state into its window (the paper starts from an arbitrary
 * configuration, Sec. 4.2): trial moves are accepted iff they do not increase the distance to the
 * window centre; no ln g / H updates.  Called automatically by the first run call.
 * REWL_ETIMEOUT if a walker needs more than init_max_moves. */
rewl_status rewl_init_walkers(rewl_handle* h);

/* Run n exchange intervals: each is exchange_interval Wang-Landau trial moves per walker (Sec. 4.2,
 * Eq. 4; trial move Sec. 4.4) in one persistent launch, then the energy check/recomputation, one
 * replica-exchange round (Sec. 4.3, Eq. 5) and the flatness check with ln f -> ln f / 2 (Sec. 4.2).
 * stats may be NULL.  Stream-ordered; blocks only when stats is non-NULL. */
rewl_status rewl_run_intervals(rewl_handle* h, int n_intervals, rewl_stage_stats* stats);

/* Run intervals until every walker that had ln f >= ln f_final at the start of the call has reduced
 * ln f at least once (one Wang-Landau iteration, Sec. 4.2), or until max_moves_per_stage / timeout_s.
 * Returns REWL_ETIMEOUT when a cap ended the stage first.  stats may be NULL. */
rewl_status rewl_run_stage(rewl_handle* h, rewl_stage_stats* stats);

/* The three steps of one exchange interval as separate stream-ordered launches (for callers that
 * interleave their own work or time each kernel): rewl_walk runs exchange_interval Wang-Landau
 * trial moves per walker (Sec. 4.2, Eq. 4; Sec. 4.4) and the energy recomputation when due;
 * rewl_flatness applies the flatness test and ln f -> ln f / 2 (Sec. 4.2).  Neither blocks. */
rewl_status rewl_walk(rewl_handle* h);
rewl_status rewl_flatness(rewl_handle* h);

/* Conflict-table autotuner of the pipelined walker (rewl_info .pipelined = 1).  The paper has no
 * counterpart: the moves it times are those of Sec. 4.2 (Eq. 4); only the launch shape changes.  Times
 * one walker launch of trial_moves (> 0) moves per walker for each table of 8192 down to 512 entries (at
 * most one per site, and with the lattice in shared memory only tables that fit beside it), twice (the
 * second round in reverse order), and keeps the table with the fastest trial.  A smaller table leaves
 * more shared memory to L1 and fits more walkers per SM (a run with more walkers than SMs then needs
 * fewer waves); sites sharing an entry cost extra exact corrections, never a different result.  The
 * default is the largest table that fits (lattice in shared memory) or 2048 entries (lattice in global
 * memory).  Other handles have nothing to tune: their table stays and no move is made.  The timed moves
 * are ordinary Wang-Landau moves: the walkers advance by them (walkers are initialised first if
 * needed).  entries_out, ms_out (host, may be NULL) receive the chosen size and its trial time (0 when
 * nothing was timed).  Blocks until the trials end. */
rewl_status rewl_autotune(rewl_handle* h, int64_t trial_moves, int32_t* entries_out, double* ms_out);

/* One replica-exchange round between adjacent windows (Sec. 4.3, Eq. 5): round t pairs windows
 * (k, k+1), k = t mod 2 (step 2), walker a with walker (a + floor(t/2)) mod m; a swap needs both
 * energies in the overlap and is accepted with min[1, g_i(E_A) g_j(E_B) / (g_i(E_B) g_j(E_A))]
 * evaluated in FP64; an accepted swap exchanges the configurations' indices and energies, never
 * the spins.  stats may be NULL (only the exchange fields are filled). */
rewl_status rewl_exchange(rewl_handle* h, rewl_stage_stats* stats);

/* Join the window fragments into ln g over all n_bins bins (Sec. 4.3): per window the m walkers are
 * averaged after removing each one's mean; adjacent windows are joined at the interior overlap bin
 * where their central-difference slopes differ least (lowest bin on ties); the result has mean 0.
 * lng_out: host, [n_bins] FP64.  e_centres_out: host, [n_bins] bin-centre energies, may be NULL. */
rewl_status rewl_merge_lng(rewl_handle* h, double* lng_out, double* e_centres_out);

/* Same as rewl_merge_lng with the result left in device memory: lng_out_dev [n_bins] FP64, device. */
rewl_status rewl_merge_lng_device(rewl_handle* h, double* lng_out_dev);

/* Join given fragments (same rule as rewl_merge_lng), all device pointers: frag [h][m][W] FP64,
 * starts [h] int32 (host), out [B] FP64 device.  bstar_out: device [h-1] int32, may be NULL.
 * The windows must cover the bins: starts[0] = 0, starts[h-1] + W = n_bins, starts increasing with
 * at least 2 overlap bins between neighbours (else REWL_EINVAL).  Scratch is allocated and freed on
 * the stream (stream-ordered allocator); the call synchronises the stream before returning. */
rewl_status rewl_stitch_device(const double* frag, const int32_t* starts_host, int n_windows,
                               int walkers_per_window, int window_bins, int n_bins, double* out,
                               int32_t* bstar_out, void* cuda_stream);

/* No-allocation variant of rewl_stitch_device.  The paper has no counterpart: this entry point
 * serves callers that must not allocate device memory, such as a host application that reserves
 * all device memory up front, or a latency-critical loop that must not trigger the implicit device
 * synchronisation of cudaMalloc / cudaFree.  Same arguments, layout, rules and result as
 * rewl_stitch_device (all pointers device memory except starts_host).
 * Scratch: one statically sized device array inside the library, 4 MiB (4194304 bytes), held by
 * every GPU that loads the library until the process exits.  The call needs
 * 8*h*W + 4*h + 4*max(h-1,1) bytes (each of the three parts rounded up to 256); larger sizes
 * return REWL_EINVAL.  The first call on a device looks up the array's device address for that
 * device (with it current); make that first call before any stream capture.  Every call shares the
 * one array and leaves its contents behind (each call writes all the scratch it reads), so calls
 * whose work overlaps on the GPU -- different streams or host threads -- race.  The call
 * synchronises cuda_stream before returning and makes no cudaMalloc, cudaFree or other allocation.
 * Errors are reported by rewl_last_error(NULL). */
rewl_status rewl_stitch_device_noalloc(const double* frag, const int32_t* starts_host, int n_windows,
                                       int walkers_per_window, int window_bins, int n_bins, double* out,
                                       int32_t* bstar_out, void* cuda_stream);

/* Thermodynamics from ln g (Sec. 4.1, Eq. 2-3, k_B = 1): for every T, the mean energy U(T),
 * the specific heat per spin C(T) = (<E^2> - <E>^2) / (N T^2) and ln Z(T).  All arrays host:
 * lng, e_centres [n_bins]; T, U_out, C_out, lnZ_out [n_T] (outputs may be NULL). Computed on
 * the device in FP64 on cuda_stream. */
rewl_status rewl_thermo(const double* lng, const double* e_centres, int n_bins, double n_spins,
                        const double* T, int n_T, double* U_out, double* C_out, double* lnZ_out,
                        void* cuda_stream);

/* Temperature of the specific-heat maximum (the paper reads the transition temperature off this peak,
 * Sec. 5; C(T) from Sec. 4.1, Eq. 3): the grid argmax b of C (lowest index on ties), refined by the
 * vertex of the parabola through (T, C) at b-1, b, b+1, i.e. T_b + (dT/2) (C_{b-1} - C_{b+1}) /
 * (C_{b-1} - 2 C_b + C_{b+1}) with dT = T_{b+1} - T_b (a uniform grid); at either end of the grid, or
 * when the denominator is 0, T_b.  T, C: host [n_T] (e.g. from rewl_thermo), increasing T; T_peak:
 * host, one double.  Computed on the device on cuda_stream; REWL_EINVAL for NULL or n_T < 1. */
rewl_status rewl_peak_temperature(const double* T, const double* C, int n_T, double* T_peak, void* cuda_stream);

/* Replace every walker's ln g by lng (host, [n_bins] over the global bins; each walker takes its
 * window's slice) and set ln f = lnf0 (> 0) for all walkers; histograms are cleared. */
rewl_status rewl_set_initial_lng(rewl_handle* h, const double* lng, double lnf0);

/* Sizes and layout. */
rewl_status rewl_get_info(const rewl_handle* h, rewl_info* out);

/* Walker state, host arrays, any may be NULL: lng [S][W] FP64 (production converts from fixed
 * point), H [S][W], E [S], bin [S] (global bin of E), lnf [S], replica [S] (configuration held by
 * slot s = k m + a), stage [S] (ln f reductions), accepts [S], steps [S] (trial moves done),
 * init_moves [S].  S = n_windows * walkers_per_window. */
rewl_status rewl_get_walkers(rewl_handle* h, double* lng, uint32_t* H, double* E, int32_t* bin,
                             double* lnf, int32_t* replica, int32_t* stage, int64_t* accepts,
                             int64_t* steps, int64_t* init_moves);

/* Spins of every configuration: host, [R][3][N] FP64 (x block, y block, z block). */
rewl_status rewl_get_spins(rewl_handle* h, double* spins);

/* Replica-exchange counters per window pair: host [n_windows - 1] each. */
rewl_status rewl_get_exchange_counts(rewl_handle* h, int64_t* attempts, int64_t* accepts);

/* Replica round trips (Sec. 5, Fig. 1), per configuration r (host arrays [S], either may be NULL):
 * counts[r] = round trips completed, last[r] = extreme window r was found in last (-1 none, 0 the
 * lowest window, 1 the highest).  A round trip is completed when a configuration is found in the
 * lowest window after having been found in the highest; the configurations of both extreme windows
 * are looked at before and after every replica-exchange round.  With one window nothing is counted. */
rewl_status rewl_get_round_trips(rewl_handle* h, int64_t* counts, int32_t* last);

/* Totals over all walkers. */
rewl_status rewl_get_counters(rewl_handle* h, rewl_counters* out);

/* The neighbour table as the device computes it: host [z][N] int32 and [z][N] FP64 couplings. */
rewl_status rewl_get_neighbours(rewl_handle* h, int32_t* nbr, double* J);

/* Full energy of every configuration recomputed on the device in FP64: host [R]. */
rewl_status rewl_replica_energies(rewl_handle* h, double* E);

/* Message for the latest failure of h (NULL: of the latest handle-less call). Never NULL. */
const char* rewl_last_error(const rewl_handle* h);

/* Release everything; NULL-safe. */
void rewl_destroy(rewl_handle* h);

/* ---- Checkpoints ---------------------------------------------------------------------------------
 * The paper has no checkpoint format; a converged large run takes hours, so the library can stop and
 * resume one.  A checkpoint holds the whole state of a handle at a call boundary: every
 * configuration's spins, the slot -> configuration permutation, every walker's energy, ln g and H of
 * its window, ln f, stage, Philox counter (trial moves done) and counters, the replica-exchange index
 * and counters, the round-trip records, and for a partitioned handle the global slot of each position.
 * Resuming from it continues the run exactly: in trajectory mode the resumed run is bit for bit the
 * uninterrupted one (in production too: the walk is deterministic for given arguments).  The
 * buffer is host memory of rewl_state_bytes bytes, about the size of the spins (production: 16 N bytes
 * per walker; trajectory: 24 N). */

/* Size in bytes of the handle's checkpoint. */
rewl_status rewl_state_bytes(rewl_handle* h, int64_t* bytes);

/* Write the checkpoint into buf (host, `bytes` = rewl_state_bytes, else REWL_EINVAL).  Blocks. */
rewl_status rewl_save_state(rewl_handle* h, void* buf, int64_t bytes);

/* Replace the handle's state by a checkpoint.  The handle must have been created with the same lattice,
 * couplings, windows, walkers, overlap, flatness, ln f_final, seed, mode, group size, exchange interval,
 * recomputation cadence, iteration reading and partition range as the one that saved it.  REWL_EINVAL, with
 * the handle unchanged, when the size, tag or version differ, when the checksum (64-bit FNV-1a over the
 * buffer) does not match (a corrupted buffer), or when the run's arguments differ.  Blocks. */
rewl_status rewl_load_state(rewl_handle* h, const void* buf, int64_t bytes);

/* ---- Partitioned runs: one REWL run split over several handles (one per GPU) -------------------
 * The paper runs every walker as its own process and exchanges replicas between processes of
 * adjacent windows (Sec. 4.3, Eq. 5).  Here a run of h windows x m walkers can be split over handles
 * by contiguous window ranges, one handle per GPU.  The window ranges are those at creation.
 * A handle hosts S = (window_end - window_begin) m positions.  Each position holds one
 * configuration (lattice and energy) for the whole run, and one slot state: the ln g and H of a
 * window, ln f, the stage, and the Philox key and counter of a global slot s = k m + a.  Exchanges
 * between two slots of one handle swap their configurations by index, as rewl_exchange does.  An
 * accepted exchange between slots of different handles moves the two slot states between the
 * handles (a few KB) and leaves the configurations where they are, so a handle comes to host slots
 * of other windows.  The run is the same Markov chain as the single handle, slot for slot: in
 * trajectory mode bit for bit.  A round of replica exchange is driven by the caller, who combines
 * per-slot arrays over the handles (elementwise max of rewl_partition_bins, sum of
 * rewl_partition_lookups: every entry is written by exactly one handle):
 *   1. bins_all  = combine(rewl_partition_bins of every handle)        (-1 before: max)
 *   2. lk_all    = combine(rewl_partition_lookups(bins_all) of every handle)   (0 before: sum)
 *   3. rewl_partition_exchange(bins_all, lk_all) on every handle -> swap_with
 *   4. for every hosted slot g with swap_with[g] = o >= 0: export g, import the state of o (exported by
 *      the handle hosting o) in its place (rewl_slot_export, rewl_slot_import)
 *   5. rewl_partition_observe on every handle (round trips).
 * Wang-Landau moves (rewl_walk) and the flatness test (rewl_flatness) run per handle.  Not available
 * on a partitioned handle: rewl_run_intervals, rewl_run_stage, rewl_exchange, the merge (gather the
 * fragments by global slot and call rewl_stitch_device), batches, REWL_ITERATION_WINDOW. */

/* Create the handle of windows [window_begin, window_end) of the run that rewl_create would create
 * with the same arguments (every handle of the run passes the same arguments but its own range).
 * REWL_EINVAL also when the range is empty or outside [0, n_windows). */
rewl_status rewl_create_partition(const rewl_lattice* lattice, const rewl_couplings* couplings,
                                  const rewl_windows* windows, int walkers_per_window, double overlap,
                                  double flatness, double lnf_final, const rewl_config* config,
                                  int window_begin, int window_end, rewl_handle** out);

/* Global slot hosted at each position: gid host [n_slots of rewl_get_info] (0..S-1 for a plain handle). */
rewl_status rewl_partition_slots(rewl_handle* h, int32_t* gid);

/* Step 1 of a round: bins host [h m]; the bin of the configuration at each position is written at
 * the global slot the position hosts; the other entries are left as they are.  Blocks. */
rewl_status rewl_partition_bins(rewl_handle* h, int32_t* bins);

/* Step 2: with bins_all (host [h m], every slot's bin), for every pair of the coming round with
 * exactly one slot here, that slot's ln g at its own configuration's bin and at the partner's:
 * lk host [2 h m], entries 2g and 2g+1 of each hosted slot g (0 where the slot is in no such pair or
 * the partner's bin lies outside its window).  The values are the 64 bits of the ln g tables:
 * 2^-40 fixed point (production) or the FP64 bit pattern (trajectory).  Other entries are left
 * as they are.  Blocks. */
rewl_status rewl_partition_lookups(rewl_handle* h, const int32_t* bins_all, int64_t* lk);

/* Step 3, the round (Sec. 4.3, Eq. 5; pairing as rewl_exchange): pairs with both slots here swap
 * their configurations; pairs with one slot here are decided from bins_all and lk_all (host [h m],
 * [2 h m], combined over the handles), D = ((ln g_i(E_A) - ln g_i(E_B)) + ln g_j(E_B)) - ln g_j(E_A)
 * in FP64 and the same Philox uniform, so both handles of a pair take the same decision.  swap_with
 * host [h m]: for each hosted slot in an accepted cross-handle pair the partner's global slot,
 * -1 elsewhere.  The handle hosting the pair's lower slot counts the attempt and the acceptance
 * (rewl_get_exchange_counts: sum over the handles).  Blocks. */
rewl_status rewl_partition_exchange(rewl_handle* h, const int32_t* bins_all, const int64_t* lk_all,
                                    int32_t* swap_with);

/* Step 5: after the slot states have moved, the configurations of the extreme windows are looked at
 * again (Sec. 5 round trips, counted per configuration of the handle).  Stream-ordered. */
rewl_status rewl_partition_observe(rewl_handle* h);

/* Size in bytes of a slot state buffer (rewl_slot_export / rewl_slot_import). */
rewl_status rewl_slot_state_bytes(rewl_handle* h, int64_t* bytes);

/* Copy the state of hosted global slot g into buf (host, rewl_slot_state_bytes): ln g and H of its
 * window, ln f, stage, trial moves done (the Philox counter), accept and correction counters, moves
 * of the initial drive, largest energy drift, resolver-path batch counts, and g itself.  Blocks. */
rewl_status rewl_slot_export(rewl_handle* h, int32_t g, void* buf);

/* Replace hosted slot g_out by the slot state in buf (exported by a handle of the same run): the
 * position keeps its configuration and from then on walks as the slot in buf (its window, Philox
 * key and counter).  REWL_EINVAL if g_out is not hosted here, the buffer is not a slot state of a run
 * with this window size and mode, or its slot is already hosted here.  Blocks. */
rewl_status rewl_slot_import(rewl_handle* h, int32_t g_out, const void* buf);

/* ---- Batches: many independent REWL jobs in one persistent walker launch ----------------------
 * A batch runs the exchange intervals (Sec. 4.2-4.3: Wang-Landau moves, replica exchange,
 * flatness check and ln f reduction) of many handles at once.  All walker slots of all jobs form
 * one work list, most expensive first; one persistent launch of the pipelined walker takes slots
 * from it, `workers_per_block` walker pairs per CTA, each pair with its own shared-memory arena
 * (a job's lattice sits in the arena or stays in global memory, per the tuning).  One launch each
 * then does the replica exchange and the flatness check of every job.  The launch sequence of an
 * interval is captured once into a CUDA graph and replayed.  The paper runs one job per machine;
 * batching is this library's own addition.  The result of every job is the same as running its
 * handle alone: in trajectory mode bit for bit, in production mode up to the order of the energy
 * recomputation's FP64 sum.
 * Requirements (else REWL_EINVAL): bcc lattices that use the pipelined walker (rewl_info
 * .pipelined = 1), all in the same mode, with the same number of coupling shells, exchange_interval
 * and recompute_every.  Walkers not yet initialised are initialised at creation (rewl_init_walkers).
 * The batch borrows the handles: they must outlive it, and must not be used on other streams
 * while a batch call runs.  Batch errors are reported by rewl_last_error(NULL). */
typedef struct rewl_batch rewl_batch; /* opaque, owned by the library */

typedef struct {
  int workers_per_block;     /* walker pairs (64 threads each) per CTA, 1..3 */
  int smem_lattice_max_n;    /* jobs with n_spins <= this keep the lattice in shared memory (if it
                                fits the arena); 0 = none; the others read it from global memory */
  int owner_entries_max;     /* jobs with the lattice in global memory: conflict-table entries at most
                                (a power of two, 256..8192; 0 = 8192).  Fewer entries fit more walker
                                pairs per SM; sites sharing an entry cost extra corrections */
} rewl_batch_tuning;

typedef struct {
  int n_jobs, n_items;       /* jobs, walker slots over all jobs */
  int n_active_jobs;         /* jobs in the work list (see rewl_batch_run_to_convergence) */
  int workers_per_block, smem_lattice_max_n, owner_entries_max;
  int grid, blocks_per_sm;   /* persistent launch: CTAs, resident CTAs per SM */
  int n_smem_lattice_jobs;   /* jobs whose lattice sits in shared memory */
  int64_t arena_bytes;       /* shared memory per walker pair */
  int64_t intervals_done;
  int graphs_built;          /* CUDA graphs instantiated so far */
} rewl_batch_info;

/* Create a batch over jobs[0..n_jobs-1] (host array of handles) on cuda_stream (NULL: the batch
 * creates its own non-blocking stream, since a graph cannot be captured on the legacy default
 * stream).  Work is ordered after each handle's pending work and each handle's stream waits for
 * the batch's work.  The initial tuning is 2 workers per block, every lattice that fits in shared
 * memory there. */
rewl_status rewl_batch_create(rewl_handle* const* jobs, int n_jobs, void* cuda_stream, rewl_batch** out);

/* Set the tuning explicitly (REWL_EINVAL if the tables of some job do not fit). */
rewl_status rewl_batch_set_tuning(rewl_batch* b, const rewl_batch_tuning* t);

/* Autotuner: time one walker launch of trial_moves moves per walker (> 0) for every candidate
 * (workers_per_block 1..3 x every lattice-size threshold of the batch's jobs x conflict tables of
 * 8192 down to 512 entries), twice (the second round in reverse order); keep the candidate with the
 * fastest trial.
 * The timed moves are ordinary Wang-Landau moves of the jobs: the walkers advance by them.
 * chosen (host, may be NULL) receives the tuning; ms_out (host, may be NULL) its trial time. */
rewl_status rewl_batch_autotune(rewl_batch* b, int64_t trial_moves, rewl_batch_tuning* chosen, double* ms_out);

/* Run n_intervals exchange intervals of every job in the work list (graph replays; the energy
 * recomputation comes every recompute_every intervals of the batch, as for a handle). */
rewl_status rewl_batch_run_intervals(rewl_batch* b, int n_intervals);

/* Run intervals until every walker of every job has ln f < ln f_final, checking every
 * check_every (>= 1) intervals; jobs that finish leave the work list.  Stops after max_intervals
 * (> 0) with REWL_ETIMEOUT.  n_done (host, may be NULL) receives the number of finished jobs. */
rewl_status rewl_batch_run_to_convergence(rewl_batch* b, int64_t max_intervals, int check_every, int* n_done);

rewl_status rewl_batch_get_info(const rewl_batch* b, rewl_batch_info* out);

/* Release the batch (not the handles); NULL-safe. */
void rewl_batch_destroy(rewl_batch* b);

/* ---- Learned warm start: an MLP from (E/N, 1/L, J1..J4) to ln g(E)/N ---------------------------
 * The paper has no learned part; this is the library's own addition.  The network is trained on
 * ln g curves that REWL runs of this library produced (over random coupling sets).  It gives every
 * walker an initial ln g; plain Wang-Landau then runs every stage from a small ln f0, so the
 * network can only save ln f reductions and never decides the result.
 * Architecture (fixed): 6 inputs x = (E/N, 1/L, J1, J2, J3, J4) (J of shells past the last = 0),
 * each shifted and scaled, x' = (x - in_shift) * in_scale; 3 hidden layers of 128 SiLU units; one
 * linear output y ~ ln g/N.  Weights and biases are used in BF16, rounded from an FP32 master copy;
 * activations and accumulations are FP32.  Parameters (REWL_MLP_PARAMS FP32 values, transposed
 * weights WT[k][j] = weight from input k to unit j):
 *   WT1 [6][128] | b1 [128] | WT2 [128][128] | b2 [128] | WT3 [128][128] | b3 [128] | WT4 [128] | b4.
 * Loss over a corpus of runs g with samples seg[g] .. seg[g+1]-1 (ln g is defined up to a constant
 * per run): L = (1/M) sum_g sum_s (r_s - mean_g r)^2, r = y - target, M = all samples.
 * Errors are reported by rewl_last_error(NULL). */
typedef struct rewl_mlp rewl_mlp; /* opaque, owned by the library */
#define REWL_MLP_INPUTS 6
#define REWL_MLP_PARAMS 34049

/* Number of FP32 parameters (REWL_MLP_PARAMS). */
int64_t rewl_mlp_param_count(void);

/* in_shift, in_scale: host [6] (finite, scales nonzero).  Initial weights uniform in
 * +-1/sqrt(fan_in) from a generator seeded by seed, biases 0.  Work runs on cuda_stream. */
rewl_status rewl_mlp_create(const float* in_shift, const float* in_scale, uint64_t seed, void* cuda_stream,
                            rewl_mlp** out);

/* Replace the FP32 master parameters (host [REWL_MLP_PARAMS]); the BF16 copy follows and the Adam
 * state is cleared. */
rewl_status rewl_mlp_set_params(rewl_mlp* m, const float* params);

/* Host copies of the FP32 master (params, may be NULL) and of the BF16 weights the kernels use
 * (params_bf16, raw bfloat16 bit patterns, may be NULL). */
rewl_status rewl_mlp_get_params(rewl_mlp* m, float* params, uint16_t* params_bf16);

/* Inference: x host [n][6] raw inputs, y host [n]. */
rewl_status rewl_mlp_forward(rewl_mlp* m, const float* x, int64_t n, float* y);

/* Full-batch loss and gradient: x [M][6], target [M], run_offsets [n_runs + 1] (0 = first, M =
 * last, increasing); loss (host, may be NULL) and grad (host [REWL_MLP_PARAMS], may be NULL).  The
 * gradient is summed in a fixed order (deterministic). */
rewl_status rewl_mlp_gradient(rewl_mlp* m, const float* x, const float* target, const int32_t* run_offsets,
                              int n_runs, double* loss, float* grad);

/* steps (>= 1) full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr > 0) on the
 * device; loss_history (host [steps], may be NULL) receives the loss before each step. */
rewl_status rewl_mlp_train(rewl_mlp* m, const float* x, const float* target, const int32_t* run_offsets,
                           int n_runs, int steps, float lr, float* loss_history);

/* Inputs of the handle's bins (bcc): x_out host [n_bins][6] at the bin centres; with lng (host
 * [n_bins], e.g. from rewl_merge_lng) t_out (host [n_bins], may be NULL) receives ln g/N. */
rewl_status rewl_mlp_features(const rewl_handle* h, const double* lng, float* x_out, float* t_out);

/* Warm start: predict ln g = N y at the handle's bins and install it in every walker with ln f =
 * lnf0 (> 0) (rewl_set_initial_lng).  lng_out (host [n_bins], may be NULL) receives the prediction. */
rewl_status rewl_mlp_warm_start(rewl_mlp* m, rewl_handle* h, double lnf0, double* lng_out);

/* Release the model; NULL-safe. */
void rewl_mlp_destroy(rewl_mlp* m);

/* Exp as used by the trajectory mode and the exchange acceptance, evaluated on the device for
 * n host inputs (FP64): Cody-Waite reduction and a degree-13 Taylor polynomial.  For tests. */
rewl_status rewl_device_exp(const double* x, double* y, int n);

/* Measures this GPU's shared-memory load bandwidth (bytes/s) with a conflict-free 16-byte-load
 * kernel on every SM; the peak the walker kernel's shared-memory traffic is compared against. */
rewl_status rewl_measure_smem_bandwidth(double* bytes_per_s, double* ms, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
