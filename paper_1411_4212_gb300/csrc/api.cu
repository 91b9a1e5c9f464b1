// api.cu -- the C ABI of the REWL library (declared in include/rewl.h): argument checks, the
// lattice geometry and window layout (Sec. 3, Sec. 4.3), device state, and the stream-ordered
// launch sequence of one exchange interval: walker kernel -> exchange kernel -> flatness kernel.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rewl.h"
#include "device_common.cuh"
#include "jobs.h"
#include "walker.h"

using namespace rewl;

// Conflict-table entries of a pipelined walker whose lattice stays in global memory (rewl_autotune
// may pick another size): bcc L = 32 with four shells ran fastest at 2048 entries.  Larger tables
// take shared memory from L1 and fit fewer walkers per SM; smaller ones make sites share entries
// often enough that the extra corrections cost more.
constexpr int kGlobalLatticeOwnEntries = 2048;

struct rewl_handle {
  int kind = 0, L = 0, N = 0, z = 0;
  int B = 0, h = 0, m = 0, W = 0, S = 0;
  double e_min = 0, e_max = 0, dE = 0;
  double overlap = 0, flatness = 0, lnf_final = 0, lnf_initial = 1.0;
  bool traj = false;
  int G = 1;
  uint64_t seed = 0;
  uint32_t key1 = 0;
  long long exchange_interval = 0, max_moves_per_stage = 0, init_cap = 0;
  int recompute_every = 1;
  bool by_window = false;         // window-synchronous iteration (REWL_ITERATION_WINDOW)
  int resolver = REWL_RESOLVER_AUTO;
  double timeout_s = 0;
  cudaStream_t stream = nullptr;
  std::vector<int32_t> starts;
  std::vector<int32_t> tab_nbr;   // [z][N] for chain/table lattices
  std::vector<double> tab_J;
  double E0 = 0;
  Geometry geo{};
  ExpCoeffs ex{};
  bool smem_lattice = false;
  size_t smem_bytes = 0;
  bool pipe = false;              // warp-specialised walker for the Wang-Landau moves
  bool pipe_smem_lattice = false;
  size_t pipe_smem_bytes = 0;
  int own_entries = 0;
  // partitioned handle (rewl_create_partition): hosts windows [k_begin, k_end) of an h-window run at
  // creation; slot states move between the run's handles on accepted cross-handle exchanges
  bool part = false;
  int k_begin = 0, k_end = 0, S_global = 0;
  std::vector<int32_t> gid_host;   // [S] global slot hosted at each position
  std::vector<int32_t> pos_host;   // [S_global] position of each hosted global slot, -1 elsewhere
  int32_t* d_gid = nullptr;
  int32_t* d_pos_of = nullptr;
  int32_t* d_part_bins = nullptr;  // [S_global]
  long long* d_part_lk = nullptr;  // [2 S_global]
  int32_t* d_part_swap = nullptr;  // [S_global]

  void* d_spins = nullptr;
  int32_t* d_perm = nullptr;
  uint32_t* d_H = nullptr;
  long long* d_lng_fx = nullptr;
  long long* d_efx = nullptr;
  long long* d_lnf_fx = nullptr;
  double* d_lng = nullptr;
  double* d_E = nullptr;
  int32_t* d_bin = nullptr;
  double* d_lnf = nullptr;
  int32_t* d_stage = nullptr;
  long long* d_steps = nullptr;
  long long* d_accepts = nullptr;
  long long* d_recomputes = nullptr;
  long long* d_path_batches = nullptr;
  long long* d_init_moves = nullptr;
  double* d_drift = nullptr;
  int32_t* d_ctrl = nullptr;
  WalkerArgs* d_wargs = nullptr;   // pipelined walker over a global-memory lattice: its arguments
  WalkerArgs wargs_host{};         // what d_wargs holds (moves and recompute zeroed)
  bool wargs_valid = false;
  long long* d_ex_index = nullptr;
  int32_t* d_rt_last = nullptr;
  long long* d_rt_count = nullptr;
  unsigned long long* d_ex_att = nullptr;
  unsigned long long* d_ex_acc = nullptr;
  int32_t* d_starts = nullptr;
  int32_t* d_tab_nbr = nullptr;
  float* d_tab_Jf = nullptr;
  double* d_tab_Jd = nullptr;
  double* d_avg = nullptr;
  int32_t* d_bstar = nullptr;
  double* d_merge = nullptr;
  std::vector<void*> allocations;

  bool initialized = false;
  bool broken = false;
  long long intervals_done = 0;
  long long prev_accepts = 0;
  unsigned long long prev_ex_att = 0, prev_ex_acc = 0;
  std::string err;
};

namespace {

thread_local std::string g_last_error;

rewl_status fail(rewl_handle* h, rewl_status s, const std::string& msg) {
  if (h) {
    h->err = msg;
    if (s == REWL_ECUDA) h->broken = true;
  } else {
    g_last_error = msg;
  }
  return s;
}

#define CUDA_TRY(h, call)                                                                       \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail((h), REWL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
  } while (0)

template <class T>
rewl_status dev_alloc(rewl_handle* h, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return fail(h, REWL_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocations.push_back(q);
  *p = static_cast<T*>(q);
  return REWL_OK;
}

// bcc offsets in half lattice units, shell by shell (squared lengths 3, 4, 8, 11), lexicographic
// (dx, dy, dz) inside a shell.  This is the slot order of the local-field sum.
int bcc_offsets(int n_shells, std::vector<std::array<int, 3>>& off, std::vector<int>& shell) {
  static const int r2s[4] = {3, 4, 8, 11};
  off.clear();
  shell.clear();
  for (int sh = 0; sh < n_shells; ++sh)
    for (int dx = -3; dx <= 3; ++dx)
      for (int dy = -3; dy <= 3; ++dy)
        for (int dz = -3; dz <= 3; ++dz) {
          const bool same_parity = ((dx ^ dy) & 1) == 0 && ((dy ^ dz) & 1) == 0;
          if (!same_parity || dx * dx + dy * dy + dz * dz != r2s[sh]) continue;
          off.push_back({dx, dy, dz});
          shell.push_back(sh);
        }
  return (int)off.size();
}

// Luttinger-Tisza ground state of a Bravais lattice: E_gs = -(N/2) max_q sum_r J(r) cos(q.r)
// over wave vectors of the periodic box (half-unit grid n in [0, 2L)^3, q.r = pi n.d / L).
double lt_ground_state(int L, const std::vector<std::array<int, 3>>& off, const std::vector<double>& Jslot) {
  const double pi = 3.14159265358979323846;
  double best = -INFINITY;
  for (int n1 = 0; n1 < 2 * L; ++n1)
    for (int n2 = 0; n2 < 2 * L; ++n2)
      for (int n3 = 0; n3 < 2 * L; ++n3) {
        double jq = 0.0;
        for (size_t j = 0; j < off.size(); ++j) {
          const int dot = n1 * off[j][0] + n2 * off[j][1] + n3 * off[j][2];
          jq = jq + Jslot[j] * std::cos(pi * (double)dot / (double)L);
        }
        if (jq > best) best = jq;
      }
  const double N = 2.0 * (double)L * (double)L * (double)L;
  return -0.5 * N * best;
}

// Window layout (Sec. 4.3): W = ceil(B / (1 + (h-1)(1-o))), start_k = floor(k (B-W)/(h-1) + 1/2).
int window_layout(int B, int h, double o, std::vector<int32_t>& starts) {
  const double denom = 1.0 + (double)(h - 1) * (1.0 - o);
  int W = (int)std::ceil((double)B / denom);
  W = std::min(W, B);
  starts.assign(h, 0);
  for (int k = 0; k < h; ++k)
    starts[k] = h == 1 ? 0 : (int32_t)std::floor((double)k * (double)(B - W) / (double)(h - 1) + 0.5);
  return W;
}

int bin_of(double E, double e_min, double dE) {
  double q = (E - e_min) / dE;
  if (q != q) return -(1 << 30);
  q = std::min(std::max(q, -1073741824.0), 1073741824.0);
  return (int)std::floor(q);
}

WalkerState state_of(rewl_handle* h) {
  WalkerState s{};
  s.spins = h->d_spins;
  s.perm = h->d_perm;
  s.H = h->d_H;
  s.lng_fx = h->d_lng_fx;
  s.efx = h->d_efx;
  s.lnf_fx = h->d_lnf_fx;
  s.lng = h->d_lng;
  s.E = h->d_E;
  s.bin = h->d_bin;
  s.lnf = h->d_lnf;
  s.stage = h->d_stage;
  s.steps = h->d_steps;
  s.accepts = h->d_accepts;
  s.recomputes = h->d_recomputes;
  s.path_batches = h->d_path_batches;
  s.init_moves = h->d_init_moves;
  s.drift = h->d_drift;
  s.ctrl = h->d_ctrl;
  s.ex_index = h->d_ex_index;
  s.rt_last = h->d_rt_last;
  s.rt_count = h->d_rt_count;
  s.ex_att = h->d_ex_att;
  s.ex_acc = h->d_ex_acc;
  s.gid = h->d_gid;
  s.pos_of = h->d_pos_of;
  s.S_global = h->S_global;
  return s;
}

Windows windows_of(rewl_handle* h) {
  Windows w{};
  w.B = h->B;
  w.h = h->h;
  w.m = h->m;
  w.W = h->W;
  w.starts = h->d_starts;
  w.e_min = h->e_min;
  w.dE = h->dE;
  w.dq_scale = (float)(kEnergyScale / h->dE);
  w.dq_scale64 = kEnergyScale / h->dE;
  const double s24 = 16777216.0 / h->dE;
  w.dq24_hi = (float)s24;
  w.dq24_lo = (float)(s24 - (double)w.dq24_hi);
  return w;
}

WalkerArgs walker_args(rewl_handle* h, bool init, bool recompute, long long moves) {
  WalkerArgs a{};
  a.geo = h->geo;
  a.win = windows_of(h);
  a.st = state_of(h);
  a.ex = h->ex;
  a.moves = moves;
  a.init_cap = h->init_cap;
  a.key1 = h->key1;
  a.G = h->G;
  a.init = init ? 1 : 0;
  a.recompute = recompute ? 1 : 0;
  a.lnf_final = h->lnf_final;
  a.own_mask = h->own_entries > 0 ? h->own_entries - 1 : 0;
  a.smem_lattice = (h->pipe ? h->pipe_smem_lattice : h->smem_lattice) ? 1 : 0;
  a.resolver = h->resolver;
  return a;
}

// The Wang-Landau moves of one exchange interval (the initial drive always uses the batch walker).
cudaError_t launch_walk(rewl_handle* h, const WalkerArgs& a) {
  if (h->pipe && h->pipe_smem_lattice)
    return launch_walkers_pipe(a, nullptr, h->S, h->traj, h->pipe_smem_bytes, h->stream);
  if (h->pipe) {
    // the global-memory walker reads its arguments from d_wargs: upload them when they change
    // (the pageable source is staged before the call returns, so wargs_host may change again)
    WalkerArgs s = a;
    s.moves = 0;
    s.recompute = 0;
    if (!h->wargs_valid || std::memcmp(&s, &h->wargs_host, sizeof s) != 0) {
      h->wargs_host = s;
      const cudaError_t e =
          cudaMemcpyAsync(h->d_wargs, &h->wargs_host, sizeof(WalkerArgs), cudaMemcpyHostToDevice, h->stream);
      if (e != cudaSuccess) return e;
      h->wargs_valid = true;
    }
    return launch_walkers_pipe(a, h->d_wargs, h->S, h->traj, h->pipe_smem_bytes, h->stream);
  }
  return launch_walkers(a, h->S, h->traj, h->smem_lattice, h->smem_bytes, h->stream);
}

ExpCoeffs exp_coeffs() {
  ExpCoeffs c{};
  c.inv_fact[0] = 1.0;
  for (int n = 1; n < 14; ++n) c.inv_fact[n] = c.inv_fact[n - 1] / (double)n;
  return c;
}

rewl_status check_ready(rewl_handle* h) {
  if (!h) return fail(nullptr, REWL_EINVAL, "null handle");
  if (h->broken) return fail(h, REWL_ESTATE, "handle saw a CUDA error; destroy it");
  return REWL_OK;
}

int global_of(const rewl_handle* h, int p) { return h->part ? h->gid_host[p] : p; }

// Calls that need every slot of the run in one handle.
rewl_status check_whole(rewl_handle* h) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (h->part)
    return fail(h, REWL_ESTATE,
                "partitioned handle: the replica exchange goes through rewl_partition_exchange and the merge "
                "through rewl_stitch_device on the gathered fragments");
  return REWL_OK;
}

}  // namespace

void rewl::set_handleless_error(const std::string& msg) { g_last_error = msg; }

extern "C" {

const char* rewl_last_error(const rewl_handle* h) {
  if (h) return h->err.c_str();
  return g_last_error.c_str();
}

void rewl_destroy(rewl_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (void* p : h->allocations) cudaFree(p);
  delete h;
}

}  // extern "C"

static rewl_status create_impl(const rewl_lattice* lat, const rewl_couplings* cpl, const rewl_windows* win,
                               int walkers_per_window, double overlap, double flatness, double lnf_final,
                               const rewl_config* cfg, bool part, int k_begin, int k_end, rewl_handle** out) {
  if (!out) return fail(nullptr, REWL_EINVAL, "out is NULL");
  *out = nullptr;
  if (!lat || !cpl || !win || !cfg) return fail(nullptr, REWL_EINVAL, "NULL argument");
  auto* h = new rewl_handle();
  auto bad = [&](const std::string& msg) {
    g_last_error = msg;
    rewl_destroy(h);
    return REWL_EINVAL;
  };
  h->kind = lat->kind;
  h->traj = cfg->mode == REWL_MODE_TRAJECTORY;
  if (cfg->mode != REWL_MODE_TRAJECTORY && cfg->mode != REWL_MODE_PRODUCTION) return bad("unknown mode");
  if (!(overlap >= 0.0 && overlap < 1.0)) return bad("overlap must be in [0, 1)");
  if (!(flatness > 0.0 && flatness < 1.0)) return bad("flatness must be in (0, 1)");
  if (!(lnf_final > 0.0)) return bad("lnf_final must be > 0");
  if (cfg->exchange_interval < 1) return bad("exchange_interval must be >= 1");
  if (walkers_per_window < 1) return bad("walkers_per_window must be >= 1");
  h->overlap = overlap;
  h->flatness = flatness;
  h->lnf_final = lnf_final;
  h->lnf_initial = cfg->lnf_initial > 0.0 ? cfg->lnf_initial : 1.0;
  if (cfg->lnf_initial < 0.0 || cfg->lnf_initial != cfg->lnf_initial) return bad("lnf_initial must be >= 0");
  h->seed = cfg->seed;
  h->key1 = (uint32_t)cfg->seed ^ (uint32_t)(cfg->seed >> 32);
  h->exchange_interval = cfg->exchange_interval;
  h->max_moves_per_stage = cfg->max_moves_per_stage;
  h->init_cap = cfg->init_max_moves > 0 ? cfg->init_max_moves : (1LL << 40);
  h->recompute_every = cfg->recompute_every > 0 ? cfg->recompute_every : (h->traj ? 1 : 8);
  if (cfg->iteration != REWL_ITERATION_WALKER && cfg->iteration != REWL_ITERATION_WINDOW)
    return bad("iteration must be REWL_ITERATION_WALKER or REWL_ITERATION_WINDOW");
  h->by_window = cfg->iteration == REWL_ITERATION_WINDOW;
  if (cfg->resolver < REWL_RESOLVER_AUTO || cfg->resolver > REWL_RESOLVER_SEQUENTIAL)
    return bad("resolver must be REWL_RESOLVER_AUTO, _SCAN, _BLOCKS or _SEQUENTIAL");
  h->resolver = cfg->resolver;
  h->timeout_s = cfg->timeout_s;
  h->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  h->ex = exp_coeffs();

  // ---- lattice ----
  Geometry& g = h->geo;
  std::vector<double> Jslot;
  if (lat->kind == REWL_LATTICE_BCC) {
    if (cpl->n_shells < 1 || cpl->n_shells > 4) return bad("n_shells must be 1..4");
    for (int s = 0; s < cpl->n_shells; ++s)
      if (!std::isfinite(cpl->J[s])) return bad("coupling is not finite");
    std::vector<std::array<int, 3>> off;
    std::vector<int> shell;
    const int z = bcc_offsets(cpl->n_shells, off, shell);
    int maxd = 0;
    for (auto& d : off) maxd = std::max({maxd, std::abs(d[0]), std::abs(d[1]), std::abs(d[2])});
    if (lat->L < 2 || lat->L <= maxd) return bad("L too small for the coupling shells (offset components must be < L/2 cells)");
    if (lat->L > 255) return bad("L must be <= 255");
    h->L = lat->L;
    h->N = 2 * lat->L * lat->L * lat->L;
    h->z = z;
    g.kind = 0;
    g.N = h->N;
    g.z = z;
    g.L = h->L;
    g.divL = (uint32_t)((0x100000000ULL + (unsigned long long)h->L - 1) / (unsigned long long)h->L);
    g.r2max = 0;
    g.n_shells = cpl->n_shells;
    for (int s2 = 0; s2 < 4; ++s2) {
      g.Jsh_d[s2] = s2 < cpl->n_shells ? cpl->J[s2] : 0.0;
      g.Jsh_f[s2] = (float)g.Jsh_d[s2];
    }
    for (int j = 0; j < z; ++j) {
      g.off[j] = (uint32_t)(off[j][0] + 8) | ((uint32_t)(off[j][1] + 8) << 8) | ((uint32_t)(off[j][2] + 8) << 16) |
                 ((uint32_t)shell[j] << 24);
      g.Jd[j] = cpl->J[shell[j]];
      g.Jf[j] = (float)cpl->J[shell[j]];
      g.r2max = std::max(g.r2max, off[j][0] * off[j][0] + off[j][1] * off[j][1] + off[j][2] * off[j][2]);
      Jslot.push_back(cpl->J[shell[j]]);
    }
    // energy recomputation: every bond once = first half of each (centrally symmetric) shell
    g.n_energy_slots = 0;
    int j0 = 0;
    while (j0 < z) {
      int j1 = j0;
      while (j1 < z && shell[j1] == shell[j0]) ++j1;
      for (int j = j0; j < j0 + (j1 - j0) / 2; ++j) g.energy_slot[g.n_energy_slots++] = (uint8_t)j;
      j0 = j1;
    }
    g.energy_weight = 1.0f;
    // E0 = -1/2 sum_i sum_j J_ij for the aligned state, site by site in slot order (production
    // uses the FP32 couplings its energy changes are computed with)
    double acc = 0.0;
    for (int i = 0; i < h->N; ++i) {
      double row = 0.0;
      for (int j = 0; j < z; ++j) row = row + (h->traj ? Jslot[j] : (double)(float)Jslot[j]);
      acc = acc + row;
    }
    h->E0 = -0.5 * acc;
    if (std::isnan(win->e_min) || std::isnan(win->e_max)) {
      h->e_min = lt_ground_state(h->L, off, Jslot);
      h->e_max = 0.0;
    } else {
      h->e_min = win->e_min;
      h->e_max = win->e_max;
    }
  } else if (lat->kind == REWL_LATTICE_CHAIN || lat->kind == REWL_LATTICE_TABLE) {
    int N, z;
    if (lat->kind == REWL_LATTICE_CHAIN) {
      if (lat->L < 2) return bad("chain needs at least 2 spins");
      if (!std::isfinite(cpl->J[0])) return bad("coupling is not finite");
      N = lat->L;
      z = 2;
      h->tab_nbr.resize(2 * (size_t)N);
      h->tab_J.resize(2 * (size_t)N);
      for (int i = 0; i < N; ++i) {   // slot 0 = left, slot 1 = right; open ends: self, J = 0
        h->tab_nbr[i] = i > 0 ? i - 1 : i;
        h->tab_J[i] = i > 0 ? cpl->J[0] : 0.0;
        h->tab_nbr[N + i] = i + 1 < N ? i + 1 : i;
        h->tab_J[N + i] = i + 1 < N ? cpl->J[0] : 0.0;
      }
    } else {
      N = lat->n_sites;
      z = lat->z;
      if (N < 1 || z < 1 || z > kMaxSlotsPerSite || !lat->nbr || !lat->J) return bad("bad table lattice");
      h->tab_nbr.assign(lat->nbr, lat->nbr + (size_t)z * N);
      h->tab_J.assign(lat->J, lat->J + (size_t)z * N);
      for (size_t t = 0; t < h->tab_nbr.size(); ++t) {
        if (h->tab_nbr[t] < 0 || h->tab_nbr[t] >= N) return bad("neighbour index out of range");
        if (!std::isfinite(h->tab_J[t])) return bad("coupling is not finite");
      }
    }
    h->L = lat->L;
    h->N = N;
    h->z = z;
    g.kind = 1;
    g.N = N;
    g.z = z;
    g.L = 0;
    g.n_energy_slots = z;
    for (int j = 0; j < z; ++j) g.energy_slot[j] = (uint8_t)j;
    g.energy_weight = 0.5f;
    double acc = 0.0;
    for (int i = 0; i < N; ++i) {
      double row = 0.0;
      for (int j = 0; j < z; ++j) {
        const double Jij = h->tab_J[(size_t)j * N + i];
        row = row + (h->traj ? Jij : (double)(float)Jij);
      }
      acc = acc + row;
    }
    h->E0 = -0.5 * acc;
    if (std::isnan(win->e_min) || std::isnan(win->e_max)) {
      if (lat->kind == REWL_LATTICE_TABLE) return bad("table lattices need an explicit energy range");
      const double a = std::fabs(cpl->J[0]) * (double)(N - 1);
      h->e_min = -a;
      h->e_max = a;
    } else {
      h->e_min = win->e_min;
      h->e_max = win->e_max;
    }
  } else {
    return bad("unknown lattice kind");
  }
  if (!(std::isfinite(h->e_min) && std::isfinite(h->e_max) && h->e_max > h->e_min)) return bad("empty or NaN energy range");

  // ---- windows ----
  h->B = win->n_bins;
  h->h = win->n_windows;
  h->m = walkers_per_window;
  if (h->B < 2) return bad("n_bins must be >= 2");
  if (h->h < 1 || h->h > h->B) return bad("n_windows must be in [1, n_bins]");
  h->dE = (h->e_max - h->e_min) / (double)h->B;
  h->W = window_layout(h->B, h->h, overlap, h->starts);
  if (h->W < 2) return bad("windows narrower than 2 bins");
  for (int k = 0; k + 1 < h->h; ++k)
    if (h->starts[k] + h->W - h->starts[k + 1] < 2) return bad("adjacent windows overlap by fewer than 2 bins");
  h->S_global = h->h * h->m;
  h->S = h->S_global;
  if (part) {
    if (k_begin < 0 || k_end > h->h || k_begin >= k_end) return bad("partition windows must satisfy 0 <= window_begin < window_end <= n_windows");
    if (h->by_window) return bad("a partitioned run needs REWL_ITERATION_WALKER (a window's walkers may sit in different handles)");
    h->part = true;
    h->k_begin = k_begin;
    h->k_end = k_end;
    h->S = (k_end - k_begin) * h->m;
    h->gid_host.resize(h->S);
    h->pos_host.assign(h->S_global, -1);
    for (int p2 = 0; p2 < h->S; ++p2) {
      h->gid_host[p2] = k_begin * h->m + p2;
      h->pos_host[k_begin * h->m + p2] = p2;
    }
  }

  // ---- lanes per move ----
  if (cfg->group_size == 0) {
    // one lane per move (the warp-specialised walker, 64-move speculation window) when few moves
    // are expected to need re-evaluation: 63 (z+1) / N * (acceptance ~ 1/2) < 1/4; else the batch
    // walker with K = 32/G moves per batch, K ~ sqrt(2 N / (z+1))
    if (lat->kind == REWL_LATTICE_BCC && 63.0 * (h->z + 1.0) / h->N * 0.5 < 0.25) {
      h->G = 1;
    } else {
      const double kk = std::sqrt(2.0 * h->N / (h->z + 1.0));
      int K = 1;
      while (K * 2 <= kk && K < 32) K *= 2;
      h->G = 32 / K;
    }
  } else {
    const int G = cfg->group_size;
    if (G != 1 && G != 2 && G != 4 && G != 8 && G != 16 && G != 32) return bad("group_size must be 0, 1, 2, 4, 8, 16 or 32");
    h->G = G;
  }

  // ---- device ----
  int dev = 0, max_smem = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (ce != cudaSuccess) {
    g_last_error = std::string("CUDA device unavailable: ") + cudaGetErrorString(ce);
    rewl_destroy(h);
    return REWL_ECUDA;
  }
  const size_t with_lattice = walker_smem_bytes(h->traj, true, h->N, h->W);
  h->smem_lattice = with_lattice + 1024 <= (size_t)max_smem;
  h->smem_bytes = walker_smem_bytes(h->traj, h->smem_lattice, h->N, h->W);
  if (h->smem_bytes + 1024 > (size_t)max_smem) return bad("window tables do not fit in shared memory");
  // warp-specialised walker: bcc, one lane per move; owner table as large as the lattice (<= 8192
  // entries), shrunk when the lattice itself occupies shared memory
  // (energy increments travel as int32 in 2^-24 bins: |dE| <= 2 sum_j |J_j| must stay below 100 bins)
  double max_dE = 0.0;
  for (int j = 0; j < h->z && g.kind == 0; ++j) max_dE += 2.0 * std::fabs(g.Jd[j]);
  if (g.kind == 0 && h->G == 1 && max_dE < 100.0 * h->dE) {
    int own_full = 256;
    while (own_full < h->N && own_full < 8192) own_full *= 2;
    const size_t base = walker_pipe_smem_bytes(h->traj, true, h->N, h->W, 0);
    if (base + 1024 + 256 * 8 <= (size_t)max_smem) {
      int e = own_full;
      while (e > 256 && base + 1024 + 8 * (size_t)e > (size_t)max_smem) e /= 2;
      h->own_entries = e;
      h->pipe_smem_lattice = true;
    } else {
      // lattice in global memory: a small table keeps the arena near 20 KB, so several walkers
      // share an SM and most of its unified L1 stays free for the lattice gathers
      h->own_entries = std::min(own_full, kGlobalLatticeOwnEntries);
      h->pipe_smem_lattice = false;
    }
    h->pipe_smem_bytes = walker_pipe_smem_bytes(h->traj, h->pipe_smem_lattice, h->N, h->W, h->own_entries);
    h->pipe = h->pipe_smem_bytes + 1024 <= (size_t)max_smem;
  }

  const size_t S = h->S, W = h->W, N = h->N;
  rewl_status st = REWL_OK;
  auto A = [&](auto** p, size_t count) {
    if (st == REWL_OK) st = dev_alloc(h, p, count);
  };
  // spins: FP64 planes [S][3][N] (trajectory) or octahedral FP32 codes [S][N] float2 (production)
  const size_t spin_bytes = h->traj ? S * 3 * N * sizeof(double) : S * N * sizeof(float2);
  void** spins_pp = &h->d_spins;
  {
    unsigned char* sp = nullptr;
    A(&sp, spin_bytes);
    *spins_pp = sp;
  }
  A(&h->d_perm, S);
  A(&h->d_H, S * W);
  if (h->traj) {
    A(&h->d_lng, S * W);
    A(&h->d_E, S);
    A(&h->d_bin, S);
  } else {
    A(&h->d_lng_fx, S * W);
    A(&h->d_efx, S);
    A(&h->d_lnf_fx, S);
  }
  A(&h->d_lnf, S);
  A(&h->d_stage, S);
  A(&h->d_steps, S);
  A(&h->d_accepts, S);
  A(&h->d_recomputes, S);
  A(&h->d_path_batches, 3 * S);
  A(&h->d_init_moves, S);
  A(&h->d_drift, S);
  A(&h->d_ctrl, 4);
  A(&h->d_wargs, 1);
  A(&h->d_ex_index, 1);
  A(&h->d_rt_last, S);
  A(&h->d_rt_count, S);
  A(&h->d_ex_att, std::max(h->h - 1, 1));
  A(&h->d_ex_acc, std::max(h->h - 1, 1));
  A(&h->d_starts, h->h);
  A(&h->d_avg, (size_t)h->h * W);
  A(&h->d_bstar, std::max(h->h - 1, 1));
  A(&h->d_merge, h->B);
  if (h->part) {
    A(&h->d_gid, S);
    A(&h->d_pos_of, h->S_global);
    A(&h->d_part_bins, h->S_global);
    A(&h->d_part_lk, 2 * (size_t)h->S_global);
    A(&h->d_part_swap, h->S_global);
  }
  if (g.kind == 1) {
    A(&h->d_tab_nbr, (size_t)h->z * N);
    A(&h->d_tab_Jf, (size_t)h->z * N);
    A(&h->d_tab_Jd, (size_t)h->z * N);
  }
  if (st != REWL_OK) {
    rewl_destroy(h);
    return st;
  }
  g.tab_nbr = h->d_tab_nbr;
  g.tab_Jf = h->d_tab_Jf;
  g.tab_Jd = h->d_tab_Jd;

  // ---- initial state: every configuration aligned along +z ----
  auto up = [&](void* d, const void* src, size_t bytes) {
    if (ce == cudaSuccess) ce = cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice);
  };
  auto zero = [&](void* d, size_t bytes) {
    if (ce == cudaSuccess) ce = cudaMemset(d, 0, bytes);
  };
  // every configuration starts aligned along +z: FP64 planes with z = 1, or the code (0, 0)
  if (h->traj) {
    std::vector<unsigned char> sp(spin_bytes, 0);
    const double one = 1.0;
    for (size_t r = 0; r < S; ++r)
      for (size_t i = 0; i < N; ++i) std::memcpy(sp.data() + (r * 3 * N + 2 * N + i) * sizeof(double), &one, sizeof one);
    up(h->d_spins, sp.data(), sp.size());
  } else {
    zero(h->d_spins, spin_bytes);
  }
  std::vector<int32_t> perm(S);
  for (size_t s = 0; s < S; ++s) perm[s] = (int32_t)s;
  up(h->d_perm, perm.data(), S * sizeof(int32_t));
  zero(h->d_H, S * W * sizeof(uint32_t));
  std::vector<double> lnf(S, h->lnf_initial);
  up(h->d_lnf, lnf.data(), S * sizeof(double));
  if (h->traj) {
    zero(h->d_lng, S * W * sizeof(double));
    std::vector<double> E(S, h->E0);
    std::vector<int32_t> b(S, bin_of(h->E0, h->e_min, h->dE));
    up(h->d_E, E.data(), S * sizeof(double));
    up(h->d_bin, b.data(), S * sizeof(int32_t));
  } else {
    zero(h->d_lng_fx, S * W * sizeof(long long));
    std::vector<long long> efx(S, std::llrint((h->E0 - h->e_min) / h->dE * kEnergyScale));
    std::vector<long long> lf(S, std::llrint(h->lnf_initial * kLngScale));
    up(h->d_efx, efx.data(), S * sizeof(long long));
    up(h->d_lnf_fx, lf.data(), S * sizeof(long long));
    for (auto& v : lnf) v = (double)lf[0] * kLngUnit;
    up(h->d_lnf, lnf.data(), S * sizeof(double));
  }
  zero(h->d_stage, S * sizeof(int32_t));
  zero(h->d_steps, S * sizeof(long long));
  zero(h->d_accepts, S * sizeof(long long));
  zero(h->d_recomputes, S * sizeof(long long));
  zero(h->d_path_batches, 3 * S * sizeof(long long));
  zero(h->d_init_moves, S * sizeof(long long));
  zero(h->d_drift, S * sizeof(double));
  zero(h->d_ctrl, 4 * sizeof(int32_t));
  zero(h->d_ex_index, sizeof(long long));
  if (ce == cudaSuccess) ce = cudaMemset(h->d_rt_last, 0xff, S * sizeof(int32_t));   // -1: no extreme seen yet
  zero(h->d_rt_count, S * sizeof(long long));
  zero(h->d_ex_att, std::max(h->h - 1, 1) * sizeof(unsigned long long));
  zero(h->d_ex_acc, std::max(h->h - 1, 1) * sizeof(unsigned long long));
  up(h->d_starts, h->starts.data(), h->h * sizeof(int32_t));
  if (h->part) {
    up(h->d_gid, h->gid_host.data(), S * sizeof(int32_t));
    up(h->d_pos_of, h->pos_host.data(), h->S_global * sizeof(int32_t));
  }
  if (g.kind == 1) {
    std::vector<float> jf(h->tab_J.size());
    for (size_t t = 0; t < jf.size(); ++t) jf[t] = (float)h->tab_J[t];
    up(h->d_tab_nbr, h->tab_nbr.data(), h->tab_nbr.size() * sizeof(int32_t));
    up(h->d_tab_Jf, jf.data(), jf.size() * sizeof(float));
    up(h->d_tab_Jd, h->tab_J.data(), h->tab_J.size() * sizeof(double));
  }
  if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
  if (ce != cudaSuccess) {
    g_last_error = std::string("initial upload: ") + cudaGetErrorString(ce);
    rewl_destroy(h);
    return REWL_ECUDA;
  }
  *out = h;
  return REWL_OK;
}

extern "C" {

rewl_status rewl_create(const rewl_lattice* lat, const rewl_couplings* cpl, const rewl_windows* win,
                        int walkers_per_window, double overlap, double flatness, double lnf_final,
                        const rewl_config* cfg, rewl_handle** out) {
  return create_impl(lat, cpl, win, walkers_per_window, overlap, flatness, lnf_final, cfg, false, 0, 0, out);
}

rewl_status rewl_create_partition(const rewl_lattice* lat, const rewl_couplings* cpl, const rewl_windows* win,
                                  int walkers_per_window, double overlap, double flatness, double lnf_final,
                                  const rewl_config* cfg, int window_begin, int window_end, rewl_handle** out) {
  return create_impl(lat, cpl, win, walkers_per_window, overlap, flatness, lnf_final, cfg, true, window_begin,
                     window_end, out);
}

rewl_status rewl_init_walkers(rewl_handle* h) {
  NvtxRange nvtx_("rewl_init_walkers");
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  const WalkerArgs a = walker_args(h, true, false, 0);
  CUDA_TRY(h, launch_walkers(a, h->S, h->traj, h->smem_lattice, h->smem_bytes, h->stream));
  int32_t ctrl[4];
  CUDA_TRY(h, cudaMemcpyAsync(ctrl, h->d_ctrl, sizeof ctrl, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (ctrl[0] == kErrInitCap) {
    CUDA_TRY(h, cudaMemsetAsync(h->d_ctrl, 0, sizeof(int32_t), h->stream));
    return fail(h, REWL_ETIMEOUT, "initial drive did not reach every window within init_max_moves");
  }
  if (ctrl[0] != kErrNone) return fail(h, REWL_ESTATE, "walker kernel reported error " + std::to_string(ctrl[0]));
  h->initialized = true;
  return REWL_OK;
}

static FlatnessArgs flatness_args(rewl_handle* h) {
  FlatnessArgs fa{};
  fa.win = windows_of(h);
  fa.st = state_of(h);
  fa.flatness = h->flatness;
  fa.lnf_final = h->lnf_final;
  fa.traj = h->traj ? 1 : 0;
  fa.by_window = h->by_window ? 1 : 0;
  return fa;
}

}  // extern "C"

// ---- accessors for the batch runner ----
void rewl::job_view(const rewl_handle* h, JobView* v) {
  v->kind = h->kind;
  v->N = h->N;
  v->z = h->z;
  v->L = h->L;
  v->S = h->S;
  v->W = h->W;
  v->h = h->h;
  v->m = h->m;
  v->n_shells = h->geo.n_shells;
  v->traj = h->traj;
  v->pipe = h->pipe;
  v->initialized = h->initialized;
  v->broken = h->broken;
  v->exchange_interval = h->exchange_interval;
  v->recompute_every = h->recompute_every;
  v->stream = h->stream;
  v->part = h->part;
}

WalkerArgs rewl::job_walker_args(rewl_handle* h, long long moves, int recompute) {
  return walker_args(h, false, recompute != 0, moves);
}

ExchangeArgs rewl::job_exchange_args(rewl_handle* h) {
  ExchangeArgs ea{};
  ea.win = windows_of(h);
  ea.st = state_of(h);
  ea.ex = h->ex;
  ea.key1 = h->key1;
  ea.traj = h->traj ? 1 : 0;
  return ea;
}

FlatnessArgs rewl::job_flatness_args(rewl_handle* h) { return flatness_args(h); }

void rewl::job_add_intervals(rewl_handle* h, long long n) { h->intervals_done += n; }

void rewl::job_couplings(const rewl_handle* h, double J[4], double* e_min, double* dE) {
  for (int s = 0; s < 4; ++s) J[s] = s < h->geo.n_shells ? h->geo.Jsh_d[s] : 0.0;
  *e_min = h->e_min;
  *dE = h->dE;
}

int rewl::job_bins(const rewl_handle* h) { return h->B; }

extern "C" {

rewl_status rewl_walk(rewl_handle* h) {
  NvtxRange nvtx_("rewl_walk");
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (!h->initialized) {
    s = rewl_init_walkers(h);
    if (s != REWL_OK) return s;
  }
  const bool recompute = ((h->intervals_done + 1) % h->recompute_every) == 0;
  const WalkerArgs a = walker_args(h, false, recompute, h->exchange_interval);
  CUDA_TRY(h, launch_walk(h, a));
  h->intervals_done += 1;
  return REWL_OK;
}

rewl_status rewl_autotune(rewl_handle* h, int64_t trial_moves, int32_t* entries_out, double* ms_out) {
  NvtxRange nvtx_("rewl_autotune");
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (trial_moves < 1) return fail(h, REWL_EINVAL, "trial_moves must be > 0");
  if (entries_out) *entries_out = h->pipe ? h->own_entries : 0;
  if (ms_out) *ms_out = 0.0;
  if (!h->pipe) return REWL_OK;
  if (!h->initialized) {
    s = rewl_init_walkers(h);
    if (s != REWL_OK) return s;
  }
  int own_full = 256;
  while (own_full < h->N && own_full < 8192) own_full *= 2;
  int dev = 0, max_smem = 0;
  CUDA_TRY(h, cudaGetDevice(&dev));
  CUDA_TRY(h, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(h, cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  const int e_prev = h->own_entries;
  // two rounds, the second in reverse order; each candidate keeps its faster trial.  With the lattice
  // in shared memory only tables that fit beside it are candidates; a smaller one can fit a second
  // walker per SM.
  std::vector<int> cands;
  for (int c = own_full; c >= 512; c /= 2)
    if (walker_pipe_smem_bytes(h->traj, h->pipe_smem_lattice, h->N, h->W, c) + 1024 <= (size_t)max_smem)
      cands.push_back(c);
  if (cands.size() < 2) {   // nothing to choose between: no trial, no move
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(h, REWL_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
    return REWL_OK;
  }
  std::vector<double> t_min(cands.size(), -1.0);
  for (int round = 0; round < 2 && e == cudaSuccess; ++round) {
    for (size_t k = 0; k < cands.size() && e == cudaSuccess; ++k) {
      const size_t c = round == 0 ? k : cands.size() - 1 - k;
      h->own_entries = cands[c];
      h->pipe_smem_bytes = walker_pipe_smem_bytes(h->traj, h->pipe_smem_lattice, h->N, h->W, cands[c]);
      const WalkerArgs a = walker_args(h, false, false, trial_moves);
      e = cudaEventRecord(e0, h->stream);
      if (e == cudaSuccess) e = launch_walk(h, a);
      if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && (t_min[c] < 0 || ms < t_min[c])) t_min[c] = ms;
    }
  }
  int best_e = e_prev;
  double best = -1.0;
  for (size_t c = 0; c < cands.size(); ++c)
    if (t_min[c] >= 0 && (best < 0 || t_min[c] < best)) {
      best = t_min[c];
      best_e = cands[c];
    }
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  h->own_entries = e == cudaSuccess ? best_e : e_prev;
  h->pipe_smem_bytes = walker_pipe_smem_bytes(h->traj, h->pipe_smem_lattice, h->N, h->W, h->own_entries);
  if (e != cudaSuccess) return fail(h, REWL_ECUDA, std::string("autotune trial: ") + cudaGetErrorString(e));
  int32_t err = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&err, h->d_ctrl, sizeof err, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (err != kErrNone) return fail(h, REWL_ESTATE, "walker kernel reported error " + std::to_string(err));
  if (entries_out) *entries_out = h->own_entries;
  if (ms_out) *ms_out = best;
  return REWL_OK;
}

rewl_status rewl_flatness(rewl_handle* h) {
  NvtxRange nvtx_("rewl_flatness");
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  CUDA_TRY(h, launch_flatness(flatness_args(h), h->S, h->stream));
  return REWL_OK;
}

static rewl_status enqueue_intervals(rewl_handle* h, int n) {
  ExchangeArgs ea{};
  ea.win = windows_of(h);
  ea.st = state_of(h);
  ea.ex = h->ex;
  ea.key1 = h->key1;
  ea.traj = h->traj ? 1 : 0;
  FlatnessArgs fa{};
  fa.win = ea.win;
  fa.st = ea.st;
  fa.flatness = h->flatness;
  fa.lnf_final = h->lnf_final;
  fa.traj = ea.traj;
  fa.by_window = h->by_window ? 1 : 0;
  for (int i = 0; i < n; ++i) {
    const bool recompute = ((h->intervals_done + 1) % h->recompute_every) == 0;
    const WalkerArgs a = walker_args(h, false, recompute, h->exchange_interval);
    CUDA_TRY(h, launch_walk(h, a));
    CUDA_TRY(h, launch_exchange(ea, h->stream));
    CUDA_TRY(h, launch_flatness(fa, h->S, h->stream));
    h->intervals_done += 1;
  }
  return REWL_OK;
}

static rewl_status fill_stats(rewl_handle* h, rewl_stage_stats* out, int intervals, long long moves,
                              int halved, double ms) {
  const size_t S = h->S;
  std::vector<long long> acc(S);
  std::vector<double> lnf(S), drift(S);
  std::vector<unsigned long long> att(std::max(h->h - 1, 1)), ex(std::max(h->h - 1, 1));
  CUDA_TRY(h, cudaMemcpyAsync(acc.data(), h->d_accepts, S * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(lnf.data(), h->d_lnf, S * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(drift.data(), h->d_drift, S * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(att.data(), h->d_ex_att, att.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(ex.data(), h->d_ex_acc, ex.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  long long tot_acc = 0;
  for (auto v : acc) tot_acc += v;
  unsigned long long ta = 0, tx = 0;
  if (h->h > 1)
    for (int k = 0; k < h->h - 1; ++k) {
      ta += att[k];
      tx += ex[k];
    }
  if (out) {
    std::memset(out, 0, sizeof *out);
    out->moves = moves;
    out->accepts = tot_acc - h->prev_accepts;
    out->exchange_attempts = (long long)(ta - h->prev_ex_att);
    out->exchange_accepts = (long long)(tx - h->prev_ex_acc);
    out->intervals = intervals;
    out->n_halved = halved;
    int done = 0;
    double mn = INFINITY, mx = -INFINITY, dr = 0;
    for (size_t s = 0; s < S; ++s) {
      if (!(lnf[s] >= h->lnf_final)) ++done;
      mn = std::min(mn, lnf[s]);
      mx = std::max(mx, lnf[s]);
      dr = std::max(dr, drift[s]);
    }
    out->n_done = done;
    out->all_done = done == (int)S;
    out->min_lnf = mn;
    out->max_lnf = mx;
    out->max_energy_drift = dr;
    out->elapsed_ms = ms;
  }
  h->prev_accepts = tot_acc;
  h->prev_ex_att = ta;
  h->prev_ex_acc = tx;
  return REWL_OK;
}

static rewl_status read_stage(rewl_handle* h, std::vector<int32_t>& stage, std::vector<double>& lnf) {
  stage.resize(h->S);
  lnf.resize(h->S);
  CUDA_TRY(h, cudaMemcpyAsync(stage.data(), h->d_stage, h->S * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(lnf.data(), h->d_lnf, h->S * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return REWL_OK;
}

rewl_status rewl_run_intervals(rewl_handle* h, int n, rewl_stage_stats* stats) {
  NvtxRange nvtx_("rewl_run_intervals");
  rewl_status s = check_whole(h);
  if (s != REWL_OK) return s;
  if (n < 0) return fail(h, REWL_EINVAL, "n_intervals must be >= 0");
  if (!h->initialized) {
    s = rewl_init_walkers(h);
    if (s != REWL_OK) return s;
  }
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<int32_t> st0, st1;
  std::vector<double> l0, l1;
  if (stats) {
    s = read_stage(h, st0, l0);
    if (s != REWL_OK) return s;
  }
  s = enqueue_intervals(h, n);
  if (s != REWL_OK) return s;
  if (stats) {
    s = read_stage(h, st1, l1);
    if (s != REWL_OK) return s;
    int halved = 0;
    for (int i = 0; i < h->S; ++i) halved += st1[i] - st0[i];
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return fill_stats(h, stats, n, (long long)n * h->exchange_interval * h->S, halved, ms);
  }
  return REWL_OK;
}

rewl_status rewl_run_stage(rewl_handle* h, rewl_stage_stats* stats) {
  NvtxRange nvtx_("rewl_run_stage");
  rewl_status s = check_whole(h);
  if (s != REWL_OK) return s;
  if (!h->initialized) {
    s = rewl_init_walkers(h);
    if (s != REWL_OK) return s;
  }
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<int32_t> st0, st;
  std::vector<double> l0, l;
  s = read_stage(h, st0, l0);
  if (s != REWL_OK) return s;
  long long moves_per_walker = 0;
  int intervals = 0;
  bool capped = false;
  // check the flags every few intervals; the chunk grows with ln f-halving time
  int chunk = 4;
  while (true) {
    s = enqueue_intervals(h, chunk);
    if (s != REWL_OK) return s;
    intervals += chunk;
    moves_per_walker += (long long)chunk * h->exchange_interval;
    s = read_stage(h, st, l);
    if (s != REWL_OK) return s;
    bool all = true;
    for (int i = 0; i < h->S; ++i)
      if (l0[i] >= h->lnf_final && st[i] <= st0[i]) all = false;
    if (all) break;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if ((h->max_moves_per_stage > 0 && moves_per_walker >= h->max_moves_per_stage) ||
        (h->timeout_s > 0 && secs >= h->timeout_s)) {
      capped = true;
      break;
    }
    chunk = std::min(chunk * 2, 64);
  }
  int halved = 0;
  for (int i = 0; i < h->S; ++i) halved += st[i] - st0[i];
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  s = fill_stats(h, stats, intervals, moves_per_walker * h->S, halved, ms);
  if (s != REWL_OK) return s;
  if (capped) return fail(h, REWL_ETIMEOUT, "stage ended by max_moves_per_stage or timeout_s");
  return REWL_OK;
}

rewl_status rewl_exchange(rewl_handle* h, rewl_stage_stats* stats) {
  NvtxRange nvtx_("rewl_exchange");
  rewl_status s = check_whole(h);
  if (s != REWL_OK) return s;
  if (!h->initialized) {
    s = rewl_init_walkers(h);
    if (s != REWL_OK) return s;
  }
  ExchangeArgs ea{};
  ea.win = windows_of(h);
  ea.st = state_of(h);
  ea.ex = h->ex;
  ea.key1 = h->key1;
  ea.traj = h->traj ? 1 : 0;
  CUDA_TRY(h, launch_exchange(ea, h->stream));
  if (stats) return fill_stats(h, stats, 0, 0, 0, 0.0);
  return REWL_OK;
}

static MergeArgs merge_args(rewl_handle* h, double* out) {
  MergeArgs a{};
  a.frag = h->traj ? h->d_lng : nullptr;
  a.frag_fx = h->traj ? nullptr : h->d_lng_fx;
  a.starts = h->d_starts;
  a.h = h->h;
  a.m = h->m;
  a.W = h->W;
  a.B = h->B;
  a.avg = h->d_avg;
  a.bstar = h->d_bstar;
  a.out = out;
  return a;
}

rewl_status rewl_merge_lng_device(rewl_handle* h, double* out) {
  NvtxRange nvtx_("rewl_merge_lng_device");
  rewl_status s = check_whole(h);
  if (s != REWL_OK) return s;
  if (!out) return fail(h, REWL_EINVAL, "lng_out_dev is NULL");
  CUDA_TRY(h, launch_merge(merge_args(h, out), h->stream));
  return REWL_OK;
}

rewl_status rewl_merge_lng(rewl_handle* h, double* lng_out, double* centres) {
  NvtxRange nvtx_("rewl_merge_lng");
  rewl_status s = check_whole(h);
  if (s != REWL_OK) return s;
  if (!lng_out) return fail(h, REWL_EINVAL, "lng_out is NULL");
  CUDA_TRY(h, launch_merge(merge_args(h, h->d_merge), h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(lng_out, h->d_merge, h->B * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (centres)
    for (int b = 0; b < h->B; ++b) centres[b] = h->e_min + ((double)b + 0.5) * h->dE;
  return REWL_OK;
}

rewl_status rewl_stitch_device(const double* frag, const int32_t* starts_host, int n_windows, int m, int W,
                               int B, double* out, int32_t* bstar_out, void* cuda_stream) {
  if (!frag || !starts_host || !out) return fail(nullptr, REWL_EINVAL, "NULL argument");
  if (n_windows < 1 || m < 1 || W < 3 || B < W) return fail(nullptr, REWL_EINVAL, "bad sizes");
  for (int k = 0; k < n_windows; ++k) {
    if (starts_host[k] < 0 || starts_host[k] + W > B) return fail(nullptr, REWL_EINVAL, "window outside [0, B)");
    if (k > 0 && starts_host[k] <= starts_host[k - 1]) return fail(nullptr, REWL_EINVAL, "window starts must increase");
    if (k > 0 && starts_host[k - 1] + W - starts_host[k] < 2)
      return fail(nullptr, REWL_EINVAL, "adjacent windows must overlap by at least 2 bins");
  }
  if (starts_host[0] != 0 || starts_host[n_windows - 1] + W != B)
    return fail(nullptr, REWL_EINVAL, "windows must cover [0, B): starts[0] = 0 and starts[h-1] + W = B");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  MergeArgs a{};
  a.frag = frag;
  a.h = n_windows;
  a.m = m;
  a.W = W;
  a.B = B;
  a.out = out;
  int32_t* d_starts = nullptr;
  double* d_avg = nullptr;
  int32_t* d_bstar = nullptr;
  cudaError_t e = cudaMallocAsync(&d_starts, sizeof(int32_t) * n_windows, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_avg, sizeof(double) * (size_t)n_windows * W, st);
  if (e == cudaSuccess && !bstar_out) e = cudaMallocAsync(&d_bstar, sizeof(int32_t) * std::max(n_windows - 1, 1), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_starts, starts_host, sizeof(int32_t) * n_windows, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    a.starts = d_starts;
    a.avg = d_avg;
    a.bstar = bstar_out ? bstar_out : d_bstar;
    e = launch_merge(a, st);
  }
  if (d_starts) cudaFreeAsync(d_starts, st);
  if (d_avg) cudaFreeAsync(d_avg, st);
  if (d_bstar) cudaFreeAsync(d_bstar, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, REWL_ECUDA, std::string("stitch: ") + cudaGetErrorString(e));
  return REWL_OK;
}

rewl_status rewl_thermo(const double* lng, const double* centres, int B, double n_spins, const double* T, int nT,
                        double* U, double* C, double* lnZ, void* cuda_stream) {
  if (!lng || !centres || !T || B < 1 || nT < 1 || !(n_spins > 0)) return fail(nullptr, REWL_EINVAL, "bad thermo arguments");
  for (int i = 0; i < nT; ++i)
    if (!(T[i] > 0)) return fail(nullptr, REWL_EINVAL, "temperatures must be > 0");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double* d = nullptr;
  const size_t bytes = sizeof(double) * (2 * (size_t)B + 4 * (size_t)nT);
  cudaError_t e = cudaMallocAsync(&d, bytes, st);
  if (e != cudaSuccess) return fail(nullptr, REWL_ENOMEM, "thermo scratch allocation failed");
  double *dl = d, *dE = d + B, *dT = d + 2 * B, *dU = dT + nT, *dC = dU + nT, *dZ = dC + nT;
  e = cudaMemcpyAsync(dl, lng, sizeof(double) * B, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dE, centres, sizeof(double) * B, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dT, T, sizeof(double) * nT, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_thermo(dl, dE, B, n_spins, dT, nT, dU, dC, dZ, st);
  if (e == cudaSuccess && U) e = cudaMemcpyAsync(U, dU, sizeof(double) * nT, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && C) e = cudaMemcpyAsync(C, dC, sizeof(double) * nT, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && lnZ) e = cudaMemcpyAsync(lnZ, dZ, sizeof(double) * nT, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, REWL_ECUDA, std::string("thermo: ") + cudaGetErrorString(e));
  return REWL_OK;
}

rewl_status rewl_peak_temperature(const double* T, const double* C, int nT, double* T_peak, void* cuda_stream) {
  if (!T || !C || !T_peak || nT < 1) return fail(nullptr, REWL_EINVAL, "bad peak arguments");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, sizeof(double) * (2 * (size_t)nT + 1), st);
  if (e != cudaSuccess) return fail(nullptr, REWL_ENOMEM, "peak scratch allocation failed");
  e = cudaMemcpyAsync(d, T, sizeof(double) * nT, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + nT, C, sizeof(double) * nT, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_peak(d, d + nT, nT, d + 2 * nT, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(T_peak, d + 2 * nT, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, REWL_ECUDA, std::string("peak: ") + cudaGetErrorString(e));
  return REWL_OK;
}

rewl_status rewl_set_initial_lng(rewl_handle* h, const double* lng, double lnf0) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (!lng || !(lnf0 > 0)) return fail(h, REWL_EINVAL, "lng must be non-NULL and lnf0 > 0");
  for (int b = 0; b < h->B; ++b)
    if (!std::isfinite(lng[b])) return fail(h, REWL_EINVAL, "lng has a non-finite entry");
  const size_t S = h->S, W = h->W;
  std::vector<double> lnf(S, lnf0);
  if (h->traj) {
    std::vector<double> t(S * W);
    for (size_t s2 = 0; s2 < S; ++s2)
      for (size_t w = 0; w < W; ++w) t[s2 * W + w] = lng[h->starts[global_of(h, (int)s2) / h->m] + w];
    CUDA_TRY(h, cudaMemcpyAsync(h->d_lng, t.data(), S * W * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  } else {
    std::vector<long long> t(S * W);
    for (size_t s2 = 0; s2 < S; ++s2)
      for (size_t w = 0; w < W; ++w) t[s2 * W + w] = std::llrint(lng[h->starts[global_of(h, (int)s2) / h->m] + w] * kLngScale);
    std::vector<long long> lf(S, std::llrint(lnf0 * kLngScale));
    for (auto& v : lnf) v = (double)lf[0] * kLngUnit;
    CUDA_TRY(h, cudaMemcpyAsync(h->d_lng_fx, t.data(), S * W * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_lnf_fx, lf.data(), S * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  CUDA_TRY(h, cudaMemcpyAsync(h->d_lnf, lnf.data(), S * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->d_H, 0, S * W * sizeof(uint32_t), h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->d_stage, 0, S * sizeof(int32_t), h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return REWL_OK;
}

rewl_status rewl_get_info(const rewl_handle* hc, rewl_info* out) {
  if (!hc || !out) return fail(nullptr, REWL_EINVAL, "NULL argument");
  rewl_handle* h = const_cast<rewl_handle*>(hc);
  std::memset(out, 0, sizeof *out);
  out->n_sites = h->N;
  out->z = h->z;
  out->n_slots = h->S;
  out->n_replicas = h->S;
  out->n_bins = h->B;
  out->n_windows = h->h;
  out->walkers_per_window = h->m;
  out->window_bins = h->W;
  out->group_size = h->G;
  out->mode = h->traj ? REWL_MODE_TRAJECTORY : REWL_MODE_PRODUCTION;
  out->e_min = h->e_min;
  out->e_max = h->e_max;
  out->bin_width = h->dE;
  out->initial_energy = h->E0;
  long long ex = 0;
  if (!h->broken && cudaMemcpy(&ex, h->d_ex_index, sizeof ex, cudaMemcpyDeviceToHost) != cudaSuccess) ex = -1;
  out->exchange_index = ex;
  out->intervals_done = h->intervals_done;
  out->shared_bytes_per_walker = h->pipe ? h->pipe_smem_bytes : h->smem_bytes;
  out->lattice_in_shared = (h->pipe ? h->pipe_smem_lattice : h->smem_lattice) ? 1 : 0;
  out->pipelined = h->pipe ? 1 : 0;
  out->conflict_entries = h->pipe ? h->own_entries : 0;
  return REWL_OK;
}

rewl_status rewl_get_walkers(rewl_handle* h, double* lng, uint32_t* H, double* E, int32_t* bin, double* lnf,
                             int32_t* replica, int32_t* stage, int64_t* accepts, int64_t* steps, int64_t* init_moves) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  const size_t S = h->S, W = h->W;
  cudaStream_t st = h->stream;
  if (lng) {
    if (h->traj) {
      CUDA_TRY(h, cudaMemcpyAsync(lng, h->d_lng, S * W * sizeof(double), cudaMemcpyDeviceToHost, st));
    } else {
      std::vector<long long> t(S * W);
      CUDA_TRY(h, cudaMemcpyAsync(t.data(), h->d_lng_fx, S * W * sizeof(long long), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(h, cudaStreamSynchronize(st));
      for (size_t i = 0; i < S * W; ++i) lng[i] = (double)t[i] * kLngUnit;
    }
  }
  if (H) CUDA_TRY(h, cudaMemcpyAsync(H, h->d_H, S * W * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  if (E || bin) {
    std::vector<double> e(S);
    std::vector<int32_t> b(S);
    if (h->traj) {
      CUDA_TRY(h, cudaMemcpyAsync(e.data(), h->d_E, S * sizeof(double), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(h, cudaMemcpyAsync(b.data(), h->d_bin, S * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(h, cudaStreamSynchronize(st));
    } else {
      std::vector<long long> f(S);
      CUDA_TRY(h, cudaMemcpyAsync(f.data(), h->d_efx, S * sizeof(long long), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(h, cudaStreamSynchronize(st));
      for (size_t i = 0; i < S; ++i) {
        e[i] = h->e_min + h->dE * ((double)f[i] / kEnergyScale);
        b[i] = (int32_t)(f[i] >> 32);
      }
    }
    if (E) std::memcpy(E, e.data(), S * sizeof(double));
    if (bin) std::memcpy(bin, b.data(), S * sizeof(int32_t));
  }
  if (lnf) CUDA_TRY(h, cudaMemcpyAsync(lnf, h->d_lnf, S * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (replica) CUDA_TRY(h, cudaMemcpyAsync(replica, h->d_perm, S * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (stage) CUDA_TRY(h, cudaMemcpyAsync(stage, h->d_stage, S * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (accepts) CUDA_TRY(h, cudaMemcpyAsync(accepts, h->d_accepts, S * sizeof(long long), cudaMemcpyDeviceToHost, st));
  if (steps) CUDA_TRY(h, cudaMemcpyAsync(steps, h->d_steps, S * sizeof(long long), cudaMemcpyDeviceToHost, st));
  if (init_moves) CUDA_TRY(h, cudaMemcpyAsync(init_moves, h->d_init_moves, S * sizeof(long long), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaStreamSynchronize(st));
  return REWL_OK;
}

rewl_status rewl_get_spins(rewl_handle* h, double* spins) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (!spins) return fail(h, REWL_EINVAL, "spins is NULL");
  const size_t n = (size_t)h->S * 3 * h->N;
  if (h->traj) {
    CUDA_TRY(h, cudaMemcpyAsync(spins, h->d_spins, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  } else {
    // device codes -> the FP32 spins the walkers see (decoded on the device) -> host FP64 planes
    float* d = nullptr;
    std::vector<float> t(n);
    CUDA_TRY(h, cudaMallocAsync(&d, n * sizeof(float), h->stream));
    CUDA_TRY(h, launch_decode_spins(static_cast<const float2*>(h->d_spins), (size_t)h->S, h->N, d, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(t.data(), d, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaFreeAsync(d, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < n; ++i) spins[i] = t[i];
  }
  return REWL_OK;
}

rewl_status rewl_get_exchange_counts(rewl_handle* h, int64_t* attempts, int64_t* accepts) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (h->h < 2) return REWL_OK;
  const size_t n = h->h - 1;
  if (attempts) CUDA_TRY(h, cudaMemcpyAsync(attempts, h->d_ex_att, n * 8, cudaMemcpyDeviceToHost, h->stream));
  if (accepts) CUDA_TRY(h, cudaMemcpyAsync(accepts, h->d_ex_acc, n * 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return REWL_OK;
}

rewl_status rewl_get_round_trips(rewl_handle* h, int64_t* counts, int32_t* last) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  const size_t S = h->S;
  if (counts) CUDA_TRY(h, cudaMemcpyAsync(counts, h->d_rt_count, S * 8, cudaMemcpyDeviceToHost, h->stream));
  if (last) CUDA_TRY(h, cudaMemcpyAsync(last, h->d_rt_last, S * 4, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return REWL_OK;
}

rewl_status rewl_get_counters(rewl_handle* h, rewl_counters* out) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (!out) return fail(h, REWL_EINVAL, "out is NULL");
  const size_t S = h->S;
  std::vector<long long> a(S), st(S), r(S), pb(3 * S);
  CUDA_TRY(h, cudaMemcpyAsync(a.data(), h->d_accepts, S * 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(st.data(), h->d_steps, S * 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(r.data(), h->d_recomputes, S * 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(pb.data(), h->d_path_batches, 3 * S * 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  std::memset(out, 0, sizeof *out);
  for (size_t i = 0; i < S; ++i) {
    out->moves += st[i];
    out->accepts += a[i];
    out->recomputes += r[i];
    out->batches_scan += pb[3 * i];
    out->batches_blocks += pb[3 * i + 1];
    out->batches_sequential += pb[3 * i + 2];
  }
  return REWL_OK;
}

rewl_status rewl_get_neighbours(rewl_handle* h, int32_t* nbr, double* J) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (!nbr || !J) return fail(h, REWL_EINVAL, "NULL argument");
  const size_t n = (size_t)h->z * h->N;
  int32_t* dn = nullptr;
  double* dj = nullptr;
  CUDA_TRY(h, cudaMallocAsync(&dn, n * sizeof(int32_t), h->stream));
  CUDA_TRY(h, cudaMallocAsync(&dj, n * sizeof(double), h->stream));
  CUDA_TRY(h, launch_neighbour_dump(h->geo, dn, dj, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(nbr, dn, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(J, dj, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaFreeAsync(dn, h->stream));
  CUDA_TRY(h, cudaFreeAsync(dj, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return REWL_OK;
}

rewl_status rewl_replica_energies(rewl_handle* h, double* E) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (!E) return fail(h, REWL_EINVAL, "E is NULL");
  double* d = nullptr;
  CUDA_TRY(h, cudaMallocAsync(&d, h->S * sizeof(double), h->stream));
  const WalkerArgs a = walker_args(h, false, false, 0);
  CUDA_TRY(h, launch_energies(a, h->S, h->traj, d, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(E, d, h->S * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaFreeAsync(d, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return REWL_OK;
}

// ---- partitioned runs ----------------------------------------------------------------------------
// Slot state (rewl_slot_export): int64 words
//   [0] tag, [1] global slot, [2] W, [3] mode, [4] ln f (FP64 bits), [5] ln f (2^-40 fixed point),
//   [6] stage, [7] trial moves done (the Philox counter), [8] accepts, [9] corrections, [10] moves of
//   the initial drive, [11] largest energy drift (FP64 bits), [12..14] batches per resolver path,
//   [15 .. 15+W) ln g (fixed point or FP64 bits), then H packed two u32 per word.
constexpr long long kSlotTag = 0x5245574c534c4f54LL;   // "REWLSLOT"
constexpr int kSlotHead = 15;

static int64_t slot_words(const rewl_handle* h) { return kSlotHead + h->W + (h->W + 1) / 2; }

static ExchangeArgs exchange_args(rewl_handle* h) {
  ExchangeArgs ea{};
  ea.win = windows_of(h);
  ea.st = state_of(h);
  ea.ex = h->ex;
  ea.key1 = h->key1;
  ea.traj = h->traj ? 1 : 0;
  if (h->part) {
    ea.part_bin_all = h->d_part_bins;
    ea.part_lk_all = h->d_part_lk;
    ea.part_swap_with = h->d_part_swap;
  }
  return ea;
}

static rewl_status check_part(rewl_handle* h) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (!h->part) return fail(h, REWL_ESTATE, "not a partitioned handle (rewl_create_partition)");
  if (!h->initialized) return fail(h, REWL_ESTATE, "walkers not initialised (rewl_init_walkers)");
  return REWL_OK;
}

rewl_status rewl_partition_slots(rewl_handle* h, int32_t* gid) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (!gid) return fail(h, REWL_EINVAL, "gid is NULL");
  for (int p2 = 0; p2 < h->S; ++p2) gid[p2] = global_of(h, p2);
  return REWL_OK;
}

rewl_status rewl_partition_bins(rewl_handle* h, int32_t* bins) {
  NvtxRange nvtx_("rewl_partition_bins");
  rewl_status s = check_part(h);
  if (s != REWL_OK) return s;
  if (!bins) return fail(h, REWL_EINVAL, "bins is NULL");
  std::vector<int32_t> t(h->S_global);
  CUDA_TRY(h, launch_partition_bins(exchange_args(h), h->S, h->d_part_bins, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(t.data(), h->d_part_bins, h->S_global * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  for (int p2 = 0; p2 < h->S; ++p2) bins[h->gid_host[p2]] = t[h->gid_host[p2]];
  return REWL_OK;
}

rewl_status rewl_partition_lookups(rewl_handle* h, const int32_t* bins_all, int64_t* lk) {
  NvtxRange nvtx_("rewl_partition_lookups");
  rewl_status s = check_part(h);
  if (s != REWL_OK) return s;
  if (!bins_all || !lk) return fail(h, REWL_EINVAL, "NULL argument");
  std::vector<long long> t(2 * (size_t)h->S_global);
  CUDA_TRY(h, cudaMemcpyAsync(h->d_part_bins, bins_all, h->S_global * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->d_part_lk, 0, t.size() * sizeof(long long), h->stream));
  CUDA_TRY(h, launch_partition_lookups(exchange_args(h), h->d_part_bins, h->d_part_lk, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(t.data(), h->d_part_lk, t.size() * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  for (int p2 = 0; p2 < h->S; ++p2) {
    const int g = h->gid_host[p2];
    lk[2 * g] = t[2 * (size_t)g];
    lk[2 * g + 1] = t[2 * (size_t)g + 1];
  }
  return REWL_OK;
}

rewl_status rewl_partition_exchange(rewl_handle* h, const int32_t* bins_all, const int64_t* lk_all, int32_t* swap_with) {
  NvtxRange nvtx_("rewl_partition_exchange");
  rewl_status s = check_part(h);
  if (s != REWL_OK) return s;
  if (!bins_all || !lk_all || !swap_with) return fail(h, REWL_EINVAL, "NULL argument");
  const size_t S = h->S_global;
  CUDA_TRY(h, cudaMemcpyAsync(h->d_part_bins, bins_all, S * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_part_lk, lk_all, 2 * S * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->d_part_swap, 0xff, S * sizeof(int32_t), h->stream));
  CUDA_TRY(h, launch_exchange(exchange_args(h), h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(swap_with, h->d_part_swap, S * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return REWL_OK;
}

rewl_status rewl_partition_observe(rewl_handle* h) {
  rewl_status s = check_part(h);
  if (s != REWL_OK) return s;
  CUDA_TRY(h, launch_partition_observe(exchange_args(h), h->stream));
  return REWL_OK;
}

rewl_status rewl_slot_state_bytes(rewl_handle* h, int64_t* bytes) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (!bytes) return fail(h, REWL_EINVAL, "bytes is NULL");
  *bytes = slot_words(h) * 8;
  return REWL_OK;
}

rewl_status rewl_slot_export(rewl_handle* h, int32_t g, void* buf) {
  NvtxRange nvtx_("rewl_slot_export");
  rewl_status s = check_part(h);
  if (s != REWL_OK) return s;
  if (!buf || g < 0 || g >= h->S_global || h->pos_host[g] < 0) return fail(h, REWL_EINVAL, "slot not hosted here or NULL buffer");
  const int p2 = h->pos_host[g];
  const size_t W = h->W;
  std::vector<long long> w(slot_words(h), 0);
  std::vector<uint32_t> H(W);
  double lnf = 0, drift = 0;
  long long lnf_fx = 0, steps = 0, acc = 0, rec = 0, init = 0, pb[3] = {0, 0, 0};
  int32_t stage = 0;
  cudaStream_t st = h->stream;
  CUDA_TRY(h, cudaMemcpyAsync(&lnf, h->d_lnf + p2, 8, cudaMemcpyDeviceToHost, st));
  if (!h->traj) CUDA_TRY(h, cudaMemcpyAsync(&lnf_fx, h->d_lnf_fx + p2, 8, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(&stage, h->d_stage + p2, 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(&steps, h->d_steps + p2, 8, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(&acc, h->d_accepts + p2, 8, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(&rec, h->d_recomputes + p2, 8, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(&init, h->d_init_moves + p2, 8, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(&drift, h->d_drift + p2, 8, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(pb, h->d_path_batches + 3 * (size_t)p2, 24, cudaMemcpyDeviceToHost, st));
  if (h->traj)
    CUDA_TRY(h, cudaMemcpyAsync(w.data() + kSlotHead, h->d_lng + (size_t)p2 * W, W * 8, cudaMemcpyDeviceToHost, st));
  else
    CUDA_TRY(h, cudaMemcpyAsync(w.data() + kSlotHead, h->d_lng_fx + (size_t)p2 * W, W * 8, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(H.data(), h->d_H + (size_t)p2 * W, W * 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaStreamSynchronize(st));
  w[0] = kSlotTag;
  w[1] = g;
  w[2] = (long long)W;
  w[3] = h->traj ? 1 : 0;
  std::memcpy(&w[4], &lnf, 8);
  w[5] = lnf_fx;
  w[6] = stage;
  w[7] = steps;
  w[8] = acc;
  w[9] = rec;
  w[10] = init;
  std::memcpy(&w[11], &drift, 8);
  w[12] = pb[0];
  w[13] = pb[1];
  w[14] = pb[2];
  std::memcpy(w.data() + kSlotHead + W, H.data(), W * 4);
  std::memcpy(buf, w.data(), w.size() * 8);
  return REWL_OK;
}

rewl_status rewl_slot_import(rewl_handle* h, int32_t g_out, const void* buf) {
  NvtxRange nvtx_("rewl_slot_import");
  rewl_status s = check_part(h);
  if (s != REWL_OK) return s;
  if (!buf || g_out < 0 || g_out >= h->S_global || h->pos_host[g_out] < 0)
    return fail(h, REWL_EINVAL, "slot not hosted here or NULL buffer");
  const size_t W = h->W;
  std::vector<long long> w(slot_words(h));
  std::memcpy(w.data(), buf, w.size() * 8);
  const long long g_in = w[1];
  if (w[0] != kSlotTag || w[2] != (long long)W || w[3] != (h->traj ? 1 : 0))
    return fail(h, REWL_EINVAL, "buffer is not a slot state of this run (tag, window size or mode differ)");
  if (g_in < 0 || g_in >= h->S_global || (g_in != g_out && h->pos_host[g_in] >= 0))
    return fail(h, REWL_EINVAL, "incoming slot is out of range or already hosted here");
  const int p2 = h->pos_host[g_out];
  double lnf, drift;
  std::memcpy(&lnf, &w[4], 8);
  std::memcpy(&drift, &w[11], 8);
  const int32_t stage = (int32_t)w[6], gi = (int32_t)g_in, none = -1;
  cudaStream_t st = h->stream;
  CUDA_TRY(h, cudaMemcpyAsync(h->d_lnf + p2, &lnf, 8, cudaMemcpyHostToDevice, st));
  if (!h->traj) CUDA_TRY(h, cudaMemcpyAsync(h->d_lnf_fx + p2, &w[5], 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_stage + p2, &stage, 4, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_steps + p2, &w[7], 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_accepts + p2, &w[8], 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_recomputes + p2, &w[9], 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_init_moves + p2, &w[10], 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_drift + p2, &drift, 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_path_batches + 3 * (size_t)p2, &w[12], 24, cudaMemcpyHostToDevice, st));
  if (h->traj)
    CUDA_TRY(h, cudaMemcpyAsync(h->d_lng + (size_t)p2 * W, w.data() + kSlotHead, W * 8, cudaMemcpyHostToDevice, st));
  else
    CUDA_TRY(h, cudaMemcpyAsync(h->d_lng_fx + (size_t)p2 * W, w.data() + kSlotHead, W * 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_H + (size_t)p2 * W, w.data() + kSlotHead + W, W * 4, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_gid + p2, &gi, 4, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_pos_of + g_out, &none, 4, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_pos_of + gi, &p2, 4, cudaMemcpyHostToDevice, st));
  // the pageable sources above are stack and vector memory: wait before they go out of scope
  CUDA_TRY(h, cudaStreamSynchronize(st));
  h->pos_host[g_out] = -1;
  h->pos_host[gi] = p2;
  h->gid_host[p2] = gi;
  h->wargs_valid = false;
  return REWL_OK;
}

// ---- checkpoints --------------------------------------------------------------------------------
// Layout: header (tag, version, total bytes, fingerprint of the run's arguments, host counters),
// then every device state array in a fixed order, then a checksum of everything before it.
constexpr unsigned long long kCkptTag = 0x5245574c434b5054ULL;   // "REWLCKPT"
constexpr long long kCkptVersion = 1;
constexpr int kCkptHead = 10;   // int64 words

struct Section {
  void* dev;
  size_t bytes;
};

static std::vector<Section> state_sections(rewl_handle* h) {
  const size_t S = h->S, W = h->W, N = h->N, X = (size_t)std::max(h->h - 1, 1);
  std::vector<Section> v;
  v.push_back({h->d_spins, h->traj ? S * 3 * N * sizeof(double) : S * N * sizeof(float2)});
  v.push_back({h->d_perm, S * 4});
  v.push_back({h->d_H, S * W * 4});
  if (h->traj) {
    v.push_back({h->d_lng, S * W * 8});
    v.push_back({h->d_E, S * 8});
    v.push_back({h->d_bin, S * 4});
  } else {
    v.push_back({h->d_lng_fx, S * W * 8});
    v.push_back({h->d_efx, S * 8});
    v.push_back({h->d_lnf_fx, S * 8});
  }
  v.push_back({h->d_lnf, S * 8});
  v.push_back({h->d_stage, S * 4});
  v.push_back({h->d_steps, S * 8});
  v.push_back({h->d_accepts, S * 8});
  v.push_back({h->d_recomputes, S * 8});
  v.push_back({h->d_path_batches, 3 * S * 8});
  v.push_back({h->d_init_moves, S * 8});
  v.push_back({h->d_drift, S * 8});
  v.push_back({h->d_ex_index, 8});
  v.push_back({h->d_rt_last, S * 4});
  v.push_back({h->d_rt_count, S * 8});
  v.push_back({h->d_ex_att, X * 8});
  v.push_back({h->d_ex_acc, X * 8});
  if (h->part) {
    v.push_back({h->d_gid, S * 4});
    v.push_back({h->d_pos_of, (size_t)h->S_global * 4});
  }
  return v;
}

static size_t state_bytes(rewl_handle* h) {
  size_t b = kCkptHead * 8;
  for (const Section& x : state_sections(h)) b += (x.bytes + 7) & ~(size_t)7;
  return b + 8;
}

// 64-bit FNV-1a over 8-byte words (the buffer length is a multiple of 8).
static unsigned long long ckpt_hash(const unsigned char* p, size_t n) {
  unsigned long long x = 0xcbf29ce484222325ULL;
  for (size_t i = 0; i < n; i += 8) {
    unsigned long long w;
    std::memcpy(&w, p + i, 8);
    x = (x ^ w) * 0x100000001b3ULL;
  }
  return x;
}

// What must agree between the handle that saved a checkpoint and the one that loads it.
static unsigned long long run_fingerprint(const rewl_handle* h) {
  std::vector<unsigned long long> f;
  auto d = [&](double v) {
    unsigned long long w;
    std::memcpy(&w, &v, 8);
    f.push_back(w);
  };
  for (long long v : {(long long)h->kind, (long long)h->L, (long long)h->N, (long long)h->z, (long long)h->B,
                      (long long)h->h, (long long)h->m, (long long)h->W, (long long)h->S, (long long)h->traj,
                      (long long)h->G, (long long)h->exchange_interval, (long long)h->recompute_every,
                      (long long)h->by_window, (long long)h->part, (long long)h->k_begin, (long long)h->k_end,
                      (long long)h->geo.n_shells})
    f.push_back((unsigned long long)v);
  f.push_back(h->seed);
  for (double v : {h->e_min, h->e_max, h->overlap, h->flatness, h->lnf_final}) d(v);
  for (int j = 0; j < 4; ++j) d(h->geo.Jsh_d[j]);
  for (double v : h->tab_J) d(v);
  for (int32_t v : h->tab_nbr) f.push_back((unsigned long long)(uint32_t)v);
  return ckpt_hash(reinterpret_cast<const unsigned char*>(f.data()), f.size() * 8);
}

rewl_status rewl_state_bytes(rewl_handle* h, int64_t* bytes) {
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  if (!bytes) return fail(h, REWL_EINVAL, "bytes is NULL");
  *bytes = (int64_t)state_bytes(h);
  return REWL_OK;
}

rewl_status rewl_save_state(rewl_handle* h, void* buf, int64_t bytes) {
  NvtxRange nvtx_("rewl_save_state");
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  const size_t n = state_bytes(h);
  if (!buf || bytes != (int64_t)n) return fail(h, REWL_EINVAL, "buffer must hold rewl_state_bytes bytes");
  unsigned char* p = static_cast<unsigned char*>(buf);
  long long head[kCkptHead] = {(long long)kCkptTag, kCkptVersion, (long long)n, (long long)run_fingerprint(h),
                               h->initialized ? 1 : 0, h->intervals_done, h->prev_accepts, (long long)h->prev_ex_att,
                               (long long)h->prev_ex_acc, 0};
  std::memcpy(p, head, sizeof head);
  size_t off = sizeof head;
  for (const Section& x : state_sections(h)) {
    CUDA_TRY(h, cudaMemcpyAsync(p + off, x.dev, x.bytes, cudaMemcpyDeviceToHost, h->stream));
    const size_t pad = ((x.bytes + 7) & ~(size_t)7) - x.bytes;
    if (pad) std::memset(p + off + x.bytes, 0, pad);
    off += x.bytes + pad;
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  const unsigned long long c = ckpt_hash(p, off);
  std::memcpy(p + off, &c, 8);
  return REWL_OK;
}

rewl_status rewl_load_state(rewl_handle* h, const void* buf, int64_t bytes) {
  NvtxRange nvtx_("rewl_load_state");
  rewl_status s = check_ready(h);
  if (s != REWL_OK) return s;
  const size_t n = state_bytes(h);
  if (!buf || bytes != (int64_t)n) return fail(h, REWL_EINVAL, "checkpoint size does not match this handle");
  const unsigned char* p = static_cast<const unsigned char*>(buf);
  long long head[kCkptHead];
  std::memcpy(head, p, sizeof head);
  unsigned long long c;
  std::memcpy(&c, p + n - 8, 8);
  if ((unsigned long long)head[0] != kCkptTag || head[1] != kCkptVersion || head[2] != (long long)n)
    return fail(h, REWL_EINVAL, "not a checkpoint of this library version and size");
  if (ckpt_hash(p, n - 8) != c) return fail(h, REWL_EINVAL, "checkpoint checksum mismatch (corrupted)");
  if ((unsigned long long)head[3] != run_fingerprint(h))
    return fail(h, REWL_EINVAL, "checkpoint of a run created with other arguments");
  size_t off = kCkptHead * 8;
  for (const Section& x : state_sections(h)) {
    CUDA_TRY(h, cudaMemcpyAsync(x.dev, p + off, x.bytes, cudaMemcpyHostToDevice, h->stream));
    off += (x.bytes + 7) & ~(size_t)7;
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->initialized = head[4] != 0;
  h->intervals_done = head[5];
  h->prev_accepts = head[6];
  h->prev_ex_att = (unsigned long long)head[7];
  h->prev_ex_acc = (unsigned long long)head[8];
  if (h->part) {
    CUDA_TRY(h, cudaMemcpy(h->gid_host.data(), h->d_gid, h->S * 4, cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(h->pos_host.data(), h->d_pos_of, (size_t)h->S_global * 4, cudaMemcpyDeviceToHost));
  }
  h->wargs_valid = false;
  return REWL_OK;
}

rewl_status rewl_device_exp(const double* x, double* y, int n) {
  if (!x || !y || n < 0) return fail(nullptr, REWL_EINVAL, "bad arguments");
  if (n == 0) return REWL_OK;
  double* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 2 * sizeof(double) * (size_t)n);
  if (e != cudaSuccess) return fail(nullptr, REWL_ENOMEM, "device_exp allocation failed");
  e = cudaMemcpy(d, x, sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_device_exp(d, d + n, n, exp_coeffs(), nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(y, d + n, sizeof(double) * n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(nullptr, REWL_ECUDA, std::string("device_exp: ") + cudaGetErrorString(e));
  return REWL_OK;
}

rewl_status rewl_measure_smem_bandwidth(double* bytes_per_s, double* ms, void* cuda_stream) {
  if (!bytes_per_s) return fail(nullptr, REWL_EINVAL, "bytes_per_s is NULL");
  cudaError_t e = measure_smem_bandwidth(bytes_per_s, ms, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return fail(nullptr, REWL_ECUDA, std::string("smem bandwidth: ") + cudaGetErrorString(e));
  return REWL_OK;
}

}  // extern "C"
