// batch.cu -- many independent REWL jobs in one persistent walker launch (declared in
// include/rewl.h): the work list over every walker slot of every job, the tuning of the launch
// (walker pairs per CTA, lattice placement) and its autotuner, and the CUDA graphs of the
// exchange-interval sequence (Sec. 4.2-4.3 per job: Wang-Landau moves, replica exchange,
// flatness check and ln f reduction).
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/rewl.h"
#include "jobs.h"
#include "walker.h"

using namespace rewl;

struct rewl_batch {
  std::vector<rewl_handle*> jobs;
  std::vector<JobView> view;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool traj = false;
  int n_shells = 0;
  long long moves = 0;     // trial moves per walker per interval
  int R = 1;               // energy recomputation every R intervals
  int max_smem = 0, n_sms = 0;

  // tuning
  int workers = 0, smem_max_n = 0, own_cap = 8192;
  size_t arena = 0;
  int grid = 0, bps = 0, n_smem_jobs = 0;
  std::vector<WalkerArgs> wargs;

  // work list
  std::vector<char> active;
  std::vector<int> active_ids;
  std::vector<int2> items;

  WalkerArgs* d_jobs = nullptr;
  ExchangeArgs* d_ex_active = nullptr;   // active jobs only
  FlatnessArgs* d_fl = nullptr;          // every job
  int2* d_items = nullptr;
  int* d_head = nullptr;
  int* d_ids = nullptr;
  int* d_count = nullptr;
  std::vector<void*> allocations;

  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};   // R intervals | 1 | 1 with recomputation
  int graphs_built = 0;
  std::vector<cudaStream_t> ext;
  std::vector<cudaEvent_t> ext_ev;
  cudaEvent_t ev_done = nullptr;
  long long intervals_done = 0;
  bool broken = false;
};

namespace {

rewl_status bfail(rewl_batch* b, rewl_status s, const std::string& msg) {
  if (b && s == REWL_ECUDA) b->broken = true;
  set_handleless_error("batch: " + msg);
  return s;
}

#define BCUDA(b, call)                                                                                \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return bfail((b), REWL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
rewl_status balloc(rewl_batch* b, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return bfail(b, REWL_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  b->allocations.push_back(q);
  *p = static_cast<T*>(q);
  return REWL_OK;
}

void drop_graphs(rewl_batch* b) {
  for (auto& g : b->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

// Conflict-table entries wanted: one per site up to 8192 (lattices in shared memory), at most
// own_cap for lattices in global memory.
int own_full_entries(int N, bool smem_lattice, int own_cap) {
  int e = 256;
  while (e < N && e < (smem_lattice ? 8192 : own_cap)) e *= 2;
  return e;
}

// Largest owner table (power of two, 256 .. own_full_entries) that fits `cap` bytes; 0 if none.
int fit_owner(bool traj, bool smem_lattice, int N, int W, size_t cap, int own_cap) {
  for (int e = own_full_entries(N, smem_lattice, own_cap); e >= 256; e /= 2)
    if (walker_pipe_smem_bytes(traj, smem_lattice, N, W, e) <= cap) return e;
  return 0;
}

// Walker arguments, arena and launch shape for `workers` pairs per CTA and lattices with at most
// smem_max_n spins in shared memory.
rewl_status apply_tuning(rewl_batch* b, int workers, int smem_max_n, int own_cap) {
  if (workers < 1 || workers > kBatchMaxWorkers) return bfail(b, REWL_EINVAL, "workers_per_block must be 1..3");
  if (smem_max_n < 0) return bfail(b, REWL_EINVAL, "smem_lattice_max_n must be >= 0");
  if (own_cap < 256 || own_cap > 8192 || (own_cap & (own_cap - 1)) != 0)
    return bfail(b, REWL_EINVAL, "owner_entries_max must be a power of two in 256..8192");
  const size_t usable = (size_t)b->max_smem - 1024;   // static shared memory of the kernel and slack
  const size_t cap = (usable / (size_t)workers) & ~(size_t)15;
  const int n = (int)b->jobs.size();
  std::vector<char> in_smem(n, 0);
  size_t arena = 0;
  for (int j = 0; j < n; ++j) {
    const JobView& v = b->view[j];
    bool s = v.N <= smem_max_n && fit_owner(b->traj, true, v.N, v.W, cap, own_cap) > 0;
    if (!s && fit_owner(b->traj, false, v.N, v.W, cap, own_cap) == 0)
      return bfail(b, REWL_EINVAL, "window tables of job " + std::to_string(j) + " do not fit the arena");
    in_smem[j] = s;
    // the smallest arena that still holds this job with its full owner table, else the cap
    const int e = fit_owner(b->traj, s, v.N, v.W, cap, own_cap);
    arena = std::max(arena, walker_pipe_smem_bytes(b->traj, s, v.N, v.W, e));
  }
  arena = (arena + 15) & ~(size_t)15;
  int bps = 0;
  BCUDA(b, setup_walkers_batch(b->traj, b->n_shells, workers, arena, &bps));
  if (bps < 1) return bfail(b, REWL_EINVAL, "batched walker does not fit on an SM with this tuning");
  b->workers = workers;
  b->smem_max_n = smem_max_n;
  b->own_cap = own_cap;
  b->arena = arena;
  b->bps = bps;
  b->n_smem_jobs = 0;
  for (int j = 0; j < n; ++j) {
    const JobView& v = b->view[j];
    WalkerArgs& a = b->wargs[j];
    a = job_walker_args(b->jobs[j], b->moves, 0);
    const int e = fit_owner(b->traj, in_smem[j] != 0, v.N, v.W, arena, own_cap);
    a.own_mask = e - 1;
    a.smem_lattice = in_smem[j];
    b->n_smem_jobs += in_smem[j];
  }
  BCUDA(b, cudaMemcpyAsync(b->d_jobs, b->wargs.data(), sizeof(WalkerArgs) * (size_t)n, cudaMemcpyHostToDevice,
                           b->stream));
  const int n_items = (int)b->items.size();
  b->grid = std::max(1, std::min(b->n_sms * bps, (n_items + workers - 1) / workers));
  drop_graphs(b);
  return REWL_OK;
}

// Work list: every slot of every active job, larger lattices (and global-memory lattices) first.
rewl_status build_work_list(rewl_batch* b) {
  b->active_ids.clear();
  for (int j = 0; j < (int)b->jobs.size(); ++j)
    if (b->active[j]) b->active_ids.push_back(j);
  std::vector<int> order = b->active_ids;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->view[x].N > b->view[y].N; });
  b->items.clear();
  for (int j : order)
    for (int s = 0; s < b->view[j].S; ++s) b->items.push_back(make_int2(j, s));
  std::vector<ExchangeArgs> ex;
  for (int j : b->active_ids) ex.push_back(job_exchange_args(b->jobs[j]));
  if (!b->items.empty()) {
    BCUDA(b, cudaMemcpyAsync(b->d_items, b->items.data(), sizeof(int2) * b->items.size(), cudaMemcpyHostToDevice,
                             b->stream));
    BCUDA(b, cudaMemcpyAsync(b->d_ex_active, ex.data(), sizeof(ExchangeArgs) * ex.size(), cudaMemcpyHostToDevice,
                             b->stream));
    BCUDA(b, cudaMemcpyAsync(b->d_ids, b->active_ids.data(), sizeof(int) * b->active_ids.size(),
                             cudaMemcpyHostToDevice, b->stream));
  }
  // host arrays above are read by the copies before they go out of scope
  BCUDA(b, cudaStreamSynchronize(b->stream));
  if (b->workers > 0)
    b->grid = std::max(1, std::min(b->n_sms * b->bps, ((int)b->items.size() + b->workers - 1) / b->workers));
  drop_graphs(b);
  return REWL_OK;
}

BatchLaunch walker_launch(const rewl_batch* b, long long moves, int recompute) {
  BatchLaunch bl{};
  bl.jobs = b->d_jobs;
  bl.items = b->d_items;
  bl.n_items = (int)b->items.size();
  bl.head = b->d_head;
  bl.moves = moves;
  bl.recompute = recompute;
  bl.traj = b->traj;
  bl.n_shells = b->n_shells;
  bl.workers = b->workers;
  bl.arena = b->arena;
  bl.grid = b->grid;
  return bl;
}

// One exchange interval of every active job: walker launch, exchange, flatness.
cudaError_t enqueue_interval(const rewl_batch* b, int recompute) {
  cudaError_t e = launch_walkers_batch(walker_launch(b, b->moves, recompute), b->stream);
  if (e == cudaSuccess) e = launch_exchange_batch(b->d_ex_active, (int)b->active_ids.size(), b->stream);
  if (e == cudaSuccess) e = launch_flatness_batch(b->d_fl, b->d_items, (int)b->items.size(), b->stream);
  return e;
}

// Graph k: 0 = R intervals with the recomputation in the last, 1 = one interval, 2 = one interval
// with the recomputation.
rewl_status get_graph(rewl_batch* b, int k, cudaGraphExec_t* out) {
  if (!b->graph[k]) {
    const int n = k == 0 ? b->R : 1;
    BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = enqueue_interval(b, (k != 1 && i == n - 1) ? 1 : 0);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[k], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, REWL_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    b->graphs_built += 1;
  }
  *out = b->graph[k];
  return REWL_OK;
}

rewl_status order_after_jobs(rewl_batch* b) {
  for (size_t i = 0; i < b->ext.size(); ++i) {
    BCUDA(b, cudaEventRecord(b->ext_ev[i], b->ext[i]));
    BCUDA(b, cudaStreamWaitEvent(b->stream, b->ext_ev[i], 0));
  }
  return REWL_OK;
}

rewl_status order_jobs_after(rewl_batch* b) {
  BCUDA(b, cudaEventRecord(b->ev_done, b->stream));
  for (cudaStream_t s : b->ext) BCUDA(b, cudaStreamWaitEvent(s, b->ev_done, 0));
  return REWL_OK;
}

rewl_status check_batch(rewl_batch* b) {
  if (!b) return bfail(nullptr, REWL_EINVAL, "null batch");
  if (b->broken) return bfail(b, REWL_ESTATE, "batch saw a CUDA error; destroy it");
  return REWL_OK;
}

rewl_status run_intervals(rewl_batch* b, long long n) {
  if (b->items.empty() || n <= 0) return REWL_OK;
  rewl_status s = order_after_jobs(b);
  if (s != REWL_OK) return s;
  long long left = n;
  while (left > 0) {
    cudaGraphExec_t g = nullptr;
    long long step;
    if (b->intervals_done % b->R == 0 && left >= b->R) {
      s = get_graph(b, 0, &g);
      step = b->R;
    } else {
      const bool rec = ((b->intervals_done + 1) % b->R) == 0;
      s = get_graph(b, rec ? 2 : 1, &g);
      step = 1;
    }
    if (s != REWL_OK) return s;
    BCUDA(b, cudaGraphLaunch(g, b->stream));
    b->intervals_done += step;
    left -= step;
    for (int j : b->active_ids) job_add_intervals(b->jobs[j], step);
  }
  return order_jobs_after(b);
}

}  // namespace

extern "C" rewl_status rewl_batch_create(rewl_handle* const* jobs, int n_jobs, void* cuda_stream, rewl_batch** out) {
  if (!out) return bfail(nullptr, REWL_EINVAL, "NULL out");
  *out = nullptr;
  if (!jobs || n_jobs < 1) return bfail(nullptr, REWL_EINVAL, "no jobs");
  auto* b = new rewl_batch();
  auto bad = [&](rewl_status s, const std::string& m) {
    rewl_batch_destroy(b);
    return bfail(nullptr, s, m);
  };
  b->jobs.assign(jobs, jobs + n_jobs);
  b->view.resize(n_jobs);
  for (int j = 0; j < n_jobs; ++j) {
    if (!jobs[j]) return bad(REWL_EINVAL, "NULL job " + std::to_string(j));
    for (int i = 0; i < j; ++i)
      if (jobs[i] == jobs[j]) return bad(REWL_EINVAL, "job " + std::to_string(j) + " listed twice");
    job_view(jobs[j], &b->view[j]);
    const JobView& v = b->view[j];
    if (v.broken) return bad(REWL_ESTATE, "job " + std::to_string(j) + " saw a CUDA error");
    if (v.kind != REWL_LATTICE_BCC || !v.pipe)
      return bad(REWL_EINVAL, "job " + std::to_string(j) + " does not use the pipelined bcc walker");
    if (v.part) return bad(REWL_EINVAL, "job " + std::to_string(j) + " is a partitioned handle");
    if (v.traj != b->view[0].traj || v.n_shells != b->view[0].n_shells ||
        v.exchange_interval != b->view[0].exchange_interval || v.recompute_every != b->view[0].recompute_every)
      return bad(REWL_EINVAL, "jobs differ in mode, shell count, exchange_interval or recompute_every");
  }
  b->traj = b->view[0].traj;
  b->n_shells = b->view[0].n_shells;
  b->moves = b->view[0].exchange_interval;
  b->R = std::max(1, b->view[0].recompute_every);
  for (int j = 0; j < n_jobs; ++j) {
    if (!b->view[j].initialized) {
      const rewl_status s = rewl_init_walkers(jobs[j]);
      if (s != REWL_OK) return bad(s, "initialising job " + std::to_string(j) + ": " + rewl_last_error(jobs[j]));
      job_view(jobs[j], &b->view[j]);
    }
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&b->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&b->n_sms, cudaDevAttrMultiProcessorCount, dev);
  if (ce == cudaSuccess) {
    if (cuda_stream) {
      b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      ce = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
      b->own_stream = ce == cudaSuccess;
    }
  }
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming);
  for (int j = 0; j < n_jobs && ce == cudaSuccess; ++j) {
    const cudaStream_t s = b->view[j].stream;
    if (s == b->stream || std::find(b->ext.begin(), b->ext.end(), s) != b->ext.end()) continue;
    cudaEvent_t ev = nullptr;
    ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (ce == cudaSuccess) {
      b->ext.push_back(s);
      b->ext_ev.push_back(ev);
    }
  }
  if (ce != cudaSuccess) return bad(REWL_ECUDA, std::string("CUDA set-up: ") + cudaGetErrorString(ce));
  size_t n_slots = 0;
  for (const auto& v : b->view) n_slots += (size_t)v.S;
  rewl_status s = REWL_OK;
  if (s == REWL_OK) s = balloc(b, &b->d_jobs, (size_t)n_jobs);
  if (s == REWL_OK) s = balloc(b, &b->d_ex_active, (size_t)n_jobs);
  if (s == REWL_OK) s = balloc(b, &b->d_fl, (size_t)n_jobs);
  if (s == REWL_OK) s = balloc(b, &b->d_items, n_slots);
  if (s == REWL_OK) s = balloc(b, &b->d_head, 1);
  if (s == REWL_OK) s = balloc(b, &b->d_ids, (size_t)n_jobs);
  if (s == REWL_OK) s = balloc(b, &b->d_count, (size_t)n_jobs);
  if (s != REWL_OK) {
    rewl_batch_destroy(b);
    return s;
  }
  std::vector<FlatnessArgs> fl(n_jobs);
  for (int j = 0; j < n_jobs; ++j) fl[j] = job_flatness_args(jobs[j]);
  ce = cudaMemcpy(b->d_fl, fl.data(), sizeof(FlatnessArgs) * (size_t)n_jobs, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) return bad(REWL_ECUDA, std::string("upload: ") + cudaGetErrorString(ce));
  b->wargs.resize(n_jobs);
  b->active.assign(n_jobs, 1);
  // the batch's stream starts after the jobs' pending work (initial drive included)
  s = order_after_jobs(b);
  if (s == REWL_OK) s = build_work_list(b);
  if (s == REWL_OK) s = apply_tuning(b, 2, 1 << 30, 8192);
  if (s == REWL_OK) {
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) s = bfail(b, REWL_ECUDA, std::string("set-up: ") + cudaGetErrorString(e));
  }
  if (s != REWL_OK) {
    const std::string msg = rewl_last_error(nullptr);
    rewl_batch_destroy(b);
    set_handleless_error(msg);
    return s;
  }
  *out = b;
  return REWL_OK;
}

extern "C" rewl_status rewl_batch_set_tuning(rewl_batch* b, const rewl_batch_tuning* t) {
  rewl_status s = check_batch(b);
  if (s != REWL_OK) return s;
  if (!t) return bfail(b, REWL_EINVAL, "NULL tuning");
  const int w0 = b->workers, n0 = b->smem_max_n, c0 = b->own_cap;
  s = apply_tuning(b, t->workers_per_block, t->smem_lattice_max_n,
                   t->owner_entries_max == 0 ? 8192 : t->owner_entries_max);
  if (s == REWL_EINVAL && w0 > 0) {
    const std::string msg = rewl_last_error(nullptr);
    apply_tuning(b, w0, n0, c0);   // keep the previous, valid tuning
    set_handleless_error(msg);
  }
  return s;
}

extern "C" rewl_status rewl_batch_autotune(rewl_batch* b, int64_t trial_moves, rewl_batch_tuning* chosen,
                                           double* ms_out) {
  NvtxRange nvtx_("rewl_batch_autotune");
  rewl_status s = check_batch(b);
  if (s != REWL_OK) return s;
  if (trial_moves < 1) return bfail(b, REWL_EINVAL, "trial_moves must be > 0");
  if (b->items.empty()) return bfail(b, REWL_ESTATE, "no active jobs");
  std::vector<int> thresholds = {0};
  for (int j : b->active_ids) thresholds.push_back(b->view[j].N);
  std::sort(thresholds.begin(), thresholds.end());
  thresholds.erase(std::unique(thresholds.begin(), thresholds.end()), thresholds.end());
  s = order_after_jobs(b);
  if (s != REWL_OK) return s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  // candidates that fit; a smaller cap is a new candidate only if it shrinks some job's table
  struct Cand {
    int w, thr, cap;
    double ms;
  };
  std::vector<Cand> cands;
  for (int own_cap : {8192, 4096, 2048, 1024, 512})
    for (int w = 1; w <= kBatchMaxWorkers; ++w)
      for (int thr : thresholds) {
        if (apply_tuning(b, w, thr, own_cap) != REWL_OK) continue;
        bool shrinks = own_cap == 8192;
        for (int j : b->active_ids)
          shrinks = shrinks || (!b->wargs[j].smem_lattice && b->view[j].N > own_cap);
        if (shrinks) cands.push_back({w, thr, own_cap, -1.0});
      }
  // two rounds, the second in reverse order; each candidate keeps its faster trial
  for (int round = 0; round < 2; ++round) {
    for (size_t k = 0; k < cands.size(); ++k) {
      Cand& c = cands[round == 0 ? k : cands.size() - 1 - k];
      if (apply_tuning(b, c.w, c.thr, c.cap) != REWL_OK) continue;
      cudaError_t e = cudaEventRecord(e0, b->stream);
      if (e == cudaSuccess) e = launch_walkers_batch(walker_launch(b, trial_moves, 0), b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return bfail(b, REWL_ECUDA, std::string("autotune trial: ") + cudaGetErrorString(e));
      }
      if (c.ms < 0 || ms < c.ms) c.ms = ms;
    }
  }
  double best = -1.0;
  int best_w = b->workers, best_n = b->smem_max_n, best_c = b->own_cap;
  for (const Cand& c : cands)
    if (c.ms >= 0 && (best < 0 || c.ms < best)) {
      best = c.ms;
      best_w = c.w;
      best_n = c.thr;
      best_c = c.cap;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s = apply_tuning(b, best_w, best_n, best_c);
  if (s != REWL_OK) return s;
  s = order_jobs_after(b);
  if (s != REWL_OK) return s;
  if (chosen) {
    chosen->workers_per_block = best_w;
    chosen->smem_lattice_max_n = best_n;
    chosen->owner_entries_max = best_c;
  }
  if (ms_out) *ms_out = best;
  return REWL_OK;
}

extern "C" rewl_status rewl_batch_run_intervals(rewl_batch* b, int n_intervals) {
  NvtxRange nvtx_("rewl_batch_run_intervals");
  rewl_status s = check_batch(b);
  if (s != REWL_OK) return s;
  if (n_intervals < 0) return bfail(b, REWL_EINVAL, "n_intervals must be >= 0");
  return run_intervals(b, n_intervals);
}

extern "C" rewl_status rewl_batch_run_to_convergence(rewl_batch* b, int64_t max_intervals, int check_every,
                                                     int* n_done) {
  NvtxRange nvtx_("rewl_batch_run_to_convergence");
  rewl_status s = check_batch(b);
  if (s != REWL_OK) return s;
  if (max_intervals < 1 || check_every < 1) return bfail(b, REWL_EINVAL, "max_intervals and check_every must be >= 1");
  const int n = (int)b->jobs.size();
  long long done_intervals = 0;
  std::vector<int> cnt;
  auto count_done = [&]() {
    int d = 0;
    for (int j = 0; j < n; ++j) d += b->active[j] ? 0 : 1;
    return d;
  };
  while (true) {
    // which jobs still have walkers at ln f >= ln f_final
    if (!b->active_ids.empty()) {
      const int na = (int)b->active_ids.size();
      BCUDA(b, launch_count_active(b->d_fl, b->d_ids, na, b->d_count, b->stream));
      cnt.assign(na, 0);
      BCUDA(b, cudaMemcpyAsync(cnt.data(), b->d_count, sizeof(int) * (size_t)na, cudaMemcpyDeviceToHost, b->stream));
      BCUDA(b, cudaStreamSynchronize(b->stream));
      bool changed = false;
      for (int i = 0; i < na; ++i)
        if (cnt[i] == 0) {
          b->active[b->active_ids[i]] = 0;
          changed = true;
        }
      if (changed) {
        s = build_work_list(b);
        if (s != REWL_OK) return s;
      }
    }
    if (b->active_ids.empty()) break;
    if (done_intervals >= max_intervals) {
      if (n_done) *n_done = count_done();
      return bfail(b, REWL_ETIMEOUT, "max_intervals reached before every job converged");
    }
    const long long k = std::min<long long>(check_every, max_intervals - done_intervals);
    s = run_intervals(b, k);
    if (s != REWL_OK) return s;
    done_intervals += k;
  }
  if (n_done) *n_done = count_done();
  return order_jobs_after(b);
}

extern "C" rewl_status rewl_batch_get_info(const rewl_batch* b, rewl_batch_info* out) {
  if (!b || !out) return bfail(nullptr, REWL_EINVAL, "NULL argument");
  out->n_jobs = (int)b->jobs.size();
  out->n_items = (int)b->items.size();
  out->n_active_jobs = (int)b->active_ids.size();
  out->workers_per_block = b->workers;
  out->smem_lattice_max_n = b->smem_max_n;
  out->owner_entries_max = b->own_cap;
  out->grid = b->grid;
  out->blocks_per_sm = b->bps;
  out->n_smem_lattice_jobs = b->n_smem_jobs;
  out->arena_bytes = (int64_t)b->arena;
  out->intervals_done = b->intervals_done;
  out->graphs_built = b->graphs_built;
  return REWL_OK;
}

extern "C" void rewl_batch_destroy(rewl_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  for (void* p : b->allocations) cudaFree(p);
  for (cudaEvent_t e : b->ext_ev) cudaEventDestroy(e);
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}
