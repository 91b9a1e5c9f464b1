// jobs.h -- what the batch runner (batch.cu) needs to know about a handle (api.cu).
#pragma once

#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rewl.h"
#include "walker.h"

namespace rewl {

// NVTX range over one C-ABI call (host timeline of a profiler; nothing happens without one attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct JobView {
  int kind, N, z, L, S, W, h, m, n_shells;
  bool traj, pipe, initialized, broken, part;
  long long exchange_interval;
  int recompute_every;
  cudaStream_t stream;
};

void job_view(const rewl_handle* h, JobView* v);
// kernel arguments of one exchange interval of the handle (owner table and lattice placement are
// set by the caller for the batched walker)
WalkerArgs job_walker_args(rewl_handle* h, long long moves, int recompute);
ExchangeArgs job_exchange_args(rewl_handle* h);
FlatnessArgs job_flatness_args(rewl_handle* h);
void job_add_intervals(rewl_handle* h, long long n);
// coupling per shell (0 past the last shell), energy range start and bin width, number of bins
void job_couplings(const rewl_handle* h, double J[4], double* e_min, double* dE);
int job_bins(const rewl_handle* h);

}  // namespace rewl
