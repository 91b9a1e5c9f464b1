// walker.h -- host-side launchers of the REWL kernels.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "rewl_types.h"

namespace rewl {

size_t walker_smem_bytes(bool traj, bool smem_lattice, int N, int W);
cudaError_t launch_walkers(const WalkerArgs& a, int n_slots, bool traj, bool smem_lattice, size_t smem,
                           cudaStream_t stream);

// Warp-specialised walker (bcc lattices, one lane per trial move, Wang-Landau moves only).
size_t walker_pipe_smem_bytes(bool traj, bool smem_lattice, int N, int W, int own_entries);
// a.smem_lattice selects the form: 1 = lattice in shared memory, arguments passed by value (d_args
// NULL); 0 = lattice in global memory, the kernel reads d_args, a device copy of a (a.moves and
// a.recompute are passed by value and may differ from the copy).
cudaError_t launch_walkers_pipe(const WalkerArgs& a, const WalkerArgs* d_args, int n_slots, bool traj, size_t smem,
                                cudaStream_t stream);

// Batched pipelined walker: one persistent launch over (job, slot) items of many jobs with the same
// mode and shell count.
constexpr int kBatchMaxWorkers = 3;    // workers (walker pairs) per CTA: barrier ids 1..15
struct BatchLaunch {
  const WalkerArgs* jobs;              // device [n_jobs]
  const int2* items;                   // device [n_items] (job, slot), most expensive first
  int n_items;
  int* head;                           // device work-list counter (reset by the launcher)
  long long moves;                     // trial moves per walker
  int recompute;                       // energy recomputation at the end of every slot
  bool traj;
  int n_shells;
  int workers;                         // per CTA
  size_t arena;                        // shared bytes per worker
  int grid;
};
cudaError_t setup_walkers_batch(bool traj, int n_shells, int workers, size_t arena, int* blocks_per_sm);
cudaError_t launch_walkers_batch(const BatchLaunch& b, cudaStream_t stream);

struct ExchangeArgs {
  Windows win;
  WalkerState st;
  ExpCoeffs ex;
  uint32_t key1;
  int traj;
  // partitioned handles (st.pos_of set): the round's gathered bins [S_global] and ln g lookups
  // [2 S_global] of every slot, and the partner of each hosted slot in an accepted cross-handle
  // swap [S_global] (written only for accepted swaps; the caller presets -1)
  const int32_t* part_bin_all;
  const long long* part_lk_all;
  int32_t* part_swap_with;
};
cudaError_t launch_exchange(const ExchangeArgs& a, cudaStream_t stream);
cudaError_t launch_exchange_batch(const ExchangeArgs* jobs, int n_jobs, cudaStream_t stream);
cudaError_t launch_partition_bins(const ExchangeArgs& a, int n_pos, int32_t* bin_all, cudaStream_t stream);
cudaError_t launch_partition_lookups(const ExchangeArgs& a, const int32_t* bin_all, long long* lk, cudaStream_t stream);
cudaError_t launch_partition_observe(const ExchangeArgs& a, cudaStream_t stream);

struct FlatnessArgs {
  Windows win;
  WalkerState st;
  double flatness;
  double lnf_final;
  int traj;
  int by_window;               // 1: the walkers of a window move on together (ln g averaged)
};
cudaError_t launch_flatness(const FlatnessArgs& a, int n_slots, cudaStream_t stream);
cudaError_t launch_flatness_batch(const FlatnessArgs* jobs, const int2* items, int n_items, cudaStream_t stream);
// walkers with ln f >= ln f_final of the jobs ids[0..n-1] -> out[0..n-1] (device arrays)
cudaError_t launch_count_active(const FlatnessArgs* jobs, const int* ids, int n, int* out, cudaStream_t stream);

// Merge: fragments are read from either an FP64 array or a 2^-40 fixed-point array [h][m][W].
struct MergeArgs {
  const double* frag;
  const long long* frag_fx;
  const int32_t* starts;     // device [h]
  int h, m, W, B;
  double* avg;               // scratch [h][W]
  int32_t* bstar;            // scratch or output [h-1] (may be null only when h == 1)
  double* out;               // [B]
};
cudaError_t launch_merge(const MergeArgs& a, cudaStream_t stream);

cudaError_t launch_thermo(const double* lng, const double* E, int B, double n_spins, const double* T, int nT,
                          double* U, double* C, double* lnZ, cudaStream_t stream);

cudaError_t launch_decode_spins(const float2* codes, size_t R, int N, float* out, cudaStream_t stream);

cudaError_t launch_peak(const double* T, const double* C, int nT, double* out, cudaStream_t stream);

cudaError_t launch_device_exp(const double* x, double* y, int n, const ExpCoeffs& c, cudaStream_t stream);

cudaError_t launch_energies(const WalkerArgs& a, int n_replicas, bool traj, double* out, cudaStream_t stream);

cudaError_t launch_neighbour_dump(const Geometry& g, int32_t* nbr, double* J, cudaStream_t stream);

cudaError_t measure_smem_bandwidth(double* bytes_per_s, double* ms, cudaStream_t stream);

// Message returned by rewl_last_error(NULL) (entry points without a handle).
void set_handleless_error(const std::string& msg);

}  // namespace rewl
