// kernels.cu -- replica exchange (Sec. 4.3, Eq. 5), flatness and ln f update (Sec. 4.2), joining
// of the ln g fragments (Sec. 4.3), thermodynamics (Sec. 4.1, Eq. 2-3), and two measurement
// kernels (device exp, shared-memory bandwidth).
#include <cmath>

#include "device_common.cuh"
#include "walker.h"

namespace rewl {

// ------------------------------------------------------------------------------------------------
// Replica exchange.  Round t pairs windows (k, k+1), k = t mod 2, t mod 2 + 2, ...; walker a of
// window k meets walker (a + floor(t/2)) mod m of window k+1.  Slot i (window k) holds
// configuration A, slot j (window k+1) holds B; the swap needs E_A in window k+1 and E_B in
// window k and is accepted with min[1, exp(D)],
//   D = ((ln g_i(E_A) - ln g_i(E_B)) + ln g_j(E_B)) - ln g_j(E_A)   (FP64),
// u = u53(x0, x1) of Philox key (k, key1 ^ 0x5eed5eed), counter (t, 3, a).  Accepted swaps exchange
// the configuration index and the energy; ln g and H stay with the slots.  One CTA, so the round
// counter is read once and advanced after every pair is done.
// ------------------------------------------------------------------------------------------------
// Replica round trips (Sec. 5, Fig. 1): a configuration completes one when it is found in the
// lowest window after having been found in the highest.  The configurations of both extreme
// windows are looked at before and after every round (looking twice at one state changes nothing);
// each configuration sits in one slot, so the threads touch distinct entries.  A partitioned handle
// looks only at the extreme-window slots it hosts (every configuration is hosted by one handle).
__device__ __forceinline__ void observe_extremes(const ExchangeArgs& a) {
  const int h = a.win.h, m = a.win.m;
  if (h < 2) return;
  for (int i = threadIdx.x; i < 2 * m; i += blockDim.x) {
    const int g = i < m ? i : (h - 1) * m + (i - m);
    const int p = a.st.pos_of ? a.st.pos_of[g] : g;
    if (p < 0) continue;
    const int r = a.st.perm[p];
    if (i < m) {
      if (a.st.rt_last[r] == 1) a.st.rt_count[r] += 1;
      a.st.rt_last[r] = 0;
    } else {
      a.st.rt_last[r] = 1;
    }
  }
}

__device__ __forceinline__ int position_bin(const ExchangeArgs& a, int p) {
  return a.traj ? a.st.bin[p] : fx_bin(a.st.efx[p]);
}

// ln g of the slot at position p at global bin b (window start s), as the 64 bits the tables hold:
// 2^-40 fixed point (production) or the FP64 bit pattern (trajectory).
__device__ __forceinline__ long long lng_bits(const ExchangeArgs& a, int p, int b, int s) {
  const size_t idx = (size_t)p * a.win.W + (b - s);
  return a.traj ? __double_as_longlong(a.st.lng[idx]) : a.st.lng_fx[idx];
}

// Eq. 5 from the four ln g values, in one fixed order: D = ((ln g_i(E_A) - ln g_i(E_B)) +
// ln g_j(E_B)) - ln g_j(E_A), accepted if D >= 0 or u < exp(D).
__device__ __forceinline__ bool exchange_accepts(const ExchangeArgs& a, long long t, int k, int aa, long long iA,
                                                 long long iB, long long jB, long long jA) {
  double D;
  if (a.traj) {
    D = __dsub_rn(__dadd_rn(__dsub_rn(__longlong_as_double(iA), __longlong_as_double(iB)), __longlong_as_double(jB)),
                  __longlong_as_double(jA));
  } else {
    const long long Dfx = ((iA - iB) + jB) - jA;
    D = __dmul_rn(__ll2double_rn(Dfx), kLngUnit);
  }
  if (D >= 0.0) return true;
  const uint4 x = philox10(make_uint4((uint32_t)t, (uint32_t)((unsigned long long)t >> 32), 3u, (uint32_t)aa),
                           make_uint2((uint32_t)k, a.key1 ^ 0x5eed5eedu));
  return uniform53(x.x, x.y) < exp_fp64(D, a.ex);
}

__device__ __forceinline__ void exchange_block(const ExchangeArgs& a) {
  __shared__ long long t_s;
  if (threadIdx.x == 0) t_s = *a.st.ex_index;
  observe_extremes(a);
  __syncthreads();
  const long long t = t_s;
  const int h = a.win.h, m = a.win.m, W = a.win.W;
  const int parity = (int)(t & 1);
  const int shift = (int)((unsigned long long)(t >> 1) % (unsigned long long)m);
  const int total = ((h - parity) / 2) * m;
  const bool part = a.st.pos_of != nullptr;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int k = parity + 2 * (idx / m);
    const int aa = idx % m;
    if (k + 1 >= h) continue;
    const int gi = k * m + aa;
    const int gj = (k + 1) * m + (aa + shift) % m;
    const int i = part ? a.st.pos_of[gi] : gi;      // positions (-1: hosted by another handle)
    const int j = part ? a.st.pos_of[gj] : gj;
    if (i < 0 && j < 0) continue;
    const int si = a.win.starts[k], sj = a.win.starts[k + 1];
    if (i >= 0 && j >= 0) {
      // both configurations here: swap them between the slots
      const int bA = position_bin(a, i), bB = position_bin(a, j);
      atomicAdd(a.st.ex_att + k, 1ull);
      if ((unsigned)(bA - sj) >= (unsigned)W || (unsigned)(bB - si) >= (unsigned)W) continue;
      if ((unsigned)(bA - si) >= (unsigned)W || (unsigned)(bB - sj) >= (unsigned)W) continue;  // defensive
      if (!exchange_accepts(a, t, k, aa, lng_bits(a, i, bA, si), lng_bits(a, i, bB, si), lng_bits(a, j, bB, sj),
                            lng_bits(a, j, bA, sj)))
        continue;
      const int32_t tp = a.st.perm[i];
      a.st.perm[i] = a.st.perm[j];
      a.st.perm[j] = tp;
      if (a.traj) {
        const double te = a.st.E[i];
        a.st.E[i] = a.st.E[j];
        a.st.E[j] = te;
        const int32_t tb = a.st.bin[i];
        a.st.bin[i] = a.st.bin[j];
        a.st.bin[j] = tb;
      } else {
        const long long te = a.st.efx[i];
        a.st.efx[i] = a.st.efx[j];
        a.st.efx[j] = te;
      }
      atomicAdd(a.st.ex_acc + k, 1ull);
    } else {
      // one side hosted elsewhere: both handles take the same decision from the gathered bins and
      // ln g values; an accepted swap moves the two slot states between the handles (the caller
      // moves them), the configurations stay.  The handle hosting slot gi counts the attempt.
      const int bA = a.part_bin_all[gi], bB = a.part_bin_all[gj];
      if (i >= 0) atomicAdd(a.st.ex_att + k, 1ull);
      if ((unsigned)(bA - sj) >= (unsigned)W || (unsigned)(bB - si) >= (unsigned)W) continue;
      if ((unsigned)(bA - si) >= (unsigned)W || (unsigned)(bB - sj) >= (unsigned)W) continue;  // defensive
      const long long* L = a.part_lk_all;
      if (!exchange_accepts(a, t, k, aa, L[2 * gi], L[2 * gi + 1], L[2 * gj], L[2 * gj + 1])) continue;
      if (i >= 0) {
        a.part_swap_with[gi] = gj;
        atomicAdd(a.st.ex_acc + k, 1ull);
      } else {
        a.part_swap_with[gj] = gi;
      }
    }
  }
  __syncthreads();
  if (!part) observe_extremes(a);   // a partitioned handle looks after the slot states have moved
  if (threadIdx.x == 0) *a.st.ex_index = t + 1;
}

// Partitioned handles, step 1 of a round: the bin of the configuration at every position, stored at
// its global slot (bin_all [S_global]; entries of slots hosted elsewhere are left alone).
__global__ void partition_bins_kernel(const ExchangeArgs a, int n_pos, int32_t* bin_all) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_pos; p += gridDim.x * blockDim.x)
    bin_all[a.st.gid[p]] = position_bin(a, p);
}

// Step 2: for every pair of the coming round with exactly one slot here, that slot's ln g at its
// own configuration's bin and at the partner's (lk [2 S_global]: lk[2 g] and lk[2 g + 1]; 0 when
// the partner's bin is outside the slot's window, i.e. the pair is rejected anyway).
__global__ void partition_lookups_kernel(const ExchangeArgs a, const int32_t* bin_all, long long* lk) {
  const long long t = *a.st.ex_index;
  const int h = a.win.h, m = a.win.m, W = a.win.W;
  const int parity = (int)(t & 1);
  const int shift = (int)((unsigned long long)(t >> 1) % (unsigned long long)m);
  const int total = ((h - parity) / 2) * m;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int k = parity + 2 * (idx / m);
    const int aa = idx % m;
    if (k + 1 >= h) continue;
    const int gi = k * m + aa;
    const int gj = (k + 1) * m + (aa + shift) % m;
    const int i = a.st.pos_of[gi], j = a.st.pos_of[gj];
    if ((i >= 0) == (j >= 0)) continue;
    const int g = i >= 0 ? gi : gj, o = i >= 0 ? gj : gi, p = i >= 0 ? i : j;
    const int s = a.win.starts[g / m];
    const int bo = bin_all[g], bp = bin_all[o];
    lk[2 * g] = (unsigned)(bo - s) < (unsigned)W ? lng_bits(a, p, bo, s) : 0;
    lk[2 * g + 1] = (unsigned)(bp - s) < (unsigned)W ? lng_bits(a, p, bp, s) : 0;
  }
}

// After the slot states of a round have moved: the second look at the extreme windows.
__global__ void partition_observe_kernel(const ExchangeArgs a) { observe_extremes(a); }

__global__ void exchange_kernel(const ExchangeArgs a) { exchange_block(a); }

// one CTA per job of a batch
__global__ void exchange_batch_kernel(const ExchangeArgs* __restrict__ jobs) { exchange_block(jobs[blockIdx.x]); }

cudaError_t launch_exchange(const ExchangeArgs& a, cudaStream_t stream) {
  exchange_kernel<<<1, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_exchange_batch(const ExchangeArgs* jobs, int n_jobs, cudaStream_t stream) {
  exchange_batch_kernel<<<n_jobs, 256, 0, stream>>>(jobs);
  return cudaGetLastError();
}

cudaError_t launch_partition_bins(const ExchangeArgs& a, int n_pos, int32_t* bin_all, cudaStream_t stream) {
  partition_bins_kernel<<<(n_pos + 255) / 256, 256, 0, stream>>>(a, n_pos, bin_all);
  return cudaGetLastError();
}

cudaError_t launch_partition_lookups(const ExchangeArgs& a, const int32_t* bin_all, long long* lk, cudaStream_t stream) {
  partition_lookups_kernel<<<1, 256, 0, stream>>>(a, bin_all, lk);
  return cudaGetLastError();
}

cudaError_t launch_partition_observe(const ExchangeArgs& a, cudaStream_t stream) {
  partition_observe_kernel<<<1, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Flatness: a walker whose ln f is still >= ln f_final is flat when min H >= p * (sum H / W) over
// the W bins of its window (and sum H > 0); then ln f -> ln f / 2, H -> 0, stage += 1.
// One warp per walker.
// ------------------------------------------------------------------------------------------------
// Flat histogram of one walker: min H >= p * (sum H / W) and sum H > 0 (every lane gets the answer).
__device__ __forceinline__ bool walker_flat(const FlatnessArgs& a, const uint32_t* H) {
  const int lane = threadIdx.x & 31;
  const int W = a.win.W;
  uint32_t mn = 0xffffffffu;
  unsigned long long sum = 0;
  for (int w = lane; w < W; w += 32) {
    const uint32_t v = H[w];
    mn = v < mn ? v : mn;
    sum += v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t om = __shfl_xor_sync(kFullMask, mn, o);
    mn = om < mn ? om : mn;
    sum += __shfl_xor_sync(kFullMask, sum, o);
  }
  const double mean = __ddiv_rn(__ull2double_rn(sum), (double)W);
  return sum > 0 && __uint2double_rn(mn) >= __dmul_rn(a.flatness, mean);
}

// Window-synchronous reading: when every walker of the (still active) window k is flat, each bin's
// ln g becomes the mean over the window's walkers (summed in walker order, FP64 in trajectory mode;
// 2^-40 fixed point in production, the sum divided by m with truncation), then ln f halves and H
// clears for all of them.  One warp.
__device__ __forceinline__ void flatness_window_warp(const FlatnessArgs& a, const int k) {
  const int lane = threadIdx.x & 31;
  const int W = a.win.W, m = a.win.m, s0 = k * m;
  const bool active = a.traj ? a.st.lnf[s0] >= a.lnf_final : (double)a.st.lnf_fx[s0] * kLngUnit >= a.lnf_final;
  if (!active) return;
  for (int i = 0; i < m; ++i)
    if (!walker_flat(a, a.st.H + (size_t)(s0 + i) * W)) return;
  for (int w = lane; w < W; w += 32) {
    if (a.traj) {
      double t = 0.0;
      for (int i = 0; i < m; ++i) t = __dadd_rn(t, a.st.lng[(size_t)(s0 + i) * W + w]);
      const double avg = __ddiv_rn(t, (double)m);
      for (int i = 0; i < m; ++i) a.st.lng[(size_t)(s0 + i) * W + w] = avg;
    } else {
      long long t = 0;
      for (int i = 0; i < m; ++i) t += a.st.lng_fx[(size_t)(s0 + i) * W + w];
      const long long avg = t / m;
      for (int i = 0; i < m; ++i) a.st.lng_fx[(size_t)(s0 + i) * W + w] = avg;
    }
    for (int i = 0; i < m; ++i) a.st.H[(size_t)(s0 + i) * W + w] = 0u;
  }
  for (int i = lane; i < m; i += 32) {
    const int slot = s0 + i;
    if (a.traj) {
      a.st.lnf[slot] = __dmul_rn(a.st.lnf[slot], 0.5);
    } else {
      const long long f = a.st.lnf_fx[slot] >> 1;
      a.st.lnf_fx[slot] = f;
      a.st.lnf[slot] = (double)f * kLngUnit;
    }
    a.st.stage[slot] += 1;
  }
}

__device__ __forceinline__ void flatness_warp(const FlatnessArgs& a, const int slot) {
  if (a.by_window) {
    // the warp of the window's first walker does the window (m <= 32 walkers per window)
    if (slot % a.win.m == 0) flatness_window_warp(a, slot / a.win.m);
    return;
  }
  const int lane = threadIdx.x;
  const int W = a.win.W;
  bool active;
  if (a.traj)
    active = a.st.lnf[slot] >= a.lnf_final;
  else
    active = (double)a.st.lnf_fx[slot] * kLngUnit >= a.lnf_final;
  if (!active) return;
  uint32_t* H = a.st.H + (size_t)slot * W;
  uint32_t mn = 0xffffffffu;
  unsigned long long sum = 0;
  for (int w = lane; w < W; w += 32) {
    const uint32_t v = H[w];
    mn = v < mn ? v : mn;
    sum += v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t om = __shfl_xor_sync(kFullMask, mn, o);
    mn = om < mn ? om : mn;
    sum += __shfl_xor_sync(kFullMask, sum, o);
  }
  const double mean = __ddiv_rn(__ull2double_rn(sum), (double)W);
  const bool flat = sum > 0 && __uint2double_rn(mn) >= __dmul_rn(a.flatness, mean);
  if (!flat) return;
  for (int w = lane; w < W; w += 32) H[w] = 0u;
  if (lane == 0) {
    if (a.traj) {
      a.st.lnf[slot] = __dmul_rn(a.st.lnf[slot], 0.5);
    } else {
      const long long f = a.st.lnf_fx[slot] >> 1;
      a.st.lnf_fx[slot] = f;
      a.st.lnf[slot] = (double)f * kLngUnit;
    }
    a.st.stage[slot] += 1;
  }
}

__global__ void flatness_kernel(const FlatnessArgs a) { flatness_warp(a, blockIdx.x); }

// one warp per (job, slot) item of a batch
__global__ void flatness_batch_kernel(const FlatnessArgs* __restrict__ jobs, const int2* __restrict__ items) {
  const int2 it = items[blockIdx.x];
  flatness_warp(jobs[it.x], it.y);
}

// Walkers still at ln f >= ln f_final, per job: out[i] for job ids[i] (one CTA per job).
__global__ void count_active_kernel(const FlatnessArgs* __restrict__ jobs, const int* __restrict__ ids, int* out) {
  const FlatnessArgs& a = jobs[ids[blockIdx.x]];
  const int S = a.win.h * a.win.m;
  int n = 0;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const bool active = a.traj ? a.st.lnf[s] >= a.lnf_final : (double)a.st.lnf_fx[s] * kLngUnit >= a.lnf_final;
    n += active ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(kFullMask, n, o);
  __shared__ int part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    out[blockIdx.x] = t;
  }
}

cudaError_t launch_count_active(const FlatnessArgs* jobs, const int* ids, int n, int* out, cudaStream_t stream) {
  count_active_kernel<<<n, 128, 0, stream>>>(jobs, ids, out);
  return cudaGetLastError();
}

cudaError_t launch_flatness(const FlatnessArgs& a, int n_slots, cudaStream_t stream) {
  flatness_kernel<<<n_slots, 32, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_flatness_batch(const FlatnessArgs* jobs, const int2* items, int n_items, cudaStream_t stream) {
  flatness_batch_kernel<<<n_items, 32, 0, stream>>>(jobs, items);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Joining the fragments.  Canonical 32-lane sum: lane l adds x[l], x[l+32], ... in order, then the
// lanes combine with partners l^16 .. l^1 (every lane ends with the same value).
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ double frag_value(const MergeArgs& a, size_t idx) {
  if (a.frag) return a.frag[idx];
  return __dmul_rn(__ll2double_rn(a.frag_fx[idx]), kLngUnit);
}

__device__ double warp_sum32_frag(const MergeArgs& a, size_t base, int n) {
  const int lane = threadIdx.x & 31;
  double p = 0.0;
  for (int i = lane; i < n; i += 32) p = __dadd_rn(p, frag_value(a, base + i));
  for (int o = 16; o > 0; o >>= 1) p = __dadd_rn(p, __shfl_xor_sync(kFullMask, p, o));
  return p;
}

__device__ double warp_sum32(const double* x, int n) {
  const int lane = threadIdx.x & 31;
  double p = 0.0;
  for (int i = lane; i < n; i += 32) p = __dadd_rn(p, x[i]);
  for (int o = 16; o > 0; o >>= 1) p = __dadd_rn(p, __shfl_xor_sync(kFullMask, p, o));
  return p;
}

// (1) per window k: A_k[w] = (sum_a (x_a[w] - mean_a)) / m, mean_a = sum32(x_a) / W.
__global__ void merge_avg_kernel(const MergeArgs a) {
  extern __shared__ double means[];
  const int k = blockIdx.x;
  const int W = a.W, m = a.m;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int w = warp; w < m; w += nw) {
    const double s = warp_sum32_frag(a, ((size_t)k * m + w) * W, W);
    if ((threadIdx.x & 31) == 0) means[w] = __ddiv_rn(s, (double)W);
  }
  __syncthreads();
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    double t = 0.0;
    for (int aa = 0; aa < m; ++aa) t = __dadd_rn(t, __dsub_rn(frag_value(a, ((size_t)k * m + aa) * W + w), means[aa]));
    a.avg[(size_t)k * W + w] = __ddiv_rn(t, (double)m);
  }
}

// (2)-(4) join points, shifts, assembly, mean removal.  One CTA.
__global__ void merge_join_kernel(const MergeArgs a) {
  extern __shared__ unsigned char js[];
  double* shift = reinterpret_cast<double*>(js);
  int* bst = reinterpret_cast<int*>(shift + a.h);
  __shared__ double mean_s;
  const int h = a.h, W = a.W, B = a.B;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  for (int k = warp; k + 1 < h; k += nw) {
    const int sk = a.starts[k], sn = a.starts[k + 1];
    const int lo = sn + 1, hi = sk + W - 2;
    const double* Ak = a.avg + (size_t)k * W;
    const double* An = a.avg + (size_t)(k + 1) * W;
    double bv = inf;
    int bb = -1;
    for (int b = lo + lane; b <= hi; b += 32) {
      const double s1 = __dsub_rn(Ak[b + 1 - sk], Ak[b - 1 - sk]);
      const double s2 = __dsub_rn(An[b + 1 - sn], An[b - 1 - sn]);
      const double v = fabs(__dsub_rn(s1, s2));
      if (v < bv) {            // lanes visit b in increasing order: first minimum kept
        bv = v;
        bb = b;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(kFullMask, bv, o);
      const int ob = __shfl_xor_sync(kFullMask, bb, o);
      if (ob >= 0 && (bb < 0 || ov < bv || (ov == bv && ob < bb))) {
        bv = ov;
        bb = ob;
      }
    }
    if (lane == 0) bst[k] = bb >= 0 ? bb : sn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    shift[0] = 0.0;
    for (int k = 0; k + 1 < h; ++k) {
      const int b = bst[k];
      shift[k + 1] = __dadd_rn(shift[k], __dsub_rn(a.avg[(size_t)k * W + (b - a.starts[k])],
                                                   a.avg[(size_t)(k + 1) * W + (b - a.starts[k + 1])]));
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    int k = 0;
    while (k + 1 < h && b >= bst[k]) ++k;
    a.out[b] = __dadd_rn(a.avg[(size_t)k * W + (b - a.starts[k])], shift[k]);
  }
  __syncthreads();
  if (warp == 0) {
    const double s = warp_sum32(a.out, B);
    if (lane == 0) mean_s = __ddiv_rn(s, (double)B);
  }
  __syncthreads();
  const double mu = mean_s;
  for (int b = threadIdx.x; b < B; b += blockDim.x) a.out[b] = __dsub_rn(a.out[b], mu);
  if (a.bstar)
    for (int k = threadIdx.x; k + 1 < h; k += blockDim.x) a.bstar[k] = bst[k];
}

cudaError_t launch_merge(const MergeArgs& a, cudaStream_t stream) {
  merge_avg_kernel<<<a.h, 256, sizeof(double) * (size_t)a.m, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t js = sizeof(double) * (size_t)a.h + sizeof(int) * (size_t)a.h;
  if (js > 48 * 1024) {
    e = cudaFuncSetAttribute(merge_join_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)js);
    if (e != cudaSuccess) return e;
  }
  merge_join_kernel<<<1, 1024, js, stream>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Thermodynamics (k_B = 1): w_b = exp(ln g_b - E_b / T - max), Z = sum w, U = sum w E / Z,
// var = sum w (E - U)^2 / Z (two passes), C/N = var / (N T^2), ln Z = max + ln(sum w).
// One CTA per temperature.
// ------------------------------------------------------------------------------------------------
__device__ double block_reduce(double v, double* red, bool is_max) {
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(kFullMask, v, o);
    v = is_max ? fmax(v, ov) : v + ov;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : (is_max ? -1e308 : 0.0);
    for (int o = 16; o > 0; o >>= 1) {
      const double ox = __shfl_xor_sync(kFullMask, x, o);
      x = is_max ? fmax(x, ox) : x + ox;
    }
    if (threadIdx.x == 0) red[32] = x;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

__global__ void thermo_kernel(const double* lng, const double* E, int B, double n_spins, const double* T,
                              double* U, double* C, double* lnZ) {
  __shared__ double red[33];
  const double t = T[blockIdx.x];
  const double beta = 1.0 / t;
  double mx = -1e308;
  for (int b = threadIdx.x; b < B; b += blockDim.x) mx = fmax(mx, lng[b] - E[b] * beta);
  mx = block_reduce(mx, red, true);
  double z = 0.0, e1 = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double w = exp(lng[b] - E[b] * beta - mx);
    z += w;
    e1 += w * E[b];
  }
  z = block_reduce(z, red, false);
  e1 = block_reduce(e1, red, false);
  const double u = e1 / z;
  double v = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double w = exp(lng[b] - E[b] * beta - mx);
    const double d = E[b] - u;
    v += w * d * d;
  }
  v = block_reduce(v, red, false) / z;
  if (threadIdx.x == 0) {
    if (U) U[blockIdx.x] = u;
    if (C) C[blockIdx.x] = v * beta * beta / n_spins;
    if (lnZ) lnZ[blockIdx.x] = mx + log(z);
  }
}

cudaError_t launch_thermo(const double* lng, const double* E, int B, double n_spins, const double* T, int nT,
                          double* U, double* C, double* lnZ, cudaStream_t stream) {
  thermo_kernel<<<nT, 256, 0, stream>>>(lng, E, B, n_spins, T, U, C, lnZ);
  return cudaGetLastError();
}

// Temperature of the specific-heat maximum: the grid argmax of C (lowest index on ties), refined by
// the vertex of the parabola through it and its two neighbours, T_b + (dT/2) (C_{b-1} - C_{b+1}) /
// (C_{b-1} - 2 C_b + C_{b+1}); at either end of the grid (or for a flat triple) the grid value.  One CTA.
__global__ void peak_kernel(const double* T, const double* C, int nT, double* out) {
  __shared__ double bv_s[32];
  __shared__ int bi_s[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double ninf = __longlong_as_double((long long)0xfff0000000000000ULL);
  double bv = ninf;
  int bi = nT;
  for (int i = threadIdx.x; i < nT; i += blockDim.x)   // increasing i: the first maximum is kept
    if (bi == nT || C[i] > bv) {
      bv = C[i];
      bi = i;
    }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(kFullMask, bv, o);
    const int oi = __shfl_xor_sync(kFullMask, bi, o);
    if (oi < nT && (bi == nT || ov > bv || (ov == bv && oi < bi))) {
      bv = ov;
      bi = oi;
    }
  }
  if (lane == 0) {
    bv_s[warp] = bv;
    bi_s[warp] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (bi_s[w] < nT && (bi == nT || bv_s[w] > bv || (bv_s[w] == bv && bi_s[w] < bi))) {
        bv = bv_s[w];
        bi = bi_s[w];
      }
    double t = T[bi];
    if (bi > 0 && bi < nT - 1) {
      const double c0 = C[bi - 1], c1 = C[bi], c2 = C[bi + 1];
      const double den = __dadd_rn(__dsub_rn(c0, __dmul_rn(2.0, c1)), c2);
      if (den != 0.0) {
        const double dT = __dsub_rn(T[bi + 1], T[bi]);
        t = __dadd_rn(t, __ddiv_rn(__dmul_rn(__dmul_rn(0.5, dT), __dsub_rn(c0, c2)), den));
      }
    }
    *out = t;
  }
}

cudaError_t launch_peak(const double* T, const double* C, int nT, double* out, cudaStream_t stream) {
  peak_kernel<<<1, 256, 0, stream>>>(T, C, nT, out);
  return cudaGetLastError();
}

// Production lattices: the octahedral codes [R][N] decoded to FP32 planes [R][3][N].
__global__ void decode_spins_kernel(const float2* c, size_t R, int N, float* out) {
  const size_t n = R * (size_t)N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t r = i / (size_t)N, k = i % (size_t)N;
    float x, y, z;
    oct_decode(c[i], x, y, z);
    out[(r * 3 + 0) * N + k] = x;
    out[(r * 3 + 1) * N + k] = y;
    out[(r * 3 + 2) * N + k] = z;
  }
}

cudaError_t launch_decode_spins(const float2* codes, size_t R, int N, float* out, cudaStream_t stream) {
  decode_spins_kernel<<<1024, 256, 0, stream>>>(codes, R, N, out);
  return cudaGetLastError();
}

__global__ void device_exp_kernel(const double* x, double* y, int n, const ExpCoeffs c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = exp_fp64(x[i], c);
}

cudaError_t launch_device_exp(const double* x, double* y, int n, const ExpCoeffs& c, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  device_exp_kernel<<<(n + 255) / 256, 256, 0, stream>>>(x, y, n, c);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Shared-memory load bandwidth: every thread reads 16-byte words of a 48 KB buffer so that each
// quarter-warp covers all 32 banks once (conflict free).  Index always inside the buffer.
// ------------------------------------------------------------------------------------------------
constexpr int kBwWords = 3072;   // float4 words = 48 KB

__global__ void smem_bw_kernel(float* out, int iters) {
  __shared__ float4 buf[kBwWords];
  for (int i = threadIdx.x; i < kBwWords; i += blockDim.x) buf[i] = make_float4((float)i, 1.f, 2.f, 3.f);
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float4 v = buf[(threadIdx.x + u * 256 + (it & 1) * 1024) % kBwWords];
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc.x + acc.y + acc.z + acc.w;
}

cudaError_t measure_smem_bandwidth(double* bytes_per_s, double* ms_out, cudaStream_t stream) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = nsm * 4, threads = 256, iters = 4096;
  float* out = nullptr;
  e = cudaMallocAsync(&out, sizeof(float) * (size_t)blocks * threads, stream);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, stream);
    smem_bw_kernel<<<blocks, threads, 0, stream>>>(out, iters);
    cudaEventRecord(e1, stream);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, stream);
  if (e != cudaSuccess) return e;
  const double bytes = (double)blocks * threads * iters * 8 * 16;
  *bytes_per_s = bytes / (best * 1e-3);
  if (ms_out) *ms_out = best;
  return cudaGetLastError();
}

}  // namespace rewl
