// stitch_static.cu -- rewl_stitch_device_noalloc: the fragment join of rewl_stitch_device for
// callers that must not allocate device memory.  Its scratch (window averages, window starts,
// join bins) lives in one statically sized device array defined in this file, so the call makes no
// cudaMalloc, cudaFree or stream-ordered allocation.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/rewl.h"
#include "walker.h"

namespace {

constexpr size_t kStitchScratchBytes = size_t(4) << 20;   // 4 MiB, held by every device that loads the library

// Scratch shared by every call on a device.  In host code this name is only a host-side stand-in
// for the symbol: the device address comes from cudaGetSymbolAddress (per device, below).
static __device__ __align__(256) unsigned char g_stitch_scratch[kStitchScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

constexpr size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

rewl_status noalloc_fail(rewl_status s, const std::string& msg) {
  rewl::set_handleless_error(msg);   // reported by rewl_last_error(NULL)
  return s;
}

}  // namespace

extern "C" rewl_status rewl_stitch_device_noalloc(const double* frag, const int32_t* starts_host, int n_windows,
                                                  int walkers_per_window, int window_bins, int n_bins, double* out,
                                                  int32_t* bstar_out, void* cuda_stream) {
  const int h = n_windows, m = walkers_per_window, W = window_bins, B = n_bins;
  if (!frag || !starts_host || !out) return noalloc_fail(REWL_EINVAL, "NULL argument");
  if (h < 1 || m < 1 || W < 3 || B < W) return noalloc_fail(REWL_EINVAL, "bad sizes");
  for (int k = 0; k < h; ++k) {
    if (starts_host[k] < 0 || starts_host[k] + W > B) return noalloc_fail(REWL_EINVAL, "window outside [0, B)");
    if (k > 0 && starts_host[k] <= starts_host[k - 1]) return noalloc_fail(REWL_EINVAL, "window starts must increase");
    if (k > 0 && starts_host[k - 1] + W - starts_host[k] < 2)
      return noalloc_fail(REWL_EINVAL, "adjacent windows must overlap by at least 2 bins");
  }
  if (starts_host[0] != 0 || starts_host[h - 1] + W != B)
    return noalloc_fail(REWL_EINVAL, "windows must cover [0, B): starts[0] = 0 and starts[h-1] + W = B");
  // scratch layout: averages [h][W] FP64 | starts [h] | join bins [h-1]
  const size_t avg_bytes = align256(sizeof(double) * (size_t)h * (size_t)W);
  const size_t starts_bytes = align256(sizeof(int32_t) * (size_t)h);
  const size_t bstar_bytes = align256(sizeof(int32_t) * (size_t)std::max(h - 1, 1));
  if (avg_bytes + starts_bytes + bstar_bytes > kStitchScratchBytes)
    return noalloc_fail(REWL_EINVAL, "n_windows * window_bins too large for the static scratch (" +
                                         std::to_string(kStitchScratchBytes) + " bytes)");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(REWL_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(REWL_EINVAL, "device index out of range");
  void* base = nullptr;
  {
    // one-time set-up per device, with that device current (the first call on a device)
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_stitch_scratch);
      if (e != cudaSuccess)
        return noalloc_fail(REWL_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  double* avg = reinterpret_cast<double*>(b);
  int32_t* starts = reinterpret_cast<int32_t*>(b + avg_bytes);
  int32_t* bstar = reinterpret_cast<int32_t*>(b + avg_bytes + starts_bytes);

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // every scratch word the kernels read is written first in this call: starts by the copy,
  // averages by the first kernel, join bins by the second
  e = cudaMemcpyAsync(starts, starts_host, sizeof(int32_t) * (size_t)h, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return noalloc_fail(REWL_ECUDA, std::string("copy of starts: ") + cudaGetErrorString(e));
  rewl::MergeArgs a{};
  a.frag = frag;
  a.frag_fx = nullptr;
  a.starts = starts;
  a.h = h;
  a.m = m;
  a.W = W;
  a.B = B;
  a.avg = avg;
  a.bstar = bstar_out ? bstar_out : bstar;
  a.out = out;
  e = rewl::launch_merge(a, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return noalloc_fail(REWL_ECUDA, std::string("stitch: ") + cudaGetErrorString(e));
  return REWL_OK;
}
