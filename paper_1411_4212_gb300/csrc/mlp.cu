// mlp.cu -- the learned warm start: a small MLP maps (E/N, 1/L, J1..J4) to ln g(E)/N and seeds every
// walker's ln g before plain Wang-Landau refines it (the paper has no learned part; Wang-Landau
// still runs every stage, so the network only saves ln f reductions).
//
// Network: 6 inputs (shifted and scaled by fixed per-input constants), 3 hidden layers of 128 SiLU
// units, 1 linear output.  Weights and biases are used in BF16 (rounded from an FP32 master copy
// that Adam updates); activations and every accumulation are FP32.
// Parameter layout (FP32 master, BF16 copy; W stored transposed, WT[k][j] = weight from input k
// to unit j): WT1 [6][128] | b1 [128] | WT2 [128][128] | b2 [128] | WT3 [128][128] | b3 [128] |
// WT4 [128] | b4 [1].
// Loss: per-run centred mean square error, L = (1/M) sum_runs sum_bins (r - mean_run r)^2 with
// r = y - ln g/N, since ln g of a run is only defined up to a constant.
//
// Kernels (CUDA-core FP32 FMAs on BF16 weights, so the activations stay FP32; a full-batch step over
// 51 840 samples is about 10 GFLOP and runs at about 7.5 TFLOP/s, far below what BF16 tensor cores
// would give, but training is not on the sampling path):
//   mlp_fwd_kernel   -- tiles of 16 samples per CTA, BF16 weights staged in shared memory;
//   mlp_loss_kernel  -- one CTA per run: centred residual, loss, dL/dy;
//   mlp_bwd_kernel   -- persistent CTAs: recompute the tile's forward pass, back-propagate, add
//                       the tile's gradient into the CTA's own partial row (fixed tile order);
//   mlp_reduce_kernel-- sum of the partial rows in CTA order (deterministic);
//   mlp_adam_kernel  -- Adam on the FP32 master, BF16 copy refreshed.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/rewl.h"
#include "jobs.h"
#include "walker.h"

namespace rewl {
namespace mlp {

constexpr int kIn = 6, kH = 128, kT = 16, kTp = kT + 4;   // tile of samples, padded row
constexpr int kWs = kH + 2;                                   // padded BF16 weight row (130)
constexpr int oW1 = 0, ob1 = oW1 + kIn * kH, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kH * kH, oW4 = ob3 + kH, ob4 = oW4 + kH, kParams = ob4 + 1;
constexpr int kThreads = kH;

// shared layout (bytes): BF16 weights WT1 [6][130], WT2, WT3 [128][130] | FP32 biases b1..b3 [128],
// W4 [128], b4 | activations A0 [6][20], Z1..Z3 [128][20], A1..A3 [128][20] | dA [2][128][20] | dy [16]
struct Smem {
  __nv_bfloat16 w1[kIn * kWs], w2[kH * kWs], w3[kH * kWs];
  alignas(16) float b1[kH];
  float b2[kH], b3[kH], w4[kH], b4;
  alignas(16) float a0[kIn * kTp];             // rows of kTp floats: every row 16-byte aligned
  alignas(16) float z[3][kH * kTp];
  alignas(16) float a[3][kH * kTp];
  alignas(16) float da[2][kH * kTp];
  float dy[kT];
  float y[kT];
};
static_assert(sizeof(Smem) <= 227 * 1024, "MLP tile does not fit in shared memory");

__device__ __forceinline__ float sigmoid(float z) { return 1.0f / (1.0f + expf(-z)); }

__device__ void stage_params(Smem& s, const __nv_bfloat16* __restrict__ p) {
  for (int i = threadIdx.x; i < kIn * kH; i += blockDim.x) s.w1[(i / kH) * kWs + i % kH] = p[oW1 + i];
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
    s.w2[(i / kH) * kWs + i % kH] = p[oW2 + i];
    s.w3[(i / kH) * kWs + i % kH] = p[oW3 + i];
  }
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    s.b1[i] = __bfloat162float(p[ob1 + i]);
    s.b2[i] = __bfloat162float(p[ob2 + i]);
    s.b3[i] = __bfloat162float(p[ob3 + i]);
    s.w4[i] = __bfloat162float(p[oW4 + i]);
  }
  if (threadIdx.x == 0) s.b4 = __bfloat162float(p[ob4]);
}

// Hidden layer: unit j = threadIdx.x, every sample of the tile.  in: [n_in][kTp].
__device__ __forceinline__ void dense_silu(const float* in, int n_in, const __nv_bfloat16* wt, const float* b,
                                           float* z, float* a) {
  const int j = threadIdx.x;
  float acc[kT];
#pragma unroll
  for (int t = 0; t < kT; ++t) acc[t] = b[j];
  for (int k = 0; k < n_in; ++k) {
    const float w = __bfloat162float(wt[k * kWs + j]);
    const float4* r = reinterpret_cast<const float4*>(in + k * kTp);
#pragma unroll
    for (int q = 0; q < kT / 4; ++q) {
      const float4 v = r[q];
      acc[4 * q + 0] = fmaf(w, v.x, acc[4 * q + 0]);
      acc[4 * q + 1] = fmaf(w, v.y, acc[4 * q + 1]);
      acc[4 * q + 2] = fmaf(w, v.z, acc[4 * q + 2]);
      acc[4 * q + 3] = fmaf(w, v.w, acc[4 * q + 3]);
    }
  }
  float4* zo = reinterpret_cast<float4*>(z + j * kTp);
  float4* ao = reinterpret_cast<float4*>(a + j * kTp);
#pragma unroll
  for (int q = 0; q < kT / 4; ++q) {
    float4 zz = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    zo[q] = zz;
    ao[q] = make_float4(zz.x * sigmoid(zz.x), zz.y * sigmoid(zz.y), zz.z * sigmoid(zz.z), zz.w * sigmoid(zz.w));
  }
}

// Forward pass of the tile starting at sample s0 (n_t valid samples); y in s.y[0..n_t).
__device__ void forward_tile(Smem& s, const float* __restrict__ x, long long s0, int n_t, const float* shift,
                             const float* scale) {
  for (int i = threadIdx.x; i < kIn * kT; i += blockDim.x) {
    const int k = i / kT, t = i % kT;
    float v = 0.0f;
    if (t < n_t) v = (x[(s0 + t) * kIn + k] - shift[k]) * scale[k];
    s.a0[k * kTp + t] = v;
  }
  __syncthreads();
  dense_silu(s.a0, kIn, s.w1, s.b1, s.z[0], s.a[0]);
  __syncthreads();
  dense_silu(s.a[0], kH, s.w2, s.b2, s.z[1], s.a[1]);
  __syncthreads();
  dense_silu(s.a[1], kH, s.w3, s.b3, s.z[2], s.a[2]);
  __syncthreads();
  if (threadIdx.x < kT) {
    const int t = threadIdx.x;
    float acc = s.b4;
    for (int k = 0; k < kH; ++k) acc = fmaf(s.w4[k], s.a[2][k * kTp + t], acc);
    s.y[t] = acc;
  }
  __syncthreads();
}

struct Net {
  const __nv_bfloat16* p;    // BF16 parameters
  float shift[kIn], scale[kIn];
};

__global__ void __launch_bounds__(kThreads) mlp_fwd_kernel(const Net net, const float* __restrict__ x, long long n,
                                                           float* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char raw[];
  Smem& s = *reinterpret_cast<Smem*>(raw);
  stage_params(s, net.p);
  __syncthreads();
  const long long n_tiles = (n + kT - 1) / kT;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long s0 = tile * kT;
    const int n_t = (int)std::min<long long>(kT, n - s0);
    forward_tile(s, x, s0, n_t, net.shift, net.scale);
    if (threadIdx.x < n_t) y[s0 + threadIdx.x] = s.y[threadIdx.x];
    __syncthreads();
  }
}

// One CTA per run g (samples seg[g] .. seg[g+1]-1): residual r = y - t, its mean, the loss part
// sum (r - mean)^2 (FP64) and dy = 2 (r - mean) / M.
__global__ void mlp_loss_kernel(const float* __restrict__ y, const float* __restrict__ t, const int* __restrict__ seg,
                                float inv_m, float* __restrict__ dy, double* __restrict__ loss_part) {
  const int g = blockIdx.x;
  const int a = seg[g], b = seg[g + 1];
  __shared__ double red[32];
  double sr = 0.0;
  for (int i = a + threadIdx.x; i < b; i += blockDim.x) sr += (double)y[i] - (double)t[i];
  for (int o = 16; o > 0; o >>= 1) sr += __shfl_xor_sync(0xffffffffu, sr, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sr;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    red[31] = b > a ? v / (double)(b - a) : 0.0;
  }
  __syncthreads();
  const double mean = red[31];
  __syncthreads();
  double sl = 0.0;
  for (int i = a + threadIdx.x; i < b; i += blockDim.x) {
    const double r = ((double)y[i] - (double)t[i]) - mean;
    sl += r * r;
    dy[i] = (float)(2.0 * r) * inv_m;
  }
  for (int o = 16; o > 0; o >>= 1) sl += __shfl_xor_sync(0xffffffffu, sl, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sl;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    loss_part[g] = v;
  }
}

// dZ = dA * silu'(Z) in place (row j = threadIdx.x), then the gradients of the layer with input
// `in` [n_in][kTp]: partial WT[k][j] += sum_t in[k][t] dZ[j][t], b[j] += sum_t dZ[j][t]; and, if
// dA_in != nullptr, dA_in[k][t] = sum_j WT[k][j] dZ[j][t].
__device__ __forceinline__ void back_layer(Smem& s, float* dA, const float* z, const float* in, int n_in,
                                           const __nv_bfloat16* wt, float* __restrict__ gW, float* __restrict__ gb,
                                           float* dA_in) {
  const int j = threadIdx.x;
  float dz[kT];
  float sb = 0.0f;
#pragma unroll
  for (int t = 0; t < kT; ++t) {
    const float zz = z[j * kTp + t];
    const float sg = sigmoid(zz);
    dz[t] = dA[j * kTp + t] * (sg * (1.0f + zz * (1.0f - sg)));
    sb += dz[t];
  }
#pragma unroll
  for (int t = 0; t < kT; ++t) dA[j * kTp + t] = dz[t];
  gb[j] += sb;
  for (int k = 0; k < n_in; ++k) {
    const float4* r = reinterpret_cast<const float4*>(in + k * kTp);
    float acc = 0.0f;
#pragma unroll
    for (int q = 0; q < kT / 4; ++q) {
      const float4 v = r[q];
      acc = fmaf(v.x, dz[4 * q], acc);
      acc = fmaf(v.y, dz[4 * q + 1], acc);
      acc = fmaf(v.z, dz[4 * q + 2], acc);
      acc = fmaf(v.w, dz[4 * q + 3], acc);
    }
    gW[k * kH + j] += acc;
  }
  __syncthreads();
  if (dA_in && j < n_in) {
    const int k = j;
    float acc[kT];
#pragma unroll
    for (int t = 0; t < kT; ++t) acc[t] = 0.0f;
    for (int jj = 0; jj < kH; ++jj) {
      const float w = __bfloat162float(wt[k * kWs + jj]);
      const float4* r = reinterpret_cast<const float4*>(dA + jj * kTp);
#pragma unroll
      for (int q = 0; q < kT / 4; ++q) {
        const float4 v = r[q];
        acc[4 * q + 0] = fmaf(w, v.x, acc[4 * q + 0]);
        acc[4 * q + 1] = fmaf(w, v.y, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(w, v.z, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(w, v.w, acc[4 * q + 3]);
      }
    }
#pragma unroll
    for (int t = 0; t < kT; ++t) dA_in[k * kTp + t] = acc[t];
  }
  __syncthreads();
}

// Persistent: CTA c takes tiles c, c + grid, ... and adds their gradient into partial[c][*].
__global__ void __launch_bounds__(kThreads) mlp_bwd_kernel(const Net net, const float* __restrict__ x,
                                                           const float* __restrict__ dy, long long n,
                                                           float* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char raw[];
  Smem& s = *reinterpret_cast<Smem*>(raw);
  stage_params(s, net.p);
  __syncthreads();
  float* g = partial + (size_t)blockIdx.x * kParams;
  const long long n_tiles = (n + kT - 1) / kT;
  const int j = threadIdx.x;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long s0 = tile * kT;
    const int n_t = (int)std::min<long long>(kT, n - s0);
    forward_tile(s, x, s0, n_t, net.shift, net.scale);
    if (j < kT) s.dy[j] = j < n_t ? dy[s0 + j] : 0.0f;
    __syncthreads();
    // output layer: y = b4 + sum_k W4[k] A3[k]
    {
      float acc = 0.0f;
      for (int t = 0; t < kT; ++t) {
        acc = fmaf(s.a[2][j * kTp + t], s.dy[t], acc);
        s.da[0][j * kTp + t] = s.w4[j] * s.dy[t];
      }
      g[oW4 + j] += acc;
      if (j == 0) {
        float sb = 0.0f;
        for (int t = 0; t < kT; ++t) sb += s.dy[t];
        g[ob4] += sb;
      }
    }
    __syncthreads();
    back_layer(s, s.da[0], s.z[2], s.a[1], kH, s.w3, g + oW3, g + ob3, s.da[1]);
    back_layer(s, s.da[1], s.z[1], s.a[0], kH, s.w2, g + oW2, g + ob2, s.da[0]);
    back_layer(s, s.da[0], s.z[0], s.a0, kIn, s.w1, g + oW1, g + ob1, nullptr);
  }
}

__global__ void mlp_reduce_kernel(const float* __restrict__ partial, int n_rows, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  float acc = 0.0f;
  for (int r = 0; r < n_rows; ++r) acc += partial[(size_t)r * kParams + p];
  grad[p] = acc;
}

struct AdamArgs {
  float lr, b1, b2, eps, c1, c2;   // c1 = 1 - b1^t, c2 = 1 - b2^t
};

__global__ void mlp_adam_kernel(float* __restrict__ w, const float* __restrict__ grad, float* __restrict__ m,
                                float* __restrict__ v, __nv_bfloat16* __restrict__ wb, const AdamArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  const float gr = grad[p];
  const float mm = a.b1 * m[p] + (1.0f - a.b1) * gr;
  const float vv = a.b2 * v[p] + (1.0f - a.b2) * gr * gr;
  m[p] = mm;
  v[p] = vv;
  const float mh = mm / a.c1, vh = vv / a.c2;
  const float nw = w[p] - a.lr * mh / (sqrtf(vh) + a.eps);
  w[p] = nw;
  wb[p] = __float2bfloat16_rn(nw);
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kParams) wb[p] = __float2bfloat16_rn(w[p]);
}

}  // namespace mlp
}  // namespace rewl

using namespace rewl;
using namespace rewl::mlp;

struct rewl_mlp {
  Net net{};
  cudaStream_t stream = nullptr;
  float* d_w = nullptr;          // FP32 master
  __nv_bfloat16* d_wb = nullptr;  // BF16 copy used by the kernels
  float* d_grad = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  float* d_partial = nullptr;
  int grid = 0;                  // persistent CTAs of the backward pass (= rows of d_partial)
  long long adam_t = 0;
  std::vector<void*> allocations;
  bool broken = false;
};

namespace {

rewl_status mfail(rewl_mlp* m, rewl_status s, const std::string& msg) {
  if (m && s == REWL_ECUDA) m->broken = true;
  set_handleless_error("mlp: " + msg);
  return s;
}

#define MCUDA(m, call)                                                                                  \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return mfail((m), REWL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
rewl_status malloc_dev(rewl_mlp* m, T** p, size_t count) {
  void* q = nullptr;
  const cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return mfail(m, REWL_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  m->allocations.push_back(q);
  *p = static_cast<T*>(q);
  return REWL_OK;
}

// device scratch of one call, freed on return
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  cudaError_t get(T** p, size_t count) {
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) {
      ptrs.push_back(q);
      *p = static_cast<T*>(q);
    }
    return e;
  }
};

rewl_status check_mlp(rewl_mlp* m) {
  if (!m) return mfail(nullptr, REWL_EINVAL, "null model");
  if (m->broken) return mfail(m, REWL_ESTATE, "model saw a CUDA error; destroy it");
  return REWL_OK;
}

int fwd_grid(long long n) {
  const long long tiles = (n + kT - 1) / kT;
  return (int)std::max<long long>(1, std::min<long long>(tiles, 4 * 152));
}

rewl_status check_segments(const int32_t* seg, int n_segs, long long n) {
  if (!seg || n_segs < 1) return mfail(nullptr, REWL_EINVAL, "no runs");
  if (seg[0] != 0 || seg[n_segs] != n) return mfail(nullptr, REWL_EINVAL, "run offsets must start at 0 and end at n");
  for (int g = 0; g < n_segs; ++g)
    if (seg[g + 1] <= seg[g]) return mfail(nullptr, REWL_EINVAL, "run offsets must increase");
  return REWL_OK;
}

// Loss and gradient of the full batch into m->d_grad; loss (FP64) to *loss.
rewl_status loss_and_grad(rewl_mlp* m, const float* dx, const float* dt, const int* dseg, int n_segs, long long n,
                          float* dy_buf, float* dydy, double* dloss, double* loss) {
  const size_t smem = sizeof(Smem);
  mlp_fwd_kernel<<<fwd_grid(n), kThreads, smem, m->stream>>>(m->net, dx, n, dy_buf);
  MCUDA(m, cudaGetLastError());
  mlp_loss_kernel<<<n_segs, 256, 0, m->stream>>>(dy_buf, dt, dseg, 1.0f / (float)n, dydy, dloss);
  MCUDA(m, cudaGetLastError());
  MCUDA(m, cudaMemsetAsync(m->d_partial, 0, sizeof(float) * (size_t)m->grid * kParams, m->stream));
  mlp_bwd_kernel<<<m->grid, kThreads, smem, m->stream>>>(m->net, dx, dydy, n, m->d_partial);
  MCUDA(m, cudaGetLastError());
  mlp_reduce_kernel<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->d_partial, m->grid, m->d_grad);
  MCUDA(m, cudaGetLastError());
  if (loss) {
    std::vector<double> parts(n_segs);
    MCUDA(m, cudaMemcpyAsync(parts.data(), dloss, sizeof(double) * (size_t)n_segs, cudaMemcpyDeviceToHost,
                             m->stream));
    MCUDA(m, cudaStreamSynchronize(m->stream));
    double s = 0.0;
    for (double v : parts) s += v;
    *loss = s / (double)n;
  }
  return REWL_OK;
}

struct Corpus {
  Scratch sc;
  float *x = nullptr, *t = nullptr, *y = nullptr, *dy = nullptr;
  int* seg = nullptr;
  double* loss = nullptr;
};

rewl_status upload_corpus(rewl_mlp* m, Corpus& c, const float* x, const float* t, const int32_t* seg, int n_segs) {
  const long long n = seg[n_segs];
  MCUDA(m, c.sc.get(&c.x, (size_t)n * kIn));
  MCUDA(m, c.sc.get(&c.t, (size_t)n));
  MCUDA(m, c.sc.get(&c.y, (size_t)n));
  MCUDA(m, c.sc.get(&c.dy, (size_t)n));
  MCUDA(m, c.sc.get(&c.seg, (size_t)n_segs + 1));
  MCUDA(m, c.sc.get(&c.loss, (size_t)n_segs));
  MCUDA(m, cudaMemcpyAsync(c.x, x, sizeof(float) * (size_t)n * kIn, cudaMemcpyHostToDevice, m->stream));
  MCUDA(m, cudaMemcpyAsync(c.t, t, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, m->stream));
  MCUDA(m, cudaMemcpyAsync(c.seg, seg, sizeof(int) * ((size_t)n_segs + 1), cudaMemcpyHostToDevice, m->stream));
  return REWL_OK;
}

}  // namespace

extern "C" int64_t rewl_mlp_param_count(void) { return kParams; }

extern "C" rewl_status rewl_mlp_create(const float* in_shift, const float* in_scale, uint64_t seed, void* cuda_stream,
                                       rewl_mlp** out) {
  if (!out) return mfail(nullptr, REWL_EINVAL, "NULL out");
  *out = nullptr;
  if (!in_shift || !in_scale) return mfail(nullptr, REWL_EINVAL, "NULL input normalisation");
  for (int k = 0; k < kIn; ++k)
    if (!std::isfinite(in_shift[k]) || !std::isfinite(in_scale[k]) || in_scale[k] == 0.0f)
      return mfail(nullptr, REWL_EINVAL, "input normalisation must be finite with nonzero scales");
  auto* m = new rewl_mlp();
  for (int k = 0; k < kIn; ++k) {
    m->net.shift[k] = in_shift[k];
    m->net.scale[k] = in_scale[k];
  }
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, n_sms = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = sizeof(Smem);
  if (ce == cudaSuccess)
    ce = cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (ce == cudaSuccess)
    ce = cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (ce != cudaSuccess) {
    delete m;
    return mfail(nullptr, REWL_ECUDA, std::string("CUDA set-up: ") + cudaGetErrorString(ce));
  }
  m->grid = std::max(1, n_sms);
  rewl_status s = malloc_dev(m, &m->d_w, kParams);
  if (s == REWL_OK) s = malloc_dev(m, &m->d_wb, kParams);
  if (s == REWL_OK) s = malloc_dev(m, &m->d_grad, kParams);
  if (s == REWL_OK) s = malloc_dev(m, &m->d_m, kParams);
  if (s == REWL_OK) s = malloc_dev(m, &m->d_v, kParams);
  if (s == REWL_OK) s = malloc_dev(m, &m->d_partial, (size_t)m->grid * kParams);
  if (s != REWL_OK) {
    rewl_mlp_destroy(m);
    return s;
  }
  m->net.p = m->d_wb;
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, from a seeded generator
  std::vector<float> w(kParams, 0.0f);
  std::mt19937_64 gen(seed);
  auto fill = [&](int off, int count, int fan_in) {
    std::uniform_real_distribution<float> d(-1.0f / std::sqrt((float)fan_in), 1.0f / std::sqrt((float)fan_in));
    for (int i = 0; i < count; ++i) w[off + i] = d(gen);
  };
  fill(oW1, kIn * kH, kIn);
  fill(oW2, kH * kH, kH);
  fill(oW3, kH * kH, kH);
  fill(oW4, kH, kH);
  s = rewl_mlp_set_params(m, w.data());
  if (s != REWL_OK) {
    rewl_mlp_destroy(m);
    return s;
  }
  *out = m;
  return REWL_OK;
}

extern "C" rewl_status rewl_mlp_set_params(rewl_mlp* m, const float* params) {
  rewl_status s = check_mlp(m);
  if (s != REWL_OK) return s;
  if (!params) return mfail(m, REWL_EINVAL, "NULL params");
  MCUDA(m, cudaMemcpyAsync(m->d_w, params, sizeof(float) * kParams, cudaMemcpyHostToDevice, m->stream));
  to_bf16_kernel<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->d_w, m->d_wb);
  MCUDA(m, cudaGetLastError());
  MCUDA(m, cudaMemsetAsync(m->d_m, 0, sizeof(float) * kParams, m->stream));
  MCUDA(m, cudaMemsetAsync(m->d_v, 0, sizeof(float) * kParams, m->stream));
  MCUDA(m, cudaStreamSynchronize(m->stream));
  m->adam_t = 0;
  return REWL_OK;
}

extern "C" rewl_status rewl_mlp_get_params(rewl_mlp* m, float* params, uint16_t* params_bf16) {
  rewl_status s = check_mlp(m);
  if (s != REWL_OK) return s;
  if (params)
    MCUDA(m, cudaMemcpyAsync(params, m->d_w, sizeof(float) * kParams, cudaMemcpyDeviceToHost, m->stream));
  if (params_bf16)
    MCUDA(m, cudaMemcpyAsync(params_bf16, m->d_wb, sizeof(uint16_t) * kParams, cudaMemcpyDeviceToHost, m->stream));
  MCUDA(m, cudaStreamSynchronize(m->stream));
  return REWL_OK;
}

extern "C" rewl_status rewl_mlp_forward(rewl_mlp* m, const float* x, int64_t n, float* y) {
  rewl_status s = check_mlp(m);
  if (s != REWL_OK) return s;
  if (!x || !y || n < 1) return mfail(m, REWL_EINVAL, "bad forward arguments");
  Corpus c;
  MCUDA(m, c.sc.get(&c.x, (size_t)n * kIn));
  MCUDA(m, c.sc.get(&c.y, (size_t)n));
  MCUDA(m, cudaMemcpyAsync(c.x, x, sizeof(float) * (size_t)n * kIn, cudaMemcpyHostToDevice, m->stream));
  mlp_fwd_kernel<<<fwd_grid(n), kThreads, sizeof(Smem), m->stream>>>(m->net, c.x, n, c.y);
  MCUDA(m, cudaGetLastError());
  MCUDA(m, cudaMemcpyAsync(y, c.y, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, m->stream));
  MCUDA(m, cudaStreamSynchronize(m->stream));
  return REWL_OK;
}

extern "C" rewl_status rewl_mlp_gradient(rewl_mlp* m, const float* x, const float* target, const int32_t* run_offsets,
                                         int n_runs, double* loss, float* grad) {
  rewl_status s = check_mlp(m);
  if (s != REWL_OK) return s;
  if (!x || !target) return mfail(m, REWL_EINVAL, "NULL corpus");
  s = check_segments(run_offsets, n_runs, run_offsets ? run_offsets[n_runs] : 0);
  if (s != REWL_OK) return s;
  Corpus c;
  s = upload_corpus(m, c, x, target, run_offsets, n_runs);
  if (s != REWL_OK) return s;
  s = loss_and_grad(m, c.x, c.t, c.seg, n_runs, run_offsets[n_runs], c.y, c.dy, c.loss, loss);
  if (s != REWL_OK) return s;
  if (grad) MCUDA(m, cudaMemcpyAsync(grad, m->d_grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost, m->stream));
  MCUDA(m, cudaStreamSynchronize(m->stream));
  return REWL_OK;
}

extern "C" rewl_status rewl_mlp_train(rewl_mlp* m, const float* x, const float* target, const int32_t* run_offsets,
                                      int n_runs, int steps, float lr, float* loss_history) {
  rewl_status s = check_mlp(m);
  if (s != REWL_OK) return s;
  if (!x || !target || steps < 1 || !(lr > 0.0f)) return mfail(m, REWL_EINVAL, "bad training arguments");
  s = check_segments(run_offsets, n_runs, run_offsets ? run_offsets[n_runs] : 0);
  if (s != REWL_OK) return s;
  const long long n = run_offsets[n_runs];
  Corpus c;
  s = upload_corpus(m, c, x, target, run_offsets, n_runs);
  if (s != REWL_OK) return s;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int it = 0; it < steps; ++it) {
    double L = 0.0;
    s = loss_and_grad(m, c.x, c.t, c.seg, n_runs, n, c.y, c.dy, c.loss, loss_history ? &L : nullptr);
    if (s != REWL_OK) return s;
    if (loss_history) loss_history[it] = (float)L;
    m->adam_t += 1;
    AdamArgs a{};
    a.lr = lr;
    a.b1 = b1;
    a.b2 = b2;
    a.eps = eps;
    a.c1 = 1.0f - std::pow(b1, (float)m->adam_t);
    a.c2 = 1.0f - std::pow(b2, (float)m->adam_t);
    mlp_adam_kernel<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->d_w, m->d_grad, m->d_m, m->d_v, m->d_wb, a);
    MCUDA(m, cudaGetLastError());
  }
  MCUDA(m, cudaStreamSynchronize(m->stream));
  return REWL_OK;
}

extern "C" rewl_status rewl_mlp_features(const rewl_handle* h, const double* lng, float* x_out, float* t_out) {
  if (!h || !x_out) return mfail(nullptr, REWL_EINVAL, "NULL argument");
  if (t_out && !lng) return mfail(nullptr, REWL_EINVAL, "targets need ln g");
  JobView v;
  job_view(h, &v);
  if (v.kind != REWL_LATTICE_BCC) return mfail(nullptr, REWL_EINVAL, "features are defined for bcc jobs");
  double Jsh[4] = {0, 0, 0, 0}, e_min = 0, dE = 0;
  job_couplings(h, Jsh, &e_min, &dE);
  const int B = job_bins(h);
  for (int b = 0; b < B; ++b) {
    const double e = (e_min + (b + 0.5) * dE) / (double)v.N;
    float* r = x_out + (size_t)b * kIn;
    r[0] = (float)e;
    r[1] = (float)(1.0 / (double)v.L);
    for (int s = 0; s < 4; ++s) r[2 + s] = (float)Jsh[s];
    if (t_out) t_out[b] = (float)(lng[b] / (double)v.N);
  }
  return REWL_OK;
}

extern "C" rewl_status rewl_mlp_warm_start(rewl_mlp* m, rewl_handle* h, double lnf0, double* lng_out) {
  rewl_status s = check_mlp(m);
  if (s != REWL_OK) return s;
  if (!h || !(lnf0 > 0.0)) return mfail(m, REWL_EINVAL, "bad warm-start arguments");
  const int B = job_bins(h);
  JobView v;
  job_view(h, &v);
  std::vector<float> x((size_t)B * kIn), y(B);
  s = rewl_mlp_features(h, nullptr, x.data(), nullptr);
  if (s != REWL_OK) return s;
  s = rewl_mlp_forward(m, x.data(), B, y.data());
  if (s != REWL_OK) return s;
  std::vector<double> lng(B);
  for (int b = 0; b < B; ++b) lng[b] = (double)y[b] * (double)v.N;
  if (lng_out) std::copy(lng.begin(), lng.end(), lng_out);
  s = rewl_set_initial_lng(h, lng.data(), lnf0);
  if (s != REWL_OK) return mfail(m, s, std::string("set_initial_lng: ") + rewl_last_error(h));
  return REWL_OK;
}

extern "C" void rewl_mlp_destroy(rewl_mlp* m) {
  if (!m) return;
  if (!m->broken) cudaStreamSynchronize(m->stream);
  for (void* p : m->allocations) cudaFree(p);
  delete m;
}
