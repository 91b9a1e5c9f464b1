// Test-only probe: cuRAND's Philox4x32-10 block function evaluated on the device for given
// counters and keys, so that the tests can pin both Philox implementations (the oracle's and the
// library's) against an independent library routine.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void probe_kernel(const uint4* ctr, const uint2* key, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_philox_probe(const uint32_t* ctr, const uint32_t* key, int n, uint32_t* out) {
  if (n <= 0) return 0;
  uint4 *dc = nullptr, *dout = nullptr;
  uint2* dk = nullptr;
  cudaError_t e = cudaMalloc(&dc, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(uint2) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dk, key, sizeof(uint2) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    probe_kernel<<<(n + 255) / 256, 256>>>(dc, dk, dout, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return (int)e;
}
