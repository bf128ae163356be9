// Test probe: runs cuRAND's device Philox-4x32-10 (curand_Philox4x32_10 from
// curand_philox4x32_x.h) on given counters so the library's own generator
// can be compared with an independent implementation.  Test code only.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void k_ref(const uint4* ctr, uint2 key, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key);
}

extern "C" int curand_philox_ref(const unsigned* ctr_host, const unsigned* key, unsigned* out_host, int n) {
  uint4 *d_ctr = nullptr, *d_out = nullptr;
  if (cudaMalloc(&d_ctr, sizeof(uint4) * n) != cudaSuccess) return 1;
  if (cudaMalloc(&d_out, sizeof(uint4) * n) != cudaSuccess) return 2;
  cudaMemcpy(d_ctr, ctr_host, sizeof(uint4) * n, cudaMemcpyHostToDevice);
  k_ref<<<(n + 127) / 128, 128>>>(d_ctr, make_uint2(key[0], key[1]), d_out, n);
  cudaError_t e = cudaMemcpy(out_host, d_out, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
  cudaFree(d_ctr);
  cudaFree(d_out);
  return e == cudaSuccess ? 0 : 3;
}
