// misc.cu -- small kernels: the initial ensemble, and the raw generator
// outputs exposed for testing (Philox words, normals).
#include "misc.cuh"
#include "mmp_internal.cuh"

namespace mmp {

// X0 = m0 + s0 z with z the tag-1 normals; evaluated in FP64 and rounded to
// the particle type, so MMP_MIXED starts from the rounded FP64 ensemble.
// The plane rotator (wrap) shifts it into [-pi, pi] in FP64 first.
template <typename R>
__global__ void k_init_u0(R* u0, long long P, int Q, double m0, double s0, uint32_t k0, uint32_t k1,
                          uint32_t ptag, int wrap) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
    double z[4];
    normals4<double>(philox4x32_10(rng_counter((uint32_t)q, 0u, 0u, 1u, ptag), k0, k1), z);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const long long p = 4LL * q + w;
      double x = __dadd_rn(m0, __dmul_rn(s0, z[w]));
      if (wrap) x = wrap_angle(x);
      u0[p] = p < P ? (R)x : (R)0;
    }
  }
}

__global__ void k_philox(const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = philox4x32_10(ctr[i], k0, k1);
}

template <typename R>
__global__ void k_normals(R* out, long long count, uint32_t tag, uint32_t j, uint32_t n, uint32_t k0,
                          uint32_t k1, uint32_t ptag) {
  const long long quads = (count + 3) / 4;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < quads;
       q += (long long)gridDim.x * blockDim.x) {
    R z[4];
    normals4<R>(philox4x32_10(rng_counter((uint32_t)q, j, n, tag, ptag), k0, k1), z);
#pragma unroll
    for (int w = 0; w < 4; ++w)
      if (4 * q + w < count) out[4 * q + w] = z[w];
  }
}

static int grid_for(long long items, int block) {
  long long g = (items + block - 1) / block;
  if (g > 65535) g = 65535;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_init_u0(int precision, void* u0, long long P, int Q, double m0, double s0,
                           uint32_t k0, uint32_t k1, uint32_t ptag, int wrap, cudaStream_t s) {
  const int grid = grid_for(Q, 256);
  if (precision == MMP_MIXED)
    k_init_u0<float><<<grid, 256, 0, s>>>((float*)u0, P, Q, m0, s0, k0, k1, ptag, wrap);
  else
    k_init_u0<double><<<grid, 256, 0, s>>>((double*)u0, P, Q, m0, s0, k0, k1, ptag, wrap);
  return cudaGetLastError();
}

cudaError_t launch_philox(const unsigned* ctr, uint32_t k0, uint32_t k1, unsigned* out, long long n,
                          cudaStream_t s) {
  k_philox<<<grid_for(n, 256), 256, 0, s>>>((const uint4*)ctr, k0, k1, (uint4*)out, n);
  return cudaGetLastError();
}

cudaError_t launch_normals(int precision, void* out, long long count, uint32_t tag, uint32_t j,
                           uint32_t n, uint32_t k0, uint32_t k1, uint32_t ptag, cudaStream_t s) {
  const int grid = grid_for((count + 3) / 4, 256);
  if (precision == MMP_MIXED)
    k_normals<float><<<grid, 256, 0, s>>>((float*)out, count, tag, j, n, k0, k1, ptag);
  else
    k_normals<double><<<grid, 256, 0, s>>>((double*)out, count, tag, j, n, k0, k1, ptag);
  return cudaGetLastError();
}

}  // namespace mmp
