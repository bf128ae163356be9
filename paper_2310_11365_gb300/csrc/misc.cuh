// misc.cuh -- launchers of the small utility kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mmp {

// wrap != 0: shift each value modulo 2 pi into [-pi, pi] (plane rotator)
cudaError_t launch_init_u0(int precision, void* u0, long long P, int Q, double m0, double s0,
                           uint32_t k0, uint32_t k1, uint32_t ptag, int wrap, cudaStream_t s);
cudaError_t launch_philox(const unsigned* ctr, uint32_t k0, uint32_t k1, unsigned* out, long long n,
                          cudaStream_t s);
cudaError_t launch_normals(int precision, void* out, long long count, uint32_t tag, uint32_t j,
                           uint32_t n, uint32_t k0, uint32_t k1, uint32_t ptag, cudaStream_t s);

}  // namespace mmp
