// selftest.cu -- the failure detection of the group exchange, exercised on
// the device: one CTA of a G-CTA group runs a group reduction whose peers
// never publish, so its bounded wait must run out, set the timeout bit of
// the status word and let the kernel return (no trap, no hang).
#include "fine_kernel.cuh"

namespace mmp {

// channel 0: the record channel (release/acquire epoch flags, group_finish);
// channel 1: the tagged 8-byte step words of float particles.
__global__ void __launch_bounds__(kTPB) k_wait_probe(double* partials, unsigned* flags, unsigned long long* tags,
                                                     unsigned* status, int G, unsigned long long limit_ns,
                                                     int channel) {
  __shared__ GroupShared sh;
  Group grp;
  grp.part = partials;
  grp.flags = flags;
  grp.tags = tags;
  grp.status = status;
  grp.limit_ns = limit_ns;
  grp.G = G;
  grp.g = 0;
  grp.epoch = 0;
  grp.tight_polls = 0;
  const int warp = threadIdx.x >> 5;
  if (channel == 0) {
    double v[1] = {1.0};
    warp_reduce_to_shared<1>(sh, v, 0u, 0u);
    __syncthreads();
    if (warp == 0) group_finish<1>(sh, grp, 0u, 0u, 0u);
  } else if (warp == 0) {
    StepSum<float>::publish(grp, 0u, make_float2(1.0f, 0.0f));
    float2 s;
    StepSum<float>::fetch(grp, 0u, s);
  }
  __syncthreads();
}

cudaError_t launch_wait_probe(double* partials, unsigned* flags, unsigned long long* tags, unsigned* status, int G,
                              unsigned long long limit_ns, int channel, cudaStream_t stream) {
  k_wait_probe<<<1, kTPB, 0, stream>>>(partials, flags, tags, status, G, limit_ns, channel);
  return cudaGetLastError();
}

}  // namespace mmp

namespace mmp {

// FMA throughput probe: every thread runs 8 independent chains
// x <- fma(x, a, b) for `iters` iterations; the sum is stored only if it
// takes a value it never takes, which keeps every chain alive.
template <typename R>
__global__ void __launch_bounds__(kTPB) k_fma_probe(R* sink, long long iters, R a, R b) {
  R x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (R)(threadIdx.x + k) * (R)1e-3;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  R s = (R)0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (R)-1.25e-30) sink[0] = s;
}

cudaError_t launch_fma_probe(int precision, void* sink, long long iters, int grid, cudaStream_t stream) {
  if (precision == MMP_FP64)
    k_fma_probe<double><<<grid, kTPB, 0, stream>>>((double*)sink, iters, 0.999999, 1e-7);
  else
    k_fma_probe<float><<<grid, kTPB, 0, stream>>>((float*)sink, iters, 0.999999f, 1e-7f);
  return cudaGetLastError();
}

}  // namespace mmp
