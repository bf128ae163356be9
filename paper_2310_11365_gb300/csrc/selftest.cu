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
