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

namespace mmp {

// Ceiling of the fine step's arithmetic without the cross-CTA exchange
// (mmp_probe_step): the additive-noise step of float particles exactly as
// the fine kernel evaluates it (Philox-4x32-10, the polar Box-Muller form,
// the mean-free partial step, the pending shift and the per-thread sum),
// on particles that stay on chip for every step.
//   form 0: kProbeQuads quads per thread in registers, no synchronisation;
//   form 1: nq quads per thread in dynamic shared memory (the fine kernel's
//           layout) with a warp butterfly and a CTA barrier every step.
// The sums are stored only if they take a value they never take, which
// keeps every chain alive.
constexpr int kProbeQuads = 4;

struct StepProbeCoef {
  uint32_t k0, k1, n, tag;  // Philox key, slice index and problem tag (runtime values, as in the fine kernel)
  float hn3, hc1, amp, d;
};

template <bool SMEM>
__global__ void __launch_bounds__(kTPB, 2) k_step_probe(float* sink, int steps, int nq, StepProbeCoef cf) {
  __shared__ float red[kWarps];
  constexpr int NQ = SMEM ? 0 : kProbeQuads;
  QuadStore<float, NQ> xs;
  xs.bind();
  const int loop_n = SMEM ? nq : kProbeQuads;
#pragma unroll kProbeQuads
  for (int i = 0; i < loop_n; ++i) {
    float v[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) v[w] = 0.01f * (float)(w + 1 + (threadIdx.x & 7));
    xs.put(i, v);
  }
  const uint32_t q0 = blockIdx.x * kTPB * loop_n + threadIdx.x;
  float acc = 0.0f;
  float d = cf.d;
  for (int j = 0; j < steps; ++j) {
    float s = 0.0f;
#pragma unroll kStepUnrollSmem
    for (int i = 0; i < loop_n; ++i) {
      float v[4];
      xs.get(i, v);
      const uint4 o = philox4x32_10(rng_counter(q0 + i * kTPB, (uint32_t)j, cf.n, 0u, cf.tag), cf.k0, cf.k1);
      float nr[2], c[2], sn[2];
      normals4_polar<float>(o, nr, c, sn);
#pragma unroll
      for (int w = 0; w < 4; ++w) v[w] = addR(v[w], d);
      em_partial_pair(v[0], v[1], nr[0], c[0], sn[0], cf.hn3, cf.hc1, cf.amp);
      em_partial_pair(v[2], v[3], nr[1], c[1], sn[1], cf.hn3, cf.hc1, cf.amp);
      s = addR(s, addR(addR(v[0], v[1]), addR(v[2], v[3])));
      xs.put(i, v);
    }
    if (SMEM) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
      __syncthreads();
      float t = 0.0f;
#pragma unroll
      for (int k = 0; k < kWarps; ++k) t += red[k];
      d = cf.d + 1e-12f * t;
      __syncthreads();
    }
    acc += s;
  }
  if (acc == -1.25e-30f) sink[0] = acc;
}

int step_probe_quads(int form) { return form == 0 ? kProbeQuads : 26; }

size_t step_probe_smem(int form) {
  return form == 0 ? 0 : (size_t)kTPB * step_probe_quads(form) * 4 * sizeof(float);
}

cudaError_t prepare_step_probe(int form) {
  if (form == 0) return cudaSuccess;
  return cudaFuncSetAttribute(k_step_probe<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)step_probe_smem(form));
}

cudaError_t launch_step_probe(int form, float* sink, int steps, int grid, cudaStream_t stream) {
  const float h = 1e-3f;
  // the config-2 model: c3 = 1, c1 = -1, sigma = 0.5, dt = 1e-3
  const StepProbeCoef cf{0x1234567u, 0x89abcdefu, 3u, 7u, -h, -h, 0.5f * sqrtf(h), 0.05f * h};
  if (form == 0)
    k_step_probe<false><<<grid, kTPB, 0, stream>>>(sink, steps, kProbeQuads, cf);
  else
    k_step_probe<true><<<grid, kTPB, step_probe_smem(form), stream>>>(sink, steps, step_probe_quads(form), cf);
  return cudaGetLastError();
}

}  // namespace mmp
