// adjoint.cuh -- arguments of the reverse (adjoint) kernel of the serial fine
// propagator.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mmp {

constexpr int kNGrad = 7;    // d/d(c3, c1, kappa, c0, B0, B, BE): MMP_N_THETA
constexpr int kAdjTPB = 512;  // threads per CTA of the reverse kernel

struct AdjointArgs {
  double nc3, c1, kappa, h, sqrt_h;  // model (nc3 = -c3), step
  double B, BE;                      // diffusion b = B x + BE m + B0 (B0 enters through the recording)
  int nf;                            // steps per slice
  long long J;                       // total steps N * nf
  int c;                             // checkpoint interval
  int n_seg;                         // ceil(J / c)
  long long P;
  int Q;
  long long pitch;
  uint32_t key0, key1, ptag;
  int G, nq;                         // CTAs (one group), quads per thread
  const void* ckpt;                  // rows at steps 0, c, 2c, ... (n_seg rows)
  const void* uni;                   // [J][3] recorded per step: (m_j, h (kappa m_j + c0), B0 sqrt h) for
                                     // additive noise, (m_j, kappa m_j + c0, (BE m_j + B0) sqrt h) otherwise
  void* segx;                        // 2 x (c + 1) rows: replayed states, two segment buffers
  void* segz;                        // 2 x c rows: the draws of the two segments (general form)
  const double* mom;                 // [(N+1)][kStat] restriction records of the serial run
  const double* gm;                  // [N] cotangents of the slice-end means (n = 1..N)
  const double* gv;                  // [N] cotangents of the slice-end variances
  double* grad;                      // [kNGrad] out: d/d(c3, c1, kappa, c0, B0, B, BE)
  double* partials;                  // [G][kSlots][kNV] group publication slots
  unsigned* flags;                   // [G] epoch flags (zeroed per launch)
  unsigned long long* tags;          // [kSlots][G] tagged step words (zeroed per launch)
  unsigned* status;
  unsigned long long wait_limit_ns;
  int sms;                           // SMs of the device
};

// mult: the general-diffusion form (B or BE nonzero)
const void* adjoint_kernel(int precision, bool mult);
size_t adjoint_smem_bytes(int precision, int nq);
cudaError_t launch_adjoint(int precision, bool mult, const AdjointArgs& args, cudaStream_t stream);

}  // namespace mmp
