// fine.cuh -- arguments and launch interface of the fused fine-propagator
// kernel (matching prologue, Euler-Maruyama steps with the per-step mean
// field, restriction epilogue).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mmp {

struct FineArgs {
  // drift a(x, m) = nc3 x^3 + c1 x + kappa m + c0 (nc3 = -c3), diffusion b = B x + BE m + B0
  double nc3, c1, kappa, c0, B, BE, B0;
  // plane rotator (family kFamRotator): a(x) = K (S cos x - C sin x) - g sin x, b = B0
  double K = 0.0, gpin = 0.0;
  double h, sqrt_h;            // fine step and its square root
  int nf;                      // steps per slice (0: matching + restriction only)
  long long P;                 // particles
  int Q;                       // quads = ceil(P / 4)
  long long pitch;             // elements between slice rows (multiple of 4)
  int n_regions;               // 1 .. kMaxRegions
  double thr, thr2, thr3;      // region boundaries t_1 < t_2 < t_3 (the first n_regions - 1)
  uint32_t key0, key1, ptag;   // Philox key and problem tag
  int slice_begin, n_tasks;    // task t is slice slice_begin + t
  const void* src0;            // input of slice 0, and of every slice when src == nullptr
  const void* src;             // rows: input of slice n is row n - 1
  void* dst;                   // output rows (nullptr: no store)
  int dst_fixed;               // 1: every task writes row 0
  const double* aff;           // matching records [row][kMaxRegions][kAff] (nullptr: identity)
  int aff_fixed;
  double* stats;               // restriction records [row][kStat]
  int stats_fixed;
  int G;                       // CTAs per slice
  int nq;                      // quads per thread (shared-memory layout)
  double* partials;            // [slot][G][kSlots][kNV] doubles: group publication slots
  unsigned* flags;             // [slot][G] epoch flags (zeroed per launch)
  unsigned long long* tags;    // [slot][kSlots][G] tagged step words (zeroed per launch)
  unsigned* status;            // device status word
  unsigned long long wait_limit_ns;
  int tight_polls = 0;         // polls before a group wait backs off (launches of <= 1 CTA per SM)
  // optional recording for the adjoint (serial runs only, one task):
  void* rec_uni = nullptr;     // [global step][3], precision R: (m_j, h (kappa m_j + c0), B0 sqrt h) in the
                               // shift form, (m_j, kappa m_j + c0, (BE m_j + B0) sqrt h) in the general form
  void* rec_ckpt = nullptr;    // particle rows at global steps 0, c, 2c, ... (row gstep / c)
  int ckpt_every = 1;          // c
  long long step_offset = 0;   // global index of this slice's first step
};

// Particle layouts of the fine kernel: quads in registers (a template per
// quads-per-thread count) or in dynamic shared memory (any count).
constexpr int kLayoutRegs = 0;
constexpr int kLayoutSmem = 1;

// Handle of one kernel instantiation (nq ignored for the shared layout;
// the plane rotator has the shared layout only, nullptr otherwise).
const void* fine_kernel(int precision, int layout, int nq, bool mult, int family = 0);
// Dynamic shared memory of a launch (three values per particle for the
// plane rotator: x, sin x, cos x).
size_t fine_smem_bytes(int precision, int layout, int nq, int family = 0);
// Cooperative launch of the instantiation (grid = slots * G CTAs).
cudaError_t launch_fine(int precision, int layout, int nq, bool mult, int grid, const FineArgs& args,
                        cudaStream_t stream, int family = 0);

}  // namespace mmp
