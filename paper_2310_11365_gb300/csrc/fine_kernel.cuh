// fine_kernel.cuh -- the fused fine-propagator kernel, templated on the
// particle precision R (float or double), the quads of particles held per
// thread NQ, whether the diffusion depends on the state (MULT), and the
// drift family FAM (the polynomial drift, or the plane rotator of Sec. 5).
//
// One slice of the Parareal sweep is one "task".  A task's P particles are
// split over a group of G co-resident CTAs (the launch is cooperative, so
// all CTAs are resident and a group barrier cannot deadlock).  Each thread
// keeps its quads of 4 particles on chip for all n_f steps: in shared memory
// (NQ = 0, the layout the planner uses, a.nq quads per thread) or in
// registers (NQ quads):
//
//   prologue  load u (coalesced 16-byte vectors), apply the matching T of
//             its region (Eq. multimodal_M), sum the inputs
//   steps     x += h a(x, m_j) + b(x, m_j) sqrt(h) xi   (Eq. Euler_Maruyama)
//             with xi from Philox(p/4, j, n, problem) and the mean m_j
//             reduced over the whole group (warp shuffles, a shared-memory
//             stage, then a cross-CTA stage through L2: one tagged 8-byte
//             word per CTA and step, read after a bounded wait; with
//             additive noise the exchange runs one step behind, see
//             fine_task)
//   epilogue  store x, restriction per region (Eq. multimodal_R): counts,
//             means, then centred sums, extremes (two passes, FP64)
//
// Every reduction runs in a fixed order (fixed particle-to-thread map,
// butterfly within warps, warps in index order, CTAs in index order), so a
// slice computed in a Parareal sweep and in the serial reference run is
// bit-identical.
#pragma once

#include <cfloat>
#include <cmath>

#include "fine.cuh"
#include "mmp_internal.cuh"

namespace mmp {

template <typename R>
struct Quad;
template <>
struct Quad<float> {
  static __device__ __forceinline__ void load(const float* p, float v[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  static __device__ __forceinline__ void store(float* p, const float v[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Quad<double> {
  static __device__ __forceinline__ void load(const double* p, double v[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  static __device__ __forceinline__ void store(double* p, const double v[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

// Per-CTA shared state of the group reductions.
template <int NW>
struct GroupSharedT {
  double red[NW][kNV];        // per-warp partials of the restriction reductions
  float2 redf[2][NW];         // per-warp double-float partials of the per-step sum (by step parity)
  double redd[2][NW];         // the same for double particles
  float2 gsumf[2];            // group sum of a step, handed from warp 0 to the CTA (by parity)
  double gsumd[2];
  double tot[kNV];            // group totals, broadcast
  float cf[16];               // float copies of the task's coefficients (see fine_task)
  float afff[kMaxRegions][3]; // the task's matching records (a, b, c) per region, float particles
  double affd[kMaxRegions][3];// the same for double particles
  int amode[kMaxRegions];     // their modes
  float cr[2];                // plane rotator: K, g as floats
  double rotd[2];             // plane rotator: ensemble means of sin X, cos X before a step
  float rotf[2];              // the same rounded to float
  int abort;
};
// The fine kernels' CTAs have kWarps warps.
using GroupShared = GroupSharedT<kWarps>;

// A compile-time region count (the prologue and the epilogue are compiled
// for at most 2 and for at most 4 regions; a task takes the first when it can).
template <int N>
struct RegionsUpTo {
  static constexpr int value = N;
};

// A compile-time switch (the step body is compiled with and without the
// checkpoint store, so that no branch splits the unrolled quads).
template <bool B>
struct Switch {
  static constexpr bool value = B;
};

// Region index of x: D_0 = {x < t1}, D_i = {t_i <= x < t_{i+1}}, D_{I-1} = {x >= t_{I-1}}.
template <typename R>
__device__ __forceinline__ int region_of(R x, int I, R t1, R t2, R t3) {
  if (I < 2 || x < t1) return 0;
  if (I < 3 || x < t2) return 1;
  if (I < 4 || x < t3) return 2;
  return 3;
}

// Group-reduction context of one CTA.
//
// Epochs number the group reductions of a CTA in program order; every CTA
// of a group runs the same sequence.  Two publication channels, each a ring
// of kSlots entries per CTA indexed by epoch:
//
// * records of up to kNV doubles: publishing epoch e writes slot e mod
//   kSlots, then stores e + 1 to the CTA's flag with release semantics; a
//   reader acquires the flag (>= e + 1) before it reads the slot;
// * per-step sums of float particles: one 8-byte word (hi, lo) whose low 16
//   bits of lo are replaced by a tag of the epoch, written and read with
//   single-copy-atomic relaxed accesses, so the word is its own flag (one
//   L2 round trip per read, no fence on the writer).  Dropping those bits
//   of lo leaves the pair accurate to about 2^-32 relative.
//
// A CTA publishes epoch e only after it has seen epoch e - 2 complete, and
// every CTA reads an epoch before it publishes the epoch after next, so no
// entry is rewritten before every CTA has read it (kSlots = 4 leaves one
// spare).
struct Group {
  double* part;             // [G][kSlots][kNV] record slots of this group
  unsigned* flags;          // [G] 1 + last record epoch published (zeroed per launch)
  unsigned long long* tags; // [kSlots][G] tagged step words (zeroed per launch)
  unsigned* status;
  unsigned long long limit_ns;
  int G, g;
  unsigned epoch;           // epochs published so far by this CTA
  int tight_polls = 0;      // polls before a wait backs off (kTightPolls or 0)
};


__device__ __forceinline__ double* group_slot(const Group& grp, int c, unsigned e) {
  return grp.part + ((size_t)c * kSlots + (e & (unsigned)(kSlots - 1))) * kNV;
}

// One thread: publish nv values as epoch e of this CTA.
__device__ __forceinline__ void group_publish(const Group& grp, unsigned e, const double* v, int nv) {
  double* s = group_slot(grp, grp.g, e);
  for (int k = 0; k < nv; ++k) __stcg(s + k, v[k]);
  st_release_gpu(grp.flags + grp.g, e + 1u);
}

// Whole warp: bounded wait until every CTA of the group has published
// epoch e.  Lane l acquires the flags of CTAs l, l + 32, ... and is the lane
// that reads those CTAs' slots afterwards.  On timeout the status word gets
// the timeout bit (which also releases every other waiter) and the result
// is false.
__device__ __forceinline__ bool group_wait(const Group& grp, unsigned e) {
  bool ok = true;
  for (int c = threadIdx.x & 31; c < grp.G && ok; c += 32) {
    if (ld_acquire_gpu(grp.flags + c) > e) continue;
    const unsigned long long t0 = globaltimer_ns();
    for (int spin = 0;; ++spin) {
      if (spin >= grp.tight_polls) __nanosleep(64);
      if (ld_acquire_gpu(grp.flags + c) > e) break;
      if (globaltimer_ns() - t0 > grp.limit_ns) {
        atomicOr(grp.status, kStatusTimeout);
        ok = false;
        break;
      }
      if (*(volatile unsigned*)grp.status & kStatusTimeout) {
        ok = false;
        break;
      }
    }
  }
  return __all_sync(0xffffffffu, ok);
}

// Warp 0 finishes a group reduction of NV values whose per-warp partials
// sit in sh.red: the CTA's values (warps in index order) are published as
// epoch e and the group's totals (CTAs in index order) land in sh.tot.
// min_mask / max_mask select values combined by min / max (all others are
// summed).  Every thread of the CTA advances grp.epoch past e itself.
// Returns false if the wait gave up.
template <int NV, int NW>
__device__ __forceinline__ bool group_finish(GroupSharedT<NW>& sh, const Group& grp, unsigned e, unsigned min_mask,
                                             unsigned max_mask) {
  const int lane = threadIdx.x & 31;
  auto comb = [&](int k, double x, double o) {
    return (min_mask >> k & 1) ? fmin(x, o) : ((max_mask >> k & 1) ? fmax(x, o) : x + o);
  };
  auto ident = [&](int k) {
    return (min_mask >> k & 1) ? (double)INFINITY : ((max_mask >> k & 1) ? -(double)INFINITY : 0.0);
  };
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = lane < NW ? sh.red[lane][k] : ident(k);
#pragma unroll
  for (int off = NW / 2; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = comb(k, v[k], __shfl_xor_sync(0xffffffffu, v[k], off));
  }
  if (grp.G > 1) {
    if (lane == 0) group_publish(grp, e, v, NV);
    if (!group_wait(grp, e)) return false;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = ident(k);
    for (int c = lane; c < grp.G; c += 32) {
      const double* s = group_slot(grp, c, e);
#pragma unroll
      for (int k = 0; k < NV; ++k) v[k] = comb(k, v[k], __ldcg(s + k));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int k = 0; k < NV; ++k) v[k] = comb(k, v[k], __shfl_xor_sync(0xffffffffu, v[k], off));
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh.tot[k] = v[k];
  }
  return true;
}

// Double-float addition (hi, lo) + (b_hi, b_lo) with error-free two-sums;
// exact to about 2^-48 relative and free of FP64 instructions, which on
// this chip issue at a small fraction of the FP32 rate.  Commutative bit for
// bit, so every lane of a butterfly ends with the same pair.
__device__ __forceinline__ float2 dd_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  float hi, lo;
  two_sum(s, e, hi, lo);
  return make_float2(hi, lo);
}
__device__ __forceinline__ float2 shfl_xor_dd(float2 v, int off) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, off), __shfl_xor_sync(0xffffffffu, v.y, off));
}

// Per-thread accumulator: double-float for float data (no FP64 instruction
// per element), double otherwise.
template <typename R>
struct Acc;
template <>
struct Acc<float> {
  float2 v = make_float2(0.0f, 0.0f);
  __device__ __forceinline__ void add(float x) { v = dd_add(v, make_float2(x, 0.0f)); }
  __device__ __forceinline__ double get() const { return (double)v.x + (double)v.y; }
};
template <>
struct Acc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double get() const { return v; }
};

// x - m for an FP64 value m, evaluated in the particle precision: for float
// particles m is split into a float pair (hi, lo) and x - m = (x - hi) - lo.
template <typename R>
struct Centre;
template <>
struct Centre<float> {
  float hi, lo;
  Centre() = default;
  __device__ __forceinline__ explicit Centre(double m) : hi((float)m), lo((float)(m - (double)(float)m)) {}
  __device__ __forceinline__ float diff(float x) const { return __fsub_rn(__fsub_rn(x, hi), lo); }
};
template <>
struct Centre<double> {
  double m;
  Centre() = default;
  __device__ __forceinline__ explicit Centre(double mm) : m(mm) {}
  __device__ __forceinline__ double diff(double x) const { return x - m; }
};

// Plain arithmetic in the particle precision with explicit rounding (no
// contraction choices left to the compiler, so every kernel that inlines
// these rounds identically).
__device__ __forceinline__ float addR(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double addR(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mulR(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mulR(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float subR(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double subR(double a, double b) { return __dsub_rn(a, b); }

// The part of one Euler-Maruyama step that does not depend on the mean, for
// the two particles that share a Box-Muller pair (normals nr (c | s)):
//   y = x + h (nc3 x^3 + c1 x) + amp xi = fma(amp nr, c | s, fma(fma(hn3, x^2, hc1), x, x)),
// with hn3 = h nc3 and hc1 = h c1 and the amplitude folded into the radius
// once per pair.  The step is x_{j+1} = y + h (kappa m_j + c0), a shift
// common to all particles (the fine kernel and the adjoint's replay both
// evaluate it through this function).
template <typename R>
__device__ __forceinline__ void em_partial_pair(R& x0, R& x1, R nr, R c, R s, R hn3, R hc1, R amp) {
  const R ar = mulR(amp, nr);
  x0 = fmaR(ar, c, fmaR(fmaR(hn3, mulR(x0, x0), hc1), x0, x0));
  x1 = fmaR(ar, s, fmaR(fmaR(hn3, mulR(x1, x1), hc1), x1, x1));
}

// The per-step sum of the particles: a double-float pair for float
// particles (no FP64 instruction in the step loop), a double otherwise.
// Stages: per-thread sum in the particle precision, warp butterfly, warps
// in index order, CTAs of the group in index order.
template <typename R>
struct StepSum;
template <>
struct StepSum<float> {
  using T = float2;
  static __device__ __forceinline__ T zero() { return make_float2(0.0f, 0.0f); }
  static __device__ __forceinline__ T of(float s) { return make_float2(s, 0.0f); }
  static __device__ __forceinline__ T add(T a, T b) { return dd_add(a, b); }
  static __device__ __forceinline__ T shfl_xor(T v, int off) { return shfl_xor_dd(v, off); }
  static __device__ __forceinline__ T bcast0(T v) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, 0), __shfl_sync(0xffffffffu, v.y, 0));
  }
  template <class SH>
  static __device__ __forceinline__ T* warp_slots(SH& sh, int parity) { return sh.redf[parity]; }
  template <class SH>
  static __device__ __forceinline__ T& gsum(SH& sh, int parity) { return sh.gsumf[parity]; }
  static __device__ __forceinline__ uint32_t tag_of(unsigned e) { return 0x8000u | ((e + 1u) & 0x7FFFu); }
  // one thread: the CTA's value of epoch e as a tagged word
  static __device__ __forceinline__ void publish(const Group& grp, unsigned e, T v) {
    const uint32_t lo = (__float_as_uint(v.y) & 0xFFFF0000u) | tag_of(e);
    const unsigned long long w = ((unsigned long long)lo << 32) | __float_as_uint(v.x);
    st_relaxed_gpu_b64(grp.tags + (size_t)(e & (unsigned)(kSlots - 1)) * grp.G + grp.g, w);
  }
  // whole warp: bounded wait for the tagged words of epoch e of every CTA
  // (lane l reads CTAs l, l + 32, ...; a lane issues its loads of up to 256
  // CTAs before examining any), their sum in CTA order
  static __device__ __forceinline__ bool fetch(const Group& grp, unsigned e, T& sum) {
    const uint32_t tag = tag_of(e);
    const unsigned long long* row = grp.tags + (size_t)(e & (unsigned)(kSlots - 1)) * grp.G;
    const int lane = threadIdx.x & 31;
    T v = zero();
    bool ok = true;
    for (int base = 0; base < grp.G; base += 256) {
      unsigned long long w[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int c = base + lane + 32 * k;
        w[k] = c < grp.G ? ld_relaxed_gpu_b64(row + c) : 0ull;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int c = base + lane + 32 * k;
        if (c < grp.G) {
          if (ok && ((uint32_t)(w[k] >> 32) & 0xFFFFu) != tag) {
            w[k] = wait_word(grp, row + c, tag);
            ok = ((uint32_t)(w[k] >> 32) & 0xFFFFu) == tag;
          }
          v = add(v, make_float2(__uint_as_float((uint32_t)w[k]),
                                 __uint_as_float((uint32_t)(w[k] >> 32) & 0xFFFF0000u)));
        }
      }
    }
    if (grp.G == 1) {
      v = bcast0(v);
    } else {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v = add(v, shfl_xor(v, off));
    }
    sum = v;
    return __all_sync(0xffffffffu, ok);
  }
  // bounded wait (with back-off) until the word at p carries the tag; on
  // timeout the result is 0, whose tag (no bit 15) never matches
  static __device__ __noinline__ unsigned long long wait_word(const Group& grp, const unsigned long long* p,
                                                              uint32_t tag) {
    const unsigned long long t0 = globaltimer_ns();
    for (int spin = 0;; ++spin) {
      if (spin >= grp.tight_polls) __nanosleep(64);
      const unsigned long long w = ld_relaxed_gpu_b64(p);
      if (((uint32_t)(w >> 32) & 0xFFFFu) == tag) return w;
      if (globaltimer_ns() - t0 > grp.limit_ns) {
        atomicOr(grp.status, kStatusTimeout);
        return 0ull;
      }
      if (*(volatile unsigned*)grp.status & kStatusTimeout) return 0ull;
    }
  }
  // sum / P with inv_p = 1 / P rounded to float
  static __device__ __forceinline__ float mean(T v, float inv_p, long long) {
    return __fmaf_rn(v.x, inv_p, __fmul_rn(v.y, inv_p));
  }
};
template <>
struct StepSum<double> {
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T of(double s) { return s; }
  static __device__ __forceinline__ T add(T a, T b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ T shfl_xor(T v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
  static __device__ __forceinline__ T bcast0(T v) { return __shfl_sync(0xffffffffu, v, 0); }
  template <class SH>
  static __device__ __forceinline__ T* warp_slots(SH& sh, int parity) { return sh.redd[parity]; }
  template <class SH>
  static __device__ __forceinline__ T& gsum(SH& sh, int parity) { return sh.gsumd[parity]; }
  // one thread: the CTA's value of epoch e in its record slot, then its flag
  static __device__ __forceinline__ void publish(const Group& grp, unsigned e, T v) {
    __stcg(group_slot(grp, grp.g, e), v);
    st_release_gpu(grp.flags + grp.g, e + 1u);
  }
  // whole warp: bounded wait for epoch e of every CTA, the sum in CTA order
  static __device__ __forceinline__ bool fetch(const Group& grp, unsigned e, T& sum) {
    if (!group_wait(grp, e)) return false;
    T v = zero();
    for (int c = threadIdx.x & 31; c < grp.G; c += 32) v = add(v, __ldcg(group_slot(grp, c, e)));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = add(v, shfl_xor(v, off));
    sum = v;
    return true;
  }
  static __device__ __forceinline__ double mean(T v, float, long long P) { return __ddiv_rn(v, (double)P); }
};

// Per-warp stage: butterfly of the per-thread sums, lane 0 stores the warp's
// partial into the slot array of the step's parity.
template <typename R, int NW>
__device__ __forceinline__ void step_sum_warp(GroupSharedT<NW>& sh, int parity, R s) {
  using S = StepSum<R>;
  typename S::T v = S::of(s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = S::add(v, S::shfl_xor(v, off));
  if ((threadIdx.x & 31) == 0) S::warp_slots(sh, parity)[threadIdx.x >> 5] = v;
}

// Every warp, after the CTA barrier that follows step_sum_warp: the CTA's
// sum (warps in index order; the same value in every warp and lane).
template <typename R, int NW>
__device__ __forceinline__ typename StepSum<R>::T step_sum_cta(GroupSharedT<NW>& sh, int parity) {
  using S = StepSum<R>;
  const int lane = threadIdx.x & 31;
  typename S::T v = lane < NW ? S::warp_slots(sh, parity)[lane] : S::zero();
#pragma unroll
  for (int off = NW / 2; off > 0; off >>= 1) v = S::add(v, S::shfl_xor(v, off));
  return S::bcast0(v);
}

// General per-warp stage of nv double values.
template <int NV, int NW>
__device__ __forceinline__ void warp_reduce_to_shared(GroupSharedT<NW>& sh, double v[NV], unsigned min_mask,
                                                      unsigned max_mask) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double o = __shfl_xor_sync(0xffffffffu, v[k], off);
      v[k] = (min_mask >> k & 1) ? fmin(v[k], o) : ((max_mask >> k & 1) ? fmax(v[k], o) : v[k] + o);
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh.red[threadIdx.x >> 5][k] = v[k];
  }
}

// Where a thread keeps its quads of particles between steps.
// NQ > 0: in registers, NQ quads (loops over quads fully unrolled).
// NQ == 0: in dynamic shared memory, a.nq quads at stride TPB quads (the
// CTA's threads), so a warp touches 512 contiguous bytes per quad
// (conflict-free 16-byte accesses) and registers stay few, which lets more
// CTAs share an SM.
extern __shared__ __align__(16) unsigned char mmp_fine_smem[];

template <typename R, int NQ, int TPB = kTPB>
struct QuadStore {
  R x[NQ][4];
  __device__ __forceinline__ void bind() {}
  __device__ __forceinline__ void get(int i, R v[4]) const {
#pragma unroll
    for (int w = 0; w < 4; ++w) v[w] = x[i][w];
  }
  __device__ __forceinline__ void put(int i, const R v[4]) {
#pragma unroll
    for (int w = 0; w < 4; ++w) x[i][w] = v[w];
  }
};
template <typename R, int TPB>
struct QuadStore<R, 0, TPB> {
  R* base;
  __device__ __forceinline__ void bind() { base = reinterpret_cast<R*>(mmp_fine_smem) + 4 * threadIdx.x; }
  __device__ __forceinline__ void get(int i, R v[4]) const { Quad<R>::load(base + 4 * (size_t)i * TPB, v); }
  __device__ __forceinline__ void put(int i, const R v[4]) { Quad<R>::store(base + 4 * (size_t)i * TPB, v); }
};

// Resident CTAs per SM the register budget is sized for.  Register layout:
// the quads a thread holds dominate its registers, so fewer CTAs fit as NQ
// grows.  Shared-memory layout (NQ == 0): a slice's particles fill the
// shared memory of two CTAs per SM at the sizes that matter, so each thread
// gets 128 registers and keeps kStepUnrollSmem quads (independent Philox
// chains) in flight.
constexpr int kStepUnrollSmem = 4;
template <typename R, int NQ>
struct FineOccupancy {
  static constexpr int value = NQ == 0 ? 2
                                       : (sizeof(R) == 4 ? (NQ <= 2 ? 5 : (NQ <= 4 ? 4 : 3)) : (NQ <= 2 ? 3 : 2));
};

// One slice ("task") n processed by rank g of its group of G CTAs:
// prologue (load, match, sum), the n_f Euler-Maruyama steps with the group
// mean each step, and the restriction epilogue.  Returns false if a group
// wait gave up; the CTA must then leave the kernel.
//
// Two forms of the step loop:
//
// * mean-additive diffusion (MULT false: b = B0, and generally whenever the
//   mean enters the step only through the drift term kappa m + c0): the
//   step is x_{j+1} = y_j + d_j with y_j = em_partial_pair(x_j) independent of
//   the mean and d_j = h (kappa m_j + c0) common to all particles.  The
//   stored state is y_j with the shift pending; since
//   m_{j+1} = mean(y_j) + d_j, the sum over y_j published at the end of
//   step j is first needed at the end of step j + 1.  Every CTA publishes
//   its step sum and reads the group's sum of the previous step, which its
//   peers published a whole step earlier: the cross-CTA exchange never
//   stalls the step loop of a CTA that keeps pace with its group.
//
// * general (MULT true: b = B x + BE m + B0): the noise amplitude depends on
//   the mean per particle, so step j + 1 waits for the group sum of step j.
//
// Either way one CTA barrier per step: every warp forms the CTA sum from
// the per-warp partials and the group sum from the published slots itself,
// in the same order, so all warps hold the same values.
//
// * plane rotator (FAM == kFamRotator, Sec. 5 Eq. SDE_plane_rotator): the
//   drift K (S cos x - C sin x) - g sin x needs the ensemble means S, C of
//   sin X and cos X of the step's own state, so step j + 1 waits for the two
//   group sums of step j (record channel, FP64); after the update each
//   particle is shifted modulo 2 pi into [-pi, pi], and its sine and cosine
//   enter the next step's sums.
template <typename R, int NQ, bool MULT, int STEP_UNROLL, int FAM = kFamPoly>
__device__ __forceinline__ bool fine_task(const FineArgs& a, const int n, const int g, Group& grp,
                                          GroupShared& sh, QuadStore<R, NQ>& xs) {
  using SS = StepSum<R>;
  using ST = typename SS::T;
  constexpr bool kRot = FAM == kFamRotator;
  constexpr bool kLag = !MULT && !kRot;
  constexpr int kUnroll = NQ > 0 ? NQ : 2;             // prologue and epilogue
  constexpr int kStepUnroll = NQ > 0 ? NQ : STEP_UNROLL;
  const int G = a.G;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nq_max = NQ > 0 ? NQ : a.nq;
  const int qb = (int)(((long long)a.Q * g) / G);
  const int qe = (int)(((long long)a.Q * (g + 1)) / G);
  const int span = qe - qb - tid;
  const int nq = span <= 0 ? 0 : min(nq_max, (span + kTPB - 1) / kTPB);
  const int qlast = a.Q - 1;
  const int plast = (int)(a.P - 4LL * qlast);  // valid lanes of the last quad, 1..4
  const int loop_n = NQ > 0 ? NQ : nq;        // quads this thread visits
  const int nf = a.nf;
  // this thread's index of the ragged last quad (lanes past P), or -1
  const int tail_off = qlast - qb - tid;
  const int tail_i = (plast < 4 && tail_off >= 0 && tail_off % kTPB == 0 && tail_off / kTPB < nq)
                         ? tail_off / kTPB : -1;

  // Coefficients in the particle precision.  For float particles they are
  // rounded once per task by one thread and read from shared memory: left
  // to the compiler, the double-to-float conversions get re-derived from the
  // double kernel arguments inside the step loop, and every such conversion
  // issues on the FP64 pipe, which runs at 2 lanes per clock per SM here.
  __syncthreads();  // the previous task's readers of sh are done
  if (sizeof(R) == 4 && tid == 0) {
    sh.cf[0] = (float)a.h;
    sh.cf[1] = (float)a.nc3;
    sh.cf[2] = (float)a.c1;
    sh.cf[3] = (float)(a.B * a.sqrt_h);
    sh.cf[4] = (float)(a.B0 * a.sqrt_h);
    sh.cf[5] = (float)a.thr;
    sh.cf[6] = (float)(1.0 / (double)a.P);
    sh.cf[7] = (float)a.kappa;
    sh.cf[8] = (float)a.c0;
    sh.cf[9] = (float)a.BE;
    sh.cf[10] = (float)a.B0;
    sh.cf[11] = (float)a.sqrt_h;
    sh.cf[12] = (float)(a.h * a.nc3);
    sh.cf[13] = (float)(a.h * a.c1);
    sh.cf[14] = (float)a.thr2;
    sh.cf[15] = (float)a.thr3;
    sh.cr[0] = (float)a.K;
    sh.cr[1] = (float)a.gpin;
  }
  if (tid < kMaxRegions) {
    // this slice's matching record of region tid (identity past n_regions)
    int mode = kMatchIdentity;
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;
    if (a.aff != nullptr && tid < a.n_regions) {
      const double* af = a.aff + ((size_t)(a.aff_fixed ? 0 : n) * kMaxRegions + tid) * kAff;
      mode = (int)af[0];
      p0 = af[1]; p1 = af[2]; p2 = af[3];
    }
    sh.amode[tid] = mode;
    sh.affd[tid][0] = p0; sh.affd[tid][1] = p1; sh.affd[tid][2] = p2;
    sh.afff[tid][0] = (float)p0; sh.afff[tid][1] = (float)p1; sh.afff[tid][2] = (float)p2;
  }
  __syncthreads();
  const bool fl = sizeof(R) == 4;
  const R h = fl ? (R)sh.cf[0] : (R)a.h;
  const R nc3 = fl ? (R)sh.cf[1] : (R)a.nc3;
  const R c1 = fl ? (R)sh.cf[2] : (R)a.c1;
  const R bsq = fl ? (R)sh.cf[3] : (R)(a.B * a.sqrt_h);    // state-proportional part of b sqrt(h)
  const R b0sq = fl ? (R)sh.cf[4] : (R)(a.B0 * a.sqrt_h);  // additive noise amplitude
  const R thr = fl ? (R)sh.cf[5] : (R)a.thr;
  const float inv_p = sh.cf[6];                             // float path only
  const R kap = fl ? (R)sh.cf[7] : (R)a.kappa;
  const R c0r = fl ? (R)sh.cf[8] : (R)a.c0;
  const R ber = fl ? (R)sh.cf[9] : (R)a.BE;
  const R b0r = fl ? (R)sh.cf[10] : (R)a.B0;
  const R sqh = fl ? (R)sh.cf[11] : (R)a.sqrt_h;
  const R hn3 = fl ? (R)sh.cf[12] : (R)(a.h * a.nc3);
  const R hc1 = fl ? (R)sh.cf[13] : (R)(a.h * a.c1);
  const R thr2 = fl ? (R)sh.cf[14] : (R)a.thr2;
  const R thr3 = fl ? (R)sh.cf[15] : (R)a.thr3;
  const R Kr = fl ? (R)sh.cr[0] : (R)a.K;      // plane rotator only
  const R gr = fl ? (R)sh.cr[1] : (R)a.gpin;
  const int nreg = a.n_regions;
  auto region = [&](R x) { return region_of<R>(x, nreg, thr, thr2, thr3); };
  auto aff_param = [&](int r, int k) -> R { return fl ? (R)sh.afff[r][k] : (R)sh.affd[r][k]; };
  const unsigned E = grp.epoch;  // first epoch of this task

  {
  const R* src = (a.src == nullptr || n == 0) ? (const R*)a.src0
                                              : (const R*)a.src + (size_t)(n - 1) * a.pitch;
  // ---------------- prologue: load, match, sum --------------------------
  int flips = 0;
  R s_in = (R)0;
  R s_sin = (R)0, s_cos = (R)0;  // plane rotator: sums of sin x, cos x of the inputs
  // The matching records of this task's regions sit in registers (NR of
  // them, loops over regions unrolled); with at most two regions the region
  // of x is one comparison.
  auto prologue = [&](auto nr_c) {
    constexpr int NR = decltype(nr_c)::value;
    int md[NR];
    R pa[NR], pb[NR], pc[NR];
    bool match = false, redraw = false;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      md[r] = sh.amode[r];
      pa[r] = aff_param(r, 0);
      pb[r] = aff_param(r, 1);
      pc[r] = aff_param(r, 2);
      match = match || md[r] != kMatchIdentity;
      redraw = redraw || md[r] == kMatchRedraw;
    }
    auto reg_of = [&](R x) -> int { return NR == 2 ? ((nreg > 1 && !(x < thr)) ? 1 : 0) : region(x); };
#pragma unroll kUnroll
    for (int i = 0; i < loop_n; ++i) {
      R v[4] = {0, 0, 0, 0};
      const int q = qb + tid + i * kTPB;
      if (i < nq) {
        if (q != qlast || plast == 4) {
          Quad<R>::load(src + 4 * (size_t)q, v);
        } else {
          // the ragged last quad: guarded scalar loads so that a buffer
          // of exactly P values is never over-read
#pragma unroll
          for (int w = 0; w < 4; ++w) v[w] = w < plast ? src[4 * (size_t)q + w] : (R)0;
        }
        if (match) {
          int reg[4];
          R y[4];
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            reg[w] = reg_of(v[w]);
            int sm = md[0];
            R sa = pa[0], sb = pb[0], sc = pc[0];
#pragma unroll
            for (int r = 1; r < NR; ++r) {
              if (reg[w] == r) {
                sm = md[r];
                sa = pa[r];
                sb = pb[r];
                sc = pc[r];
              }
            }
            y[w] = sm == kMatchAffine ? apply_affine(v[w], sa, sb, sc) : v[w];
          }
          if (redraw) {
            // V u = 0 branch: tag-2 draws of region r's stream (j = r)
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              if (md[r] != kMatchRedraw) continue;
              if (reg[0] != r && reg[1] != r && reg[2] != r && reg[3] != r) continue;
              R z[4];
              normals4<R>(philox4x32_10(rng_counter((uint32_t)q, (uint32_t)r, (uint32_t)n, 2u, a.ptag), a.key0,
                                        a.key1), z);
#pragma unroll
              for (int w = 0; w < 4; ++w)
                if (reg[w] == r) y[w] = fmaR(pb[r], z[w], pa[r]);
            }
          }
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            if (nreg > 1 && reg_of(y[w]) != reg[w] && (4 * (long long)q + w < a.P)) flips += 1;
            v[w] = y[w];
          }
        }
        // zero the lanes past P so that sums see only real particles
        if (q == qlast) {
          if (plast < 4) v[3] = (R)0;
          if (plast < 3) v[2] = (R)0;
          if (plast < 2) v[1] = (R)0;
        }
        s_in = addR(s_in, addR(addR(v[0], v[1]), addR(v[2], v[3])));
        if constexpr (kRot) {
          // sin x and cos x are kept beside x (slots nq_max + i, 2 nq_max + i)
          const int valid = q == qlast ? plast : 4;
          R sv[4], cv[4];
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            sincosR(v[w], &sv[w], &cv[w]);
            if (w < valid) {
              s_sin = addR(s_sin, sv[w]);
              s_cos = addR(s_cos, cv[w]);
            }
          }
          xs.put(nq_max + i, sv);
          xs.put(2 * nq_max + i, cv);
        }
      }
      xs.put(i, v);
    }
  };
  if (nreg <= 2) {
    prologue(RegionsUpTo<2>{});
  } else {
    prologue(RegionsUpTo<kMaxRegions>{});
  }
  // The sum of the inputs is epoch E.  The shift form reads it at the end
  // of step 0 (or right here when there are no steps); the general form
  // needs m_0 before step 0.  Warp 0 does all cross-CTA work: after each
  // CTA barrier it publishes the CTA's sum of the step just finished, and
  // before the next barrier it reads the group sum that the other warps need
  // after it (through sh.gsum).
  double m_in = 0.0;
  R d = (R)0;                  // shift form: the pending shift d_{j-1}
  R base = (R)0, boff = (R)0;  // general form: kappa m_j + c0, (BE m_j + B0) sqrt(h)
  R mj = (R)0;                 // general form: m_j (recorded for the adjoint)
  // Plane rotator: the group sums of (sin x, cos x, x) of the inputs; warp 0
  // leaves the means of sin and cos in sh.rotd / sh.rotf for every thread.
  auto rot_exchange = [&](int nv, double v0, double v1, double v2) -> bool {
    double v[3] = {v0, v1, v2};
    if (nv == 3) warp_reduce_to_shared<3>(sh, v, 0u, 0u);
    else warp_reduce_to_shared<2>(sh, v, 0u, 0u);
    __syncthreads();
    const unsigned e = grp.epoch++;
    if (warp == 0) {
      const bool ok = nv == 3 ? group_finish<3>(sh, grp, e, 0u, 0u) : group_finish<2>(sh, grp, e, 0u, 0u);
      if (lane == 0) {
        if (!ok) sh.abort = 1;
        const double S = sh.tot[0] / (double)a.P, C = sh.tot[1] / (double)a.P;
        sh.rotd[0] = S;
        sh.rotd[1] = C;
        sh.rotf[0] = (float)S;
        sh.rotf[1] = (float)C;
      }
    }
    __syncthreads();
    return !sh.abort;
  };
  if constexpr (kRot) {
    if (!rot_exchange(3, (double)s_sin, (double)s_cos, (double)s_in)) return false;
    m_in = sh.tot[2] / (double)a.P;
  } else {
  step_sum_warp<R>(sh, 1, s_in);
  __syncthreads();
  if (warp == 0) {
    const ST cta = step_sum_cta<R>(sh, 1);
    if (lane == 0) SS::publish(grp, E, cta);
  }
  grp.epoch = E + 1u;
  }
  if (!kRot && (!kLag || nf == 0)) {
    if (warp == 0) {
      ST sum;
      const bool ok = SS::fetch(grp, E, sum);
      if (lane == 0) {
        SS::gsum(sh, 1) = sum;
        if (!ok) sh.abort = 1;
      }
    }
    __syncthreads();
    if (sh.abort) return false;
    const R m = (R)SS::mean(SS::gsum(sh, 1), inv_p, a.P);
    m_in = (double)m;
    mj = m;
    base = fmaR(kap, m, c0r);
    boff = mulR(fmaR(ber, m, b0r), sqh);
  }

  // ---------------- Euler-Maruyama steps --------------------------------
  if constexpr (kRot) {
    // Each step in two phases around the group sums of sin x_j and cos x_j:
    //   A: y = x - h g sin x + B0 sqrt(h) xi        (no ensemble sum needed)
    //   B: x' = wrap(y + h K (S cos x - C sin x)), then sin x', cos x' and
    //      their sums for the next step.
    // Warp 0 publishes a step's sums at the end of its phase B and collects
    // the group's after the next phase A, so the exchange travels while
    // phase A computes.  The sums of step 0 come from the prologue.
    const R hK = mulR(h, Kr);
    const R hg = mulR(h, gr);
    double cta_s = 0.0, cta_c = 0.0;  // warp 0: this CTA's sums of the pending epoch
    unsigned e_pub = 0;
    bool pending = false;
    for (int j = 0; j < nf; ++j) {
#pragma unroll kStepUnroll
      for (int i = 0; i < loop_n; ++i) {
        if (i < nq) {
          const int q = qb + tid + i * kTPB;
          R v[4], sv[4];
          xs.get(i, v);
          xs.get(nq_max + i, sv);
          const uint4 o = philox4x32_10(rng_counter((uint32_t)q, (uint32_t)j, (uint32_t)n, 0u, a.ptag), a.key0,
                                        a.key1);
          R z[4];
          normals4<R>(o, z);
#pragma unroll
          for (int w = 0; w < 4; ++w) v[w] = addR(subR(v[w], mulR(hg, sv[w])), mulR(b0sq, z[w]));
          xs.put(i, v);
        }
      }
      if (pending) {
        if (warp == 0) {
          double gs0 = 0.0, gs1 = 0.0;
          bool ok = true;
          if (grp.G > 1) {
            ok = group_wait(grp, e_pub);
            for (int c = lane; c < grp.G; c += 32) {
              const double* sl = group_slot(grp, c, e_pub);
              gs0 += __ldcg(sl);
              gs1 += __ldcg(sl + 1);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
              gs0 += __shfl_xor_sync(0xffffffffu, gs0, off);
              gs1 += __shfl_xor_sync(0xffffffffu, gs1, off);
            }
          } else {
            gs0 = cta_s;
            gs1 = cta_c;
          }
          if (lane == 0) {
            if (!ok) sh.abort = 1;
            const double S = gs0 / (double)a.P, C = gs1 / (double)a.P;
            sh.rotd[0] = S;
            sh.rotd[1] = C;
            sh.rotf[0] = (float)S;
            sh.rotf[1] = (float)C;
          }
        }
        __syncthreads();
        if (sh.abort) return false;
        pending = false;
      }
      const R sb = fl ? (R)sh.rotf[0] : (R)sh.rotd[0];
      const R cb = fl ? (R)sh.rotf[1] : (R)sh.rotd[1];
      const bool more = j + 1 < nf;  // the last step's sines, cosines and sums are not needed
      R ss = (R)0, cs = (R)0;
#pragma unroll kStepUnroll
      for (int i = 0; i < loop_n; ++i) {
        if (i < nq) {
          const int q = qb + tid + i * kTPB;
          R v[4], sv[4], cv[4];
          xs.get(i, v);
          xs.get(nq_max + i, sv);
          xs.get(2 * nq_max + i, cv);
          const int valid = q == qlast ? plast : 4;
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            v[w] = wrap_angle(addR(v[w], mulR(hK, subR(mulR(sb, cv[w]), mulR(cb, sv[w])))));
            if (more) {
              sincosR(v[w], &sv[w], &cv[w]);
              if (w < valid) {
                ss = addR(ss, sv[w]);
                cs = addR(cs, cv[w]);
              }
            }
          }
          xs.put(i, v);
          if (more) {
            xs.put(nq_max + i, sv);
            xs.put(2 * nq_max + i, cv);
          }
        }
      }
      if (more) {
        double v2[2] = {(double)ss, (double)cs};
        warp_reduce_to_shared<2>(sh, v2, 0u, 0u);
        __syncthreads();
        e_pub = grp.epoch++;
        if (warp == 0) {
          double w0 = lane < kWarps ? sh.red[lane][0] : 0.0;
          double w1 = lane < kWarps ? sh.red[lane][1] : 0.0;
#pragma unroll
          for (int off = kWarps / 2; off > 0; off >>= 1) {
            w0 += __shfl_xor_sync(0xffffffffu, w0, off);
            w1 += __shfl_xor_sync(0xffffffffu, w1, off);
          }
          cta_s = __shfl_sync(0xffffffffu, w0, 0);
          cta_c = __shfl_sync(0xffffffffu, w1, 0);
          if (grp.G > 1 && lane == 0) {
            const double pub[2] = {cta_s, cta_c};
            group_publish(grp, e_pub, pub, 2);
          }
        }
        pending = true;
      }
    }
  } else
  for (int j = 0; j < nf; ++j) {
    const long long gs = a.step_offset + j;
    const bool ckpt = a.rec_ckpt != nullptr && gs % a.ckpt_every == 0;
    R* ck_row = ckpt ? (R*)a.rec_ckpt + (size_t)(gs / a.ckpt_every) * a.pitch : nullptr;
    if constexpr (!kLag) {
      if (a.rec_uni != nullptr && g == 0 && tid == 0) {
        // the adjoint replays step j from exactly these values
        R* u = (R*)a.rec_uni + 3 * gs;
        u[0] = mj;
        u[1] = base;
        u[2] = boff;
      }
    }
    // the step over this thread's quads, with (CK) or without the
    // checkpoint row of the step's states
    auto step_quads = [&](auto ck_c) -> R {
      constexpr bool CK = decltype(ck_c)::value;
      R sq = (R)0;
#pragma unroll kStepUnroll
      for (int i = 0; i < loop_n; ++i) {
        if (i < nq) {
          const uint32_t q = (uint32_t)(qb + tid + i * kTPB);
          R v[4];
          xs.get(i, v);
          const uint4 o = philox4x32_10(rng_counter(q, (uint32_t)j, (uint32_t)n, 0u, a.ptag), a.key0, a.key1);
          if constexpr (kLag) {
            R nr[2], c[2], sn[2];
            normals4_polar<R>(o, nr, c, sn);
#pragma unroll
            for (int w = 0; w < 4; ++w) v[w] = addR(v[w], d);  // x_j = y_{j-1} + d_{j-1}
            if constexpr (CK) Quad<R>::store(ck_row + 4 * (size_t)q, v);
            em_partial_pair(v[0], v[1], nr[0], c[0], sn[0], hn3, hc1, b0sq);
            em_partial_pair(v[2], v[3], nr[1], c[1], sn[1], hn3, hc1, b0sq);
          } else {
            if constexpr (CK) Quad<R>::store(ck_row + 4 * (size_t)q, v);
            R z[4];
            normals4<R>(o, z);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              const R xv = v[w];
              const R drift = fmaR(fmaR(nc3, mulR(xv, xv), c1), xv, base);
              const R amp = fmaR(bsq, xv, boff);
              v[w] = fmaR(amp, z[w], fmaR(h, drift, xv));
            }
          }
          // lanes past P evolve like particles; their values leave the sum below
          sq = addR(sq, addR(addR(v[0], v[1]), addR(v[2], v[3])));
          xs.put(i, v);
        }
      }
      return sq;
    };
    R s = ckpt ? step_quads(Switch<true>{}) : step_quads(Switch<false>{});
    if (tail_i >= 0) {
      // the lanes past P of the ragged last quad (this thread's, if any)
      // leave the sum: they evolve like particles but are none
      R pad = (R)0;
      if constexpr (NQ > 0) {
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
          if (i == tail_i) {
            R v[4];
            xs.get(i, v);
#pragma unroll
            for (int w = 3; w >= 1; --w)
              if (w >= plast) pad = addR(pad, v[w]);
          }
        }
      } else {
        R v[4];
        xs.get(tail_i, v);
#pragma unroll
        for (int w = 3; w >= 1; --w)
          if (w >= plast) pad = addR(pad, v[w]);
      }
      s = addR(s, -pad);
    }
    step_sum_warp<R>(sh, j & 1, s);
    if constexpr (kLag) {
      // m_j = mean(y_{j-1}) + d_{j-1},  d_j = h (kappa m_j + c0), from the
      // group sum of epoch E + j, which the peers published when their
      // step j - 1 ended
      if (warp == 0) {
        ST sum;
        const bool ok = SS::fetch(grp, E + (unsigned)j, sum);
        if (lane == 0) {
          SS::gsum(sh, j & 1) = sum;
          if (!ok) sh.abort = 1;
        }
      }
      __syncthreads();
      if (sh.abort) return false;
      const R m = addR((R)SS::mean(SS::gsum(sh, j & 1), inv_p, a.P), d);
      if (j == 0) m_in = (double)m;
      d = mulR(h, fmaR(kap, m, c0r));
      if (a.rec_uni != nullptr && g == 0 && tid == 0) {
        // the adjoint replays step j from exactly these values
        R* u = (R*)a.rec_uni + 3 * gs;
        u[0] = m;
        u[1] = d;
        u[2] = b0sq;
      }
      // this step's sum becomes epoch E + 1 + j (unless nothing reads it)
      if (j + 1 < nf) {
        if (warp == 0) {
          const ST cta = step_sum_cta<R>(sh, j & 1);
          if (lane == 0) SS::publish(grp, E + 1u + (unsigned)j, cta);
        }
        grp.epoch = E + 2u + (unsigned)j;
      }
    } else {
      __syncthreads();
      const unsigned e = E + 1u + (unsigned)j;
      if (warp == 0) {
        ST sum = step_sum_cta<R>(sh, j & 1);
        if (lane == 0) SS::publish(grp, e, sum);
        const bool ok = SS::fetch(grp, e, sum);
        if (lane == 0) {
          SS::gsum(sh, j & 1) = sum;
          if (!ok) sh.abort = 1;
        }
      }
      grp.epoch = e + 1u;
      __syncthreads();
      if (sh.abort) return false;
      const R m = (R)SS::mean(SS::gsum(sh, j & 1), inv_p, a.P);
      mj = m;
      base = fmaR(kap, m, c0r);
      boff = mulR(fmaR(ber, m, b0r), sqh);
    }
  }
  __syncthreads();

  // ---------------- epilogue: store and restrict -----------------------
  // Group reductions, values in this order (the first entries are those of
  // two regions, so tasks of at most two regions reduce 5 and 7 values):
  //   pass 1: count_0, sum_0, count_1, sum_1, flips, then (count_r, sum_r), r >= 2;
  //   pass 2: centred_0, centred_1, centred_global, min_0, max_0, min_1, max_1,
  //           then centred_r (r >= 2), then (min_r, max_r) (r >= 2).
  auto epilogue = [&](auto nr_c) -> bool {
    constexpr int NR = decltype(nr_c)::value;
    constexpr int NV1 = 2 * NR + 1;
    constexpr int NV2 = 3 * NR + 1;
    auto reg_of = [&](R x) -> int { return NR == 2 ? ((nreg > 1 && !(x < thr)) ? 1 : 0) : region(x); };
    auto i_cnt = [](int r) { return r < 2 ? 2 * r : 5 + 2 * (r - 2); };
    auto i_ss = [](int r) { return r < 2 ? r : NR + 3 + (r - 2); };
    auto i_lo = [](int r) { return r < 2 ? 3 + 2 * r : 2 * NR + 1 + 2 * (r - 2); };
    // pass 1 (with the store): apply the pending shift, counts and sums per region
    {
      R* dst = a.dst != nullptr ? (R*)a.dst + (size_t)(a.dst_fixed ? 0 : n) * a.pitch : nullptr;
      int cnt[NR];
      Acc<R> sum[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) cnt[r] = 0;
      const bool shift = kLag && nf > 0;
#pragma unroll kUnroll
      for (int i = 0; i < loop_n; ++i) {
        if (i < nq) {
          const int q = qb + tid + i * kTPB;
          R x4[4];
          xs.get(i, x4);
          if (shift) {
#pragma unroll
            for (int w = 0; w < 4; ++w) x4[w] = addR(x4[w], d);
            xs.put(i, x4);
          }
          if (dst != nullptr) {
            if (q != qlast || plast == 4) {
              Quad<R>::store(dst + 4 * (size_t)q, x4);
            } else {
#pragma unroll
              for (int w = 0; w < 4; ++w)
                if (w < plast) dst[4 * (size_t)q + w] = x4[w];
            }
          }
          const int valid = q == qlast ? plast : 4;
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            if (w < valid) {
              const int r = reg_of(x4[w]);
#pragma unroll
              for (int rr = 0; rr < NR; ++rr) {
                if (rr == r) {
                  cnt[rr] += 1;
                  sum[rr].add(x4[w]);
                }
              }
            }
          }
        }
      }
      double v[NV1];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        v[i_cnt(r)] = (double)cnt[r];
        v[i_cnt(r) + 1] = sum[r].get();
      }
      v[4] = (double)flips;
      warp_reduce_to_shared<NV1>(sh, v, 0u, 0u);
      __syncthreads();
      const unsigned e = grp.epoch++;
      if (warp == 0 && !group_finish<NV1>(sh, grp, e, 0u, 0u) && lane == 0) sh.abort = 1;
      __syncthreads();
      if (sh.abort) return false;
    }
    double cnt[NR], mean[NR];
    double gsum = sh.tot[1] + sh.tot[3];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      cnt[r] = sh.tot[i_cnt(r)];
      mean[r] = cnt[r] > 0 ? sh.tot[i_cnt(r) + 1] / cnt[r] : 0.0;
      if (r >= 2) gsum = gsum + sh.tot[i_cnt(r) + 1];
    }
    const double gmean = gsum / (double)a.P;
    const double flips_tot = sh.tot[4];
    __syncthreads();
    // pass 2: centred sums and extremes
    {
      const Centre<R> cg(gmean);
      Centre<R> cc[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) cc[r] = Centre<R>(mean[r]);
      Acc<R> ss[NR], ssg;
      R lo[NR], hi[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        lo[r] = (R)INFINITY;
        hi[r] = (R)-INFINITY;
      }
#pragma unroll kUnroll
      for (int i = 0; i < loop_n; ++i) {
        if (i < nq) {
          const int q = qb + tid + i * kTPB;
          const int valid = q == qlast ? plast : 4;
          R x4[4];
          xs.get(i, x4);
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            if (w < valid) {
              const R xv = x4[w];
              const R dg = cg.diff(xv);
              ssg.add(dg * dg);
              const int r = reg_of(xv);
#pragma unroll
              for (int rr = 0; rr < NR; ++rr) {
                if (rr == r) {
                  const R dd = cc[rr].diff(xv);
                  ss[rr].add(dd * dd);
                  lo[rr] = lo[rr] < xv ? lo[rr] : xv;
                  hi[rr] = hi[rr] > xv ? hi[rr] : xv;
                }
              }
            }
          }
        }
      }
      double v[NV2];
      unsigned mn = 0u, mx = 0u;
      v[2] = ssg.get();
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        v[i_ss(r)] = ss[r].get();
        v[i_lo(r)] = (double)lo[r];
        v[i_lo(r) + 1] = (double)hi[r];
        mn |= 1u << i_lo(r);
        mx |= 1u << (i_lo(r) + 1);
      }
      warp_reduce_to_shared<NV2>(sh, v, mn, mx);
      __syncthreads();
      const unsigned e = grp.epoch++;
      if (warp == 0 && !group_finish<NV2>(sh, grp, e, mn, mx) && lane == 0) sh.abort = 1;
      __syncthreads();
      if (sh.abort) return false;
    }
    if (g == 0 && tid == 0 && a.stats != nullptr) {
      double* st = a.stats + (size_t)(a.stats_fixed ? 0 : n) * kStat;
      for (int k = 0; k < kStat; ++k) st[k] = 0.0;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        double* sr = st + stat_region(r);
        sr[0] = cnt[r];
        sr[1] = mean[r];
        sr[2] = cnt[r] > 0 ? sh.tot[i_ss(r)] / cnt[r] : 0.0;
        sr[3] = sh.tot[i_lo(r)];
        sr[4] = sh.tot[i_lo(r) + 1];
      }
      st[kStatM] = gmean;
      st[kStatV] = sh.tot[2] / (double)a.P;
      st[kStatFlips] = flips_tot;
      st[kStatInMean] = m_in;
      if (!(fabs(gmean) < INFINITY) || !(st[kStatV] < INFINITY)) atomicOr(a.status, kStatusNumeric);
      if (flips_tot > 0.0) atomicOr(a.status, kStatusRegionFlip);
    }
    return true;
  };
  if (nreg <= 2 ? !epilogue(RegionsUpTo<2>{}) : !epilogue(RegionsUpTo<kMaxRegions>{})) return false;
  }
  return true;
}

template <typename R, int NQ, bool MULT, int FAM = kFamPoly>
__global__ void __launch_bounds__(kTPB, (FineOccupancy<R, NQ>::value)) k_fine(const FineArgs a) {
  __shared__ GroupShared sh;
  const int G = a.G;
  const int n_slots = gridDim.x / G;
  const int slot = blockIdx.x / G;
  const int g = blockIdx.x - slot * G;
  if (slot >= n_slots) return;
  Group grp;
  grp.part = a.partials + (size_t)slot * G * kSeatDoubles;
  grp.flags = a.flags + (size_t)slot * G;
  grp.tags = a.tags + (size_t)slot * kSlots * G;
  grp.status = a.status;
  grp.limit_ns = a.wait_limit_ns;
  grp.G = G;
  grp.g = g;
  grp.epoch = 0;
  grp.tight_polls = a.tight_polls;
  if (threadIdx.x == 0) sh.abort = 0;
  QuadStore<R, NQ> xs;
  xs.bind();
  for (int task = slot; task < a.n_tasks; task += n_slots) {
    if (!fine_task<R, NQ, MULT, kStepUnrollSmem, FAM>(a, a.slice_begin + task, g, grp, sh, xs)) return;
  }
}

}  // namespace mmp
