// mmp_internal.cuh -- device helpers shared by the kernels of libmmp.
//
// Random numbers: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the
// counter-based generator that lets every Parareal iteration redraw the
// same noise (Property 3.3 needs identical draws in every iteration).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mmp.h"

namespace mmp {

constexpr int kTPB = 256;          // threads per block of the fine kernel
constexpr int kWarps = kTPB / 32;
constexpr int kNV = 16;            // values per group reduction slot
constexpr int kSlots = 4;          // publication slots per CTA (a ring indexed by epoch)
constexpr int kSeatDoubles = kSlots * kNV;  // reduction scratch per CTA of a group
constexpr int kStat = MMP_STAT_STRIDE;
constexpr int kMom = MMP_MOMENT_STRIDE;
constexpr int kAff = 4;            // doubles per (slice, region) matching record
constexpr int kMaxRegions = MMP_MAX_REGIONS;
// offsets of region r's values in a moment row and a restriction record
__host__ __device__ constexpr int mom_region(int r) { return MMP_MOMENT_REGION(r); }
__host__ __device__ constexpr int stat_region(int r) { return MMP_STAT_REGION(r); }
constexpr int kMomM = 6, kMomV = 7;        // global mean, variance in a moment row
constexpr int kStatM = 10, kStatV = 11;    // global mean, variance in a restriction record
constexpr int kStatFlips = 12, kStatInMean = 13;
constexpr int kMaxNQ = 8;          // largest quads-per-thread template
constexpr int kFamPoly = MMP_FAMILY_POLY;
constexpr int kFamRotator = MMP_FAMILY_ROTATOR;

// Polls of a bounded group wait before it backs off with nanosleep, for
// launches with at most one CTA per SM: a word about to land is then picked
// up at L2 latency rather than at sleep granularity, and no co-resident CTA
// loses issue slots to the spinning warp.  With co-resident CTAs a wait
// sleeps from the first miss.
constexpr int kTightPolls = 256;

// Device status bits (or-ed into the status word).
constexpr unsigned kStatusTimeout = 1u;
constexpr unsigned kStatusNumeric = 2u;
constexpr unsigned kStatusRegionFlip = 4u;

// Matching modes of a (slice, region) record {mode, a, b, c}:
//   identity: x unchanged
//   affine:   x + (a + b (x - c)), a = mu - E u, b = sqrt(sigma / V u) - 1, c = E u
//   redraw:   a + b xi (tag-2 draw), a = mu, b = sqrt(sigma)       (V u = 0)
constexpr int kMatchIdentity = 0;
constexpr int kMatchAffine = 1;
constexpr int kMatchRedraw = 2;

// ---------------------------------------------------------------------------
// Philox-4x32-10.  One round maps (c0, c1, c2, c3) with key (k0, k1) to
//   (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0));
// the key advances by the Weyl increments (W0, W1) between rounds.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Both halves of the 64-bit product a * b from one wide multiply.
__device__ __forceinline__ void mul_hilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
  uint64_t p;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
  lo = (uint32_t)p;
  hi = (uint32_t)(p >> 32);
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t rk0 = k0 + (uint32_t)r * kPhiloxW0;
    const uint32_t rk1 = k1 + (uint32_t)r * kPhiloxW1;
    uint32_t hi0, lo0, hi1, lo1;
    mul_hilo(kPhiloxM0, c.x, hi0, lo0);
    mul_hilo(kPhiloxM1, c.z, hi1, lo1);
    c = make_uint4(hi1 ^ c.y ^ rk0, lo1, hi0 ^ c.w ^ rk1, lo0);
  }
  return c;
}

// Uniform u = ((o >> 9) + 1/2) 2^-23 in (0, 1).
// float: the bit pattern 1.m with m = o >> 9 is 1 + (o >> 9) 2^-23; subtracting
// 1 - 2^-24 is exact (Sterbenz) and lands on the same grid point.
__device__ __forceinline__ float uniform_f(uint32_t o) {
  return __uint_as_float(0x3F800000u | (o >> 9)) - 0x1.fffffep-1f;
}
__device__ __forceinline__ double uniform_d(uint32_t o) {
  return __fma_rn((double)(o >> 9), 0x1p-23, 0x1p-24);
}

// Fused multiply-add in the particle precision (never promoted to FP64).
__device__ __forceinline__ float fmaR(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaR(double a, double b, double c) { return __fma_rn(a, b, c); }

// Box-Muller: z = sqrt(-2 ln ua) (cos 2 pi ub, sin 2 pi ub).
// FP32 form on the special-function unit: ln ua from the hardware log2,
// the hardware square root, and sin/cos of theta = 2 pi (ub - 1/2), which lies
// in [-pi, pi) where the hardware sin/cos are accurate; then
// cos 2 pi ub = -cos theta and sin 2 pi ub = -sin theta.  The draws differ
// from the FP64 definition by a few 1e-6 absolute (bounded in the tests).
// ub enters as fb = 1 + (o >> 9) 2^-23 in [1, 2): ub - 1/2 = (fb - 3/2) + 2^-24,
// where fb - 3/2 is exact, so theta takes one add and one fused multiply-add.
// Polar form: the pair is (nr c, nr s) with nr = -sqrt(t), c = cos theta,
// s = sin theta, so a caller that scales both normals by one amplitude can
// scale nr once.
__device__ __forceinline__ void polar_f(float ua, float fb, float& nr, float& c, float& s) {
  const float t = -1.38629436f * __log2f(ua);  // -2 ln 2 log2(ua) > 0 for ua < 1
  float r;  // sqrt t on the special-function unit (one instruction)
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
  __sincosf(__fmaf_rn(__fsub_rn(fb, 1.5f), 6.28318531f, 3.74507028e-7f), &s, &c);  // 2 pi 2^-24
  nr = -r;
}
__device__ __forceinline__ void box_muller_f(float ua, float fb, float& z0, float& z1) {
  float nr, c, s;
  polar_f(ua, fb, nr, c, s);
  z0 = __fmul_rn(nr, c);
  z1 = __fmul_rn(nr, s);
}
__device__ __forceinline__ float unit_f(uint32_t o) { return __uint_as_float(0x3F800000u | (o >> 9)); }
__device__ __forceinline__ void polar_d(double ua, double ub, double& nr, double& c, double& s) {
  nr = sqrt(-2.0 * log(ua));
  sincospi(2.0 * ub, &s, &c);
}
__device__ __forceinline__ void box_muller(double ua, double ub, double& z0, double& z1) {
  double nr, c, s;
  polar_d(ua, ub, nr, c, s);
  z0 = nr * c;
  z1 = nr * s;
}

template <typename R>
__device__ __forceinline__ void normals4(uint4 o, R z[4]);
template <>
__device__ __forceinline__ void normals4<float>(uint4 o, float z[4]) {
  box_muller_f(uniform_f(o.x), unit_f(o.y), z[0], z[1]);
  box_muller_f(uniform_f(o.z), unit_f(o.w), z[2], z[3]);
}
template <>
__device__ __forceinline__ void normals4<double>(uint4 o, double z[4]) {
  box_muller(uniform_d(o.x), uniform_d(o.y), z[0], z[1]);
  box_muller(uniform_d(o.z), uniform_d(o.w), z[2], z[3]);
}

// The same four normals in polar form: normal 2k + i is nr[k] (c[k] | s[k]).
template <typename R>
__device__ __forceinline__ void normals4_polar(uint4 o, R nr[2], R c[2], R s[2]);
template <>
__device__ __forceinline__ void normals4_polar<float>(uint4 o, float nr[2], float c[2], float s[2]) {
  polar_f(uniform_f(o.x), unit_f(o.y), nr[0], c[0], s[0]);
  polar_f(uniform_f(o.z), unit_f(o.w), nr[1], c[1], s[1]);
}
template <>
__device__ __forceinline__ void normals4_polar<double>(uint4 o, double nr[2], double c[2], double s[2]) {
  polar_d(uniform_d(o.x), uniform_d(o.y), nr[0], c[0], s[0]);
  polar_d(uniform_d(o.z), uniform_d(o.w), nr[1], c[1], s[1]);
}

// Counter of the draw for particle quad q under (tag, step j, slice n).
__device__ __forceinline__ uint4 rng_counter(uint32_t q, uint32_t j, uint32_t n, uint32_t tag,
                                             uint32_t problem_tag) {
  return make_uint4(q, j, n | (tag << 24), problem_tag);
}

// ---------------------------------------------------------------------------
// Matching T (Eq. multimodal_M), affine branch written as
//   x + (delta + sm1 (x - m)),  delta = mu - E u,  sm1 = sqrt(sigma / V u) - 1,
// so that delta = sm1 = 0 (T(S u, u), Lemma 3.1) returns x bit for bit.
// The same function decides acceptance in the driver (Def. 3.2's
// fractions-unchanged test), so the test and the move agree to the bit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float apply_affine(float x, float delta, float sm1, float m) {
  return __fadd_rn(x, __fmaf_rn(sm1, __fsub_rn(x, m), delta));
}
__device__ __forceinline__ double apply_affine(double x, double delta, double sm1, double m) {
  return __dadd_rn(x, __fma_rn(sm1, __dsub_rn(x, m), delta));
}

// ---------------------------------------------------------------------------
// The plane rotator's shift of x modulo 2 pi into [-pi, pi]:
// x - 2 pi floor((x + pi) / (2 pi)), each operation rounded once (FP64: the
// division, as written; FP32: a product with 1 / (2 pi) rounded to float).
// ---------------------------------------------------------------------------
constexpr double kPi = 3.141592653589793238462643383280;
constexpr double kTwoPi = 6.283185307179586476925286766559;
__device__ __forceinline__ double wrap_angle(double x) {
  return __dsub_rn(x, __dmul_rn(kTwoPi, floor(__ddiv_rn(__dadd_rn(x, kPi), kTwoPi))));
}
__device__ __forceinline__ float wrap_angle(float x) {
  return __fsub_rn(x, __fmul_rn((float)kTwoPi, floorf(__fmul_rn(__fadd_rn(x, (float)kPi), (float)(1.0 / kTwoPi)))));
}
__device__ __forceinline__ void sincosR(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincosR(double x, double* s, double* c) { sincos(x, s, c); }

// ---------------------------------------------------------------------------
// Memory-model helpers for the cross-CTA group barrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_gpu_b64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_gpu_b64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Two-sum of floats (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

}  // namespace mmp
