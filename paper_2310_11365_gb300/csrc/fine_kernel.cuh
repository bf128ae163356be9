// fine_kernel.cuh -- the fused fine-propagator kernel, templated on the
// particle precision R (float or double), the quads of particles held per
// thread NQ, and whether the diffusion depends on the state (MULT).
//
// One slice of the Parareal sweep is one "task".  A task's P particles are
// split over a group of G co-resident CTAs (the launch is cooperative, so
// all CTAs are resident and a group barrier cannot deadlock).  Each thread
// holds up to NQ quads of 4 particles in registers for all n_f steps:
//
//   prologue  load u (coalesced 16-byte vectors), apply the matching T of
//             its region (Eq. multimodal_M), reduce the mean m_0
//   steps     x += h a(x, m_j) + b(x, m_j) sqrt(h) xi   (Eq. Euler_Maruyama)
//             with xi from Philox(p/4, j, n, problem) and the mean
//             m_{j+1} reduced over the whole group (warp shuffles, a shared
//             memory stage, then a cross-CTA stage through L2 guarded by a
//             bounded spin on an arrival counter)
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
struct GroupShared {
  double red[kWarps][kNV];  // per-warp partials
  float2 redf[kWarps];      // per-warp double-float partials of the per-step sum
  double tot[kNV];          // group totals, broadcast
  double uni[4];            // per-step uniforms derived from the mean
  float unif[4];            // the same, rounded once for float particles
  float cf[12];             // float copies of the task's coefficients (see fine_task)
  int abort;
};

template <typename R>
__device__ __forceinline__ R uniform_of(const GroupShared& sh, int k);
template <>
__device__ __forceinline__ float uniform_of<float>(const GroupShared& sh, int k) { return sh.unif[k]; }
template <>
__device__ __forceinline__ double uniform_of<double>(const GroupShared& sh, int k) { return sh.uni[k]; }

// Group-reduction context of one CTA.
struct Group {
  double* part;         // [2][G][kNV] doubles, then [2][G] float2, for this slot
  unsigned* counter;    // arrivals of this slot
  unsigned* status;
  unsigned long long limit_ns;
  int G, g;
  unsigned epoch;
};

// Warp 0 finishes a group reduction of nv values whose per-warp partials
// sit in sh.red.  min_mask / max_mask select values combined by min / max
// (all others are summed).  Returns false if the cross-CTA wait gave up.
__device__ __forceinline__ bool group_wait(Group& grp);

template <int NV>
__device__ __forceinline__ bool group_finish(GroupShared& sh, Group& grp, unsigned min_mask,
                                             unsigned max_mask) {
  constexpr int nv = NV;
  const int lane = threadIdx.x & 31;
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double ident = (min_mask >> k & 1) ? INFINITY : ((max_mask >> k & 1) ? -INFINITY : 0.0);
    v[k] = (k < nv && lane < kWarps) ? sh.red[lane][k] : ident;
  }
  // butterfly over the kWarps lanes that hold values
#pragma unroll
  for (int off = kWarps / 2; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      if (k < nv) {
        const double o = __shfl_xor_sync(0xffffffffu, v[k], off);
        v[k] = (min_mask >> k & 1) ? fmin(v[k], o) : ((max_mask >> k & 1) ? fmax(v[k], o) : v[k] + o);
      }
    }
  }
  if (grp.G > 1) {
    const unsigned parity = grp.epoch & 1u;
    grp.epoch += 1;
    double* mine = grp.part + ((size_t)parity * grp.G + grp.g) * kNV;
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k)
        if (k < nv) mine[k] = v[k];
      red_release_gpu_add(grp.counter, 1u);
    }
    if (!group_wait(grp)) return false;
    const double* all = grp.part + (size_t)parity * grp.G * kNV;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double ident = (min_mask >> k & 1) ? INFINITY : ((max_mask >> k & 1) ? -INFINITY : 0.0);
      v[k] = ident;
    }
    for (int c = lane; c < grp.G; c += 32) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        if (k < nv) {
          const double o = __ldcg(all + (size_t)c * kNV + k);
          v[k] = (min_mask >> k & 1) ? fmin(v[k], o) : ((max_mask >> k & 1) ? fmax(v[k], o) : v[k] + o);
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        if (k < nv) {
          const double o = __shfl_xor_sync(0xffffffffu, v[k], off);
          v[k] = (min_mask >> k & 1) ? fmin(v[k], o) : ((max_mask >> k & 1) ? fmax(v[k], o) : v[k] + o);
        }
      }
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
      if (k < nv) sh.tot[k] = v[k];
  }
  return true;
}

// Double-float addition (hi, lo) + (b_hi, b_lo) with error-free two-sums;
// exact to about 2^-48 relative and free of FP64 instructions, which on
// this chip issue at a small fraction of the FP32 rate.
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
  __device__ __forceinline__ explicit Centre(double m) : hi((float)m), lo((float)(m - (double)(float)m)) {}
  __device__ __forceinline__ float diff(float x) const { return __fsub_rn(__fsub_rn(x, hi), lo); }
};
template <>
struct Centre<double> {
  double m;
  __device__ __forceinline__ explicit Centre(double mm) : m(mm) {}
  __device__ __forceinline__ double diff(double x) const { return x - m; }
};

// Per-warp stage of the per-step sum: float input is carried as a
// double-float pair, double input as a double.
__device__ __forceinline__ void warp_sum_to_shared(GroupShared& sh, float s) {
  float2 v = make_float2(s, 0.0f);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = dd_add(v, shfl_xor_dd(v, off));
  if ((threadIdx.x & 31) == 0) sh.redf[threadIdx.x >> 5] = v;
}
__device__ __forceinline__ void warp_sum_to_shared(GroupShared& sh, double s) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5][0] = s;
}

// Bounded wait of warp 0 for all G arrivals of the current epoch.
__device__ __forceinline__ bool group_wait(Group& grp) {
  const unsigned target = grp.epoch * (unsigned)grp.G;
  bool ok = true;
  unsigned long long t0 = 0;
  int spins = 0;
  while (ld_acquire_gpu(grp.counter) < target) {
    if (++spins >= 32) {
      spins = 0;
      const unsigned long long now = globaltimer_ns();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > grp.limit_ns) {
        ok = false;
      }
      if (*(volatile unsigned*)grp.status & kStatusTimeout) ok = false;
      if (!ok) break;
    }
  }
  ok = __all_sync(0xffffffffu, ok);
  if (!ok && (threadIdx.x & 31) == 0) atomicOr(grp.status, kStatusTimeout);
  return ok;
}

// Warp 0 finishes the per-step sum of float particles entirely in FP32
// double-float arithmetic (warps in index order, then CTAs in index order)
// and publishes the per-step uniforms as floats.  Returns false on timeout.
__device__ __forceinline__ bool step_sum_finish_f(GroupShared& sh, Group& grp, float inv_p, float kappa,
                                                  float c0, float be, float b0, float sqrt_h) {
  const int lane = threadIdx.x & 31;
  float2 v = lane < kWarps ? sh.redf[lane] : make_float2(0.0f, 0.0f);
#pragma unroll
  for (int off = kWarps / 2; off > 0; off >>= 1) v = dd_add(v, shfl_xor_dd(v, off));
  if (grp.G > 1) {
    const unsigned parity = grp.epoch & 1u;
    grp.epoch += 1;
    // dense per-step partials after the [2][G][kNV] double area
    float2* part = reinterpret_cast<float2*>(grp.part + (size_t)2 * grp.G * kNV) + (size_t)parity * grp.G;
    if (lane == 0) {
      part[grp.g] = v;
      red_release_gpu_add(grp.counter, 1u);
    }
    if (!group_wait(grp)) return false;
    v = make_float2(0.0f, 0.0f);
    for (int c = lane; c < grp.G; c += 32) {
      const float2 o = __ldcg(part + c);
      v = dd_add(v, o);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = dd_add(v, shfl_xor_dd(v, off));
  }
  if (lane == 0) {
    const float m = __fmaf_rn(v.x, inv_p, v.y * inv_p);
    sh.unif[0] = m;
    sh.unif[1] = __fmaf_rn(kappa, m, c0);
    sh.unif[2] = __fmaf_rn(be, m, b0) * sqrt_h;
  }
  return true;
}

// General per-warp stage of nv double values.
template <int NV>
__device__ __forceinline__ void warp_reduce_to_shared(GroupShared& sh, double v[NV], unsigned min_mask,
                                                      unsigned max_mask) {
  constexpr int nv = NV;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      if (k < nv) {
        const double o = __shfl_xor_sync(0xffffffffu, v[k], off);
        v[k] = (min_mask >> k & 1) ? fmin(v[k], o) : ((max_mask >> k & 1) ? fmax(v[k], o) : v[k] + o);
      }
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
      if (k < nv) sh.red[threadIdx.x >> 5][k] = v[k];
  }
}

// After a reduction of the running sum: publish the per-step uniforms
// (mean, kappa m + c0, diffusion offset) so that no thread does FP64 work
// in the step loop.
__device__ __forceinline__ void publish_uniforms(GroupShared& sh, const FineArgs& a) {
  const double m = sh.tot[0] / (double)a.P;
  sh.uni[0] = m;
  sh.uni[1] = __fma_rn(a.kappa, m, a.c0);
  sh.uni[2] = __dmul_rn(__fma_rn(a.BE, m, a.B0), a.sqrt_h);
  sh.unif[0] = (float)sh.uni[0];
  sh.unif[1] = (float)sh.uni[1];
  sh.unif[2] = (float)sh.uni[2];
}

// Where a thread keeps its quads of particles between steps.
// NQ > 0: in registers, NQ quads (loops over quads fully unrolled).
// NQ == 0: in dynamic shared memory, a.nq quads at stride kTPB quads, so a
// warp touches 512 contiguous bytes per quad (conflict-free 16-byte
// accesses) and registers stay few, which lets more CTAs share an SM.
extern __shared__ __align__(16) unsigned char mmp_fine_smem[];

template <typename R, int NQ>
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
template <typename R>
struct QuadStore<R, 0> {
  R* base;
  __device__ __forceinline__ void bind() { base = reinterpret_cast<R*>(mmp_fine_smem) + 4 * threadIdx.x; }
  __device__ __forceinline__ void get(int i, R v[4]) const { Quad<R>::load(base + 4 * (size_t)i * kTPB, v); }
  __device__ __forceinline__ void put(int i, const R v[4]) { Quad<R>::store(base + 4 * (size_t)i * kTPB, v); }
};

// Resident CTAs per SM the register budget is sized for.  Register layout:
// the quads a thread holds dominate its registers, so fewer CTAs fit as NQ
// grows.  Shared-memory layout (NQ == 0): registers hold one quad in flight.
template <typename R, int NQ>
struct FineOccupancy {
  static constexpr int value = NQ == 0 ? (sizeof(R) == 4 ? 5 : 4)
                                       : (sizeof(R) == 4 ? (NQ <= 2 ? 5 : (NQ <= 4 ? 4 : 3)) : (NQ <= 2 ? 3 : 2));
};

// One slice ("task") n processed by rank g of its group of G CTAs:
// prologue (load, match, first mean), the n_f Euler-Maruyama steps with
// the group mean each step, and the restriction epilogue.  Returns false if
// a group wait gave up; the CTA must then leave the kernel.
template <typename R, int NQ, bool MULT>
__device__ __forceinline__ bool fine_task(const FineArgs& a, const int n, const int g, Group& grp,
                                          GroupShared& sh, QuadStore<R, NQ>& xs) {
  constexpr int kUnroll = NQ > 0 ? NQ : 2;
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

  // Coefficients in the particle precision.  For float particles they are
  // rounded once per task by one thread and read from shared memory: left
  // to the compiler, the double-to-float conversions get re-derived from the
  // double kernel arguments inside the step loop, and every such conversion
  // issues on the FP64 pipe, which runs at 2 lanes per clock per SM here.
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
  }
  __syncthreads();
  const bool fl = sizeof(R) == 4;
  const R h = fl ? (R)sh.cf[0] : (R)a.h;
  const R nc3 = fl ? (R)sh.cf[1] : (R)a.nc3;
  const R c1 = fl ? (R)sh.cf[2] : (R)a.c1;
  const R bsq = fl ? (R)sh.cf[3] : (R)(a.B * a.sqrt_h);    // state-proportional part of b sqrt(h)
  const R b0sq = fl ? (R)sh.cf[4] : (R)(a.B0 * a.sqrt_h);  // additive noise amplitude
  const R thr = fl ? (R)sh.cf[5] : (R)a.thr;
  const bool two = a.n_regions > 1;
  // per-step uniforms of the float path are formed in FP32 by warp 0
  const float inv_p = sh.cf[6];
  const float kappa_f = sh.cf[7], c0_f = sh.cf[8], be_f = sh.cf[9], b0_f = sh.cf[10];
  const float sqrt_h_f = sh.cf[11];

  {
  const R* src = (a.src == nullptr || n == 0) ? (const R*)a.src0
                                              : (const R*)a.src + (size_t)(n - 1) * a.pitch;
  // ---------------- prologue: load, match, first mean ------------------
  int flips = 0;
  R s_in = (R)0;
  {
    int mode0 = kMatchIdentity, mode1 = kMatchIdentity;
    R a0 = 0, b0 = 0, c0m = 0, a1 = 0, b1 = 0, c1m = 0;
    if (a.aff != nullptr) {
      const double* af = a.aff + (size_t)(a.aff_fixed ? 0 : n) * 2 * kAff;
      mode0 = (int)af[0];
      mode1 = two ? (int)af[kAff] : kMatchIdentity;
      a0 = (R)af[1]; b0 = (R)af[2]; c0m = (R)af[3];
      a1 = (R)af[kAff + 1]; b1 = (R)af[kAff + 2]; c1m = (R)af[kAff + 3];
    }
    const bool match = mode0 != kMatchIdentity || mode1 != kMatchIdentity;
    const bool redraw = mode0 == kMatchRedraw || mode1 == kMatchRedraw;
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
          R z[4] = {0, 0, 0, 0};
          R zr[4] = {0, 0, 0, 0};
          if (redraw) {
            normals4<R>(philox4x32_10(rng_counter((uint32_t)q, 0u, (uint32_t)n, 2u, a.ptag), a.key0, a.key1), z);
            if (two)
              normals4<R>(philox4x32_10(rng_counter((uint32_t)q, 1u, (uint32_t)n, 2u, a.ptag), a.key0, a.key1), zr);
          }
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const R xv = v[w];
            const int r = (two && !(xv < thr)) ? 1 : 0;
            const int mode = r ? mode1 : mode0;
            R y = xv;
            if (mode == kMatchAffine) {
              y = r ? apply_affine(xv, a1, b1, c1m) : apply_affine(xv, a0, b0, c0m);
            } else if (mode == kMatchRedraw) {
              y = r ? fmaR(b1, zr[w], a1) : fmaR(b0, z[w], a0);
            }
            v[w] = y;
            if (two && ((!(y < thr)) ? 1 : 0) != r && (4 * (long long)q + w < a.P)) flips += 1;
          }
        }
        // zero the lanes past P so that sums see only real particles
        if (q == qlast) {
          if (plast < 4) v[3] = (R)0;
          if (plast < 3) v[2] = (R)0;
          if (plast < 2) v[1] = (R)0;
        }
        s_in += (v[0] + v[1]) + (v[2] + v[3]);
      }
      xs.put(i, v);
    }
  }
  {
    double v[2];
    v[0] = (double)s_in;
    v[1] = (double)flips;
    warp_reduce_to_shared<2>(sh, v, 0u, 0u);
    __syncthreads();
    if (warp == 0) {
      if (!group_finish<2>(sh, grp, 0u, 0u)) {
        if (lane == 0) sh.abort = 1;
      } else if (lane == 0) {
        publish_uniforms(sh, a);
      }
    }
    __syncthreads();
    if (sh.abort) return false;
  }
  const double flips_tot = sh.tot[1];
  const double m_in = sh.uni[0];

  // ---------------- Euler-Maruyama steps --------------------------------
  for (int j = 0; j < a.nf; ++j) {
    const R base = uniform_of<R>(sh, 1);  // kappa m_j + c0
    const R boff = uniform_of<R>(sh, 2);  // (BE m_j + B0) sqrt(h)
    if (a.rec_uni != nullptr) {
      // the adjoint replays steps from exactly these values
      const long long gs = a.step_offset + j;
      if (g == 0 && tid == 0) {
        R* u = (R*)a.rec_uni + 3 * gs;
        u[0] = uniform_of<R>(sh, 0);
        u[1] = base;
        u[2] = MULT ? boff : b0sq;  // the noise amplitude this step used
      }
      if (gs % a.ckpt_every == 0) {
        R* row = (R*)a.rec_ckpt + (size_t)(gs / a.ckpt_every) * a.pitch;
#pragma unroll kUnroll
        for (int i = 0; i < loop_n; ++i) {
          if (i < nq) {
            R v[4];
            xs.get(i, v);
            Quad<R>::store(row + 4 * (size_t)(qb + tid + i * kTPB), v);
          }
        }
      }
    }
    R s = (R)0;
#pragma unroll kUnroll
    for (int i = 0; i < loop_n; ++i) {
      if (i < nq) {
        const uint32_t q = (uint32_t)(qb + tid + i * kTPB);
        R v[4];
        xs.get(i, v);
        R z[4];
        normals4<R>(philox4x32_10(rng_counter(q, (uint32_t)j, (uint32_t)n, 0u, a.ptag), a.key0, a.key1), z);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const R xv = v[w];
          const R drift = fmaR(fmaR(nc3, xv * xv, c1), xv, base);
          const R amp = MULT ? fmaR(bsq, xv, boff) : b0sq;
          v[w] = fmaR(amp, z[w], fmaR(h, drift, xv));
        }
        if (q == (uint32_t)qlast) {
          if (plast < 4) v[3] = (R)0;
          if (plast < 3) v[2] = (R)0;
          if (plast < 2) v[1] = (R)0;
        }
        s += (v[0] + v[1]) + (v[2] + v[3]);
        xs.put(i, v);
      }
    }
    warp_sum_to_shared(sh, s);
    __syncthreads();
    if (warp == 0) {
      bool ok;
      if constexpr (sizeof(R) == 4) {
        ok = step_sum_finish_f(sh, grp, inv_p, kappa_f, c0_f, be_f, b0_f, sqrt_h_f);
      } else {
        ok = group_finish<1>(sh, grp, 0u, 0u);
        if (ok && lane == 0) publish_uniforms(sh, a);
      }
      if (!ok && lane == 0) sh.abort = 1;
    }
    __syncthreads();
    if (sh.abort) return false;
  }

  // ---------------- epilogue: store and restrict -----------------------
  // pass 1 (with the store): counts and sums per region
  {
    R* dst = a.dst != nullptr ? (R*)a.dst + (size_t)(a.dst_fixed ? 0 : n) * a.pitch : nullptr;
    int n0 = 0, n1 = 0;
    Acc<R> s0, s1;
#pragma unroll kUnroll
    for (int i = 0; i < loop_n; ++i) {
      if (i < nq) {
        const int q = qb + tid + i * kTPB;
        R x4[4];
        xs.get(i, x4);
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
            if (two && !(x4[w] < thr)) {
              n1 += 1;
              s1.add(x4[w]);
            } else {
              n0 += 1;
              s0.add(x4[w]);
            }
          }
        }
      }
    }
    double v[4] = {(double)n0, s0.get(), (double)n1, s1.get()};
    warp_reduce_to_shared<4>(sh, v, 0u, 0u);
    __syncthreads();
    if (warp == 0 && !group_finish<4>(sh, grp, 0u, 0u) && lane == 0) sh.abort = 1;
    __syncthreads();
    if (sh.abort) return false;
  }
  const double cnt0 = sh.tot[0], cnt1 = sh.tot[2];
  const double mean0 = cnt0 > 0 ? sh.tot[1] / cnt0 : 0.0;
  const double mean1 = cnt1 > 0 ? sh.tot[3] / cnt1 : 0.0;
  const double gmean = (sh.tot[1] + sh.tot[3]) / (double)a.P;
  __syncthreads();
  // pass 2: centred sums and extremes
  {
    const Centre<R> cg(gmean), c0c(mean0), c1c(mean1);
    Acc<R> ss0, ss1, ssg;
    R lo0 = (R)INFINITY, hi0 = (R)-INFINITY, lo1 = (R)INFINITY, hi1 = (R)-INFINITY;
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
            if (two && !(xv < thr)) {
              const R d = c1c.diff(xv);
              ss1.add(d * d);
              lo1 = lo1 < xv ? lo1 : xv;
              hi1 = hi1 > xv ? hi1 : xv;
            } else {
              const R d = c0c.diff(xv);
              ss0.add(d * d);
              lo0 = lo0 < xv ? lo0 : xv;
              hi0 = hi0 > xv ? hi0 : xv;
            }
          }
        }
      }
    }
    double v[7] = {ss0.get(), ss1.get(), ssg.get(), (double)lo0, (double)hi0, (double)lo1, (double)hi1};
    const unsigned mn = (1u << 3) | (1u << 5), mx = (1u << 4) | (1u << 6);
    warp_reduce_to_shared<7>(sh, v, mn, mx);
    __syncthreads();
    if (warp == 0 && !group_finish<7>(sh, grp, mn, mx) && lane == 0) sh.abort = 1;
    __syncthreads();
    if (sh.abort) return false;
  }
  if (g == 0 && tid == 0 && a.stats != nullptr) {
    double* st = a.stats + (size_t)(a.stats_fixed ? 0 : n) * kStat;
    st[0] = cnt0;
    st[1] = mean0;
    st[2] = cnt0 > 0 ? sh.tot[0] / cnt0 : 0.0;
    st[3] = sh.tot[3];
    st[4] = sh.tot[4];
    st[5] = cnt1;
    st[6] = mean1;
    st[7] = cnt1 > 0 ? sh.tot[1] / cnt1 : 0.0;
    st[8] = sh.tot[5];
    st[9] = sh.tot[6];
    st[10] = gmean;
    st[11] = sh.tot[2] / (double)a.P;
    st[12] = flips_tot;
    st[13] = m_in;
    st[14] = 0.0;
    st[15] = 0.0;
    if (!(fabs(gmean) < INFINITY) || !(st[11] < INFINITY)) atomicOr(a.status, kStatusNumeric);
    if (flips_tot > 0.0) atomicOr(a.status, kStatusRegionFlip);
  }
    __syncthreads();
  }
  return true;
}

template <typename R, int NQ, bool MULT>
__global__ void __launch_bounds__(kTPB, (FineOccupancy<R, NQ>::value)) k_fine(const FineArgs a) {
  __shared__ GroupShared sh;
  const int G = a.G;
  const int n_slots = gridDim.x / G;
  const int slot = blockIdx.x / G;
  const int g = blockIdx.x - slot * G;
  if (slot >= n_slots) return;
  Group grp;
  grp.part = a.partials + (size_t)slot * 2 * G * (kNV + 1);
  grp.counter = a.counters + slot;
  grp.status = a.status;
  grp.limit_ns = a.wait_limit_ns;
  grp.G = G;
  grp.g = g;
  grp.epoch = 0;
  if (threadIdx.x == 0) sh.abort = 0;
  QuadStore<R, NQ> xs;
  xs.bind();
  for (int task = slot; task < a.n_tasks; task += n_slots) {
    if (!fine_task<R, NQ, MULT>(a, a.slice_begin + task, g, grp, sh, xs)) return;
  }
}

}  // namespace mmp
