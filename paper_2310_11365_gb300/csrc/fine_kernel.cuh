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
  double tot[kNV];          // group totals, broadcast
  double uni[4];            // per-step uniforms derived from the mean
  int abort;
};

// Group-reduction context of one CTA.
struct Group {
  double* part;         // [2][G][kNV] for this slot
  unsigned* counter;    // arrivals of this slot
  unsigned* status;
  unsigned long long limit_ns;
  int G, g;
  unsigned epoch;
};

// Warp 0 finishes a group reduction of nv values whose per-warp partials
// sit in sh.red.  min_mask / max_mask select values combined by min / max
// (all others are summed).  Returns false if the cross-CTA wait gave up.
__device__ __forceinline__ bool group_finish(GroupShared& sh, Group& grp, int nv, unsigned min_mask,
                                             unsigned max_mask) {
  const int lane = threadIdx.x & 31;
  double v[kNV];
#pragma unroll
  for (int k = 0; k < kNV; ++k) {
    const double ident = (min_mask >> k & 1) ? INFINITY : ((max_mask >> k & 1) ? -INFINITY : 0.0);
    v[k] = (k < nv && lane < kWarps) ? sh.red[lane][k] : ident;
  }
  // butterfly over the kWarps lanes that hold values
#pragma unroll
  for (int off = kWarps / 2; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < kNV; ++k) {
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
      for (int k = 0; k < kNV; ++k)
        if (k < nv) mine[k] = v[k];
      red_release_gpu_add(grp.counter, 1u);
    }
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
    if (!ok) {
      if (lane == 0) atomicOr(grp.status, kStatusTimeout);
      return false;
    }
    const double* all = grp.part + (size_t)parity * grp.G * kNV;
#pragma unroll
    for (int k = 0; k < kNV; ++k) {
      const double ident = (min_mask >> k & 1) ? INFINITY : ((max_mask >> k & 1) ? -INFINITY : 0.0);
      v[k] = ident;
    }
    for (int c = lane; c < grp.G; c += 32) {
#pragma unroll
      for (int k = 0; k < kNV; ++k) {
        if (k < nv) {
          const double o = __ldcg(all + (size_t)c * kNV + k);
          v[k] = (min_mask >> k & 1) ? fmin(v[k], o) : ((max_mask >> k & 1) ? fmax(v[k], o) : v[k] + o);
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int k = 0; k < kNV; ++k) {
        if (k < nv) {
          const double o = __shfl_xor_sync(0xffffffffu, v[k], off);
          v[k] = (min_mask >> k & 1) ? fmin(v[k], o) : ((max_mask >> k & 1) ? fmax(v[k], o) : v[k] + o);
        }
      }
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kNV; ++k)
      if (k < nv) sh.tot[k] = v[k];
  }
  return true;
}

// Per-warp stage of a sum of one per-thread value, exact to double-float for
// float input (error-free two-sums) and plain double otherwise.
__device__ __forceinline__ void warp_sum_to_shared(GroupShared& sh, float s) {
  float hi = s, lo = 0.0f;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, off);
    const float olo = __shfl_xor_sync(0xffffffffu, lo, off);
    float t, e;
    two_sum(hi, ohi, t, e);
    lo = __fadd_rn(__fadd_rn(lo, olo), e);
    hi = t;
  }
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5][0] = (double)hi + (double)lo;
}
__device__ __forceinline__ void warp_sum_to_shared(GroupShared& sh, double s) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5][0] = s;
}

// General per-warp stage of nv double values.
__device__ __forceinline__ void warp_reduce_to_shared(GroupShared& sh, double v[kNV], int nv,
                                                      unsigned min_mask, unsigned max_mask) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < kNV; ++k) {
      if (k < nv) {
        const double o = __shfl_xor_sync(0xffffffffu, v[k], off);
        v[k] = (min_mask >> k & 1) ? fmin(v[k], o) : ((max_mask >> k & 1) ? fmax(v[k], o) : v[k] + o);
      }
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < kNV; ++k)
      if (k < nv) sh.red[threadIdx.x >> 5][k] = v[k];
  }
}

// After a reduction of the running sum: publish the per-step uniforms
// (mean, kappa m + c0, diffusion offset) so that no thread does FP64 work
// in the step loop.
__device__ __forceinline__ void publish_uniforms(GroupShared& sh, const FineArgs& a) {
  const double m = sh.tot[0] / (double)a.P;
  sh.uni[0] = m;
  sh.uni[1] = a.kappa * m + a.c0;
  sh.uni[2] = (a.BE * m + a.B0) * a.sqrt_h;
}

// Resident CTAs per SM the register budget is sized for: the quads a thread
// holds dominate its registers, so fewer CTAs fit as NQ grows.
template <typename R, int NQ>
struct FineOccupancy {
  static constexpr int value = sizeof(R) == 4 ? (NQ <= 2 ? 5 : (NQ <= 4 ? 4 : 3)) : (NQ <= 2 ? 3 : 2);
};

template <typename R, int NQ, bool MULT>
__global__ void __launch_bounds__(kTPB, (FineOccupancy<R, NQ>::value)) k_fine(const FineArgs a) {
  __shared__ GroupShared sh;
  const int G = a.G;
  const int n_slots = gridDim.x / G;
  const int slot = blockIdx.x / G;
  const int g = blockIdx.x - slot * G;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  if (slot >= n_slots) return;

  const int qb = (int)(((long long)a.Q * g) / G);
  const int qe = (int)(((long long)a.Q * (g + 1)) / G);
  const int span = qe - qb - tid;
  const int nq = span <= 0 ? 0 : min(NQ, (span + kTPB - 1) / kTPB);
  const int qlast = a.Q - 1;
  const int plast = (int)(a.P - 4LL * qlast);  // valid lanes of the last quad, 1..4

  Group grp;
  grp.part = a.partials + (size_t)slot * 2 * G * kNV;
  grp.counter = a.counters + slot;
  grp.status = a.status;
  grp.limit_ns = a.wait_limit_ns;
  grp.G = G;
  grp.g = g;
  grp.epoch = 0;
  if (tid == 0) sh.abort = 0;

  const R h = (R)a.h;
  const R nc3 = (R)a.nc3;
  const R c1 = (R)a.c1;
  const R bsq = (R)(a.B * a.sqrt_h);      // state-proportional part of b sqrt(h)
  const R b0sq = (R)(a.B0 * a.sqrt_h);    // additive noise amplitude
  const R thr = (R)a.thr;
  const bool two = a.n_regions > 1;

  for (int task = slot; task < a.n_tasks; task += n_slots) {
    const int n = a.slice_begin + task;
    const R* src = (a.src == nullptr || n == 0) ? (const R*)a.src0
                                                : (const R*)a.src + (size_t)(n - 1) * a.pitch;
    R x[NQ][4];
    // ---------------- prologue: load and match --------------------------
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
      const int q = qb + tid + i * kTPB;
      if (i < nq && (q != qlast || plast == 4)) {
        Quad<R>::load(src + 4 * (size_t)q, x[i]);
      } else {
        // past the group's range, or the ragged last quad: guarded scalar
        // loads so that a buffer of exactly P values is never over-read
#pragma unroll
        for (int w = 0; w < 4; ++w) x[i][w] = (i < nq && w < plast) ? src[4 * (size_t)q + w] : (R)0;
      }
    }
    double flips = 0.0;
    if (a.aff != nullptr) {
      const double* af = a.aff + (size_t)(a.aff_fixed ? 0 : n) * 2 * kAff;
      const int mode0 = (int)af[0], mode1 = (int)af[kAff];
      const R a0 = (R)af[1], b0 = (R)af[2], c0m = (R)af[3];
      const R a1 = (R)af[kAff + 1], b1 = (R)af[kAff + 2], c1m = (R)af[kAff + 3];
      if (mode0 != kMatchIdentity || (two && mode1 != kMatchIdentity)) {
        const bool redraw = mode0 == kMatchRedraw || (two && mode1 == kMatchRedraw);
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
          if (i < nq) {
            const uint32_t q = (uint32_t)(qb + tid + i * kTPB);
            R z[4] = {0, 0, 0, 0};
            R zr[4] = {0, 0, 0, 0};
            if (redraw) {
              normals4<R>(philox4x32_10(rng_counter(q, 0u, (uint32_t)n, 2u, a.ptag), a.key0, a.key1), z);
              if (two)
                normals4<R>(philox4x32_10(rng_counter(q, 1u, (uint32_t)n, 2u, a.ptag), a.key0, a.key1), zr);
            }
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              const R xv = x[i][w];
              const int r = (two && !(xv < thr)) ? 1 : 0;
              const int mode = r ? mode1 : mode0;
              R y = xv;
              if (mode == kMatchAffine) {
                y = r ? apply_affine(xv, a1, b1, c1m) : apply_affine(xv, a0, b0, c0m);
              } else if (mode == kMatchRedraw) {
                y = r ? a1 + b1 * zr[w] : a0 + b0 * z[w];
              }
              x[i][w] = y;
              if (two && ((!(y < thr)) ? 1 : 0) != r && (4 * (long long)q + w < a.P)) flips += 1.0;
            }
          }
        }
      }
    }
    // zero the lanes past P so that sums see only real particles
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
      if (i < nq && qb + tid + i * kTPB == qlast) {
        if (plast < 4) x[i][3] = (R)0;
        if (plast < 3) x[i][2] = (R)0;
        if (plast < 2) x[i][1] = (R)0;
      }
    }
    {
      double v[kNV];
      R s = (R)0;
#pragma unroll
      for (int i = 0; i < NQ; ++i)
        if (i < nq) s += (x[i][0] + x[i][1]) + (x[i][2] + x[i][3]);
      v[0] = (double)s;
      v[1] = flips;
      warp_reduce_to_shared(sh, v, 2, 0u, 0u);
      __syncthreads();
      if (warp == 0) {
        if (!group_finish(sh, grp, 2, 0u, 0u)) {
          if (lane == 0) sh.abort = 1;
        } else if (lane == 0) {
          publish_uniforms(sh, a);
        }
      }
      __syncthreads();
      if (sh.abort) return;
    }
    const double flips_tot = sh.tot[1];
    const double m_in = sh.uni[0];

    // ---------------- Euler-Maruyama steps --------------------------------
    for (int j = 0; j < a.nf; ++j) {
      const R base = (R)sh.uni[1];   // kappa m_j + c0
      const R boff = (R)sh.uni[2];   // (BE m_j + B0) sqrt(h)
      R s = (R)0;
#pragma unroll
      for (int i = 0; i < NQ; ++i) {
        if (i < nq) {
          const uint32_t q = (uint32_t)(qb + tid + i * kTPB);
          R z[4];
          normals4<R>(philox4x32_10(rng_counter(q, (uint32_t)j, (uint32_t)n, 0u, a.ptag), a.key0, a.key1), z);
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const R xv = x[i][w];
            const R drift = fma(fma(nc3, xv * xv, c1), xv, base);
            const R amp = MULT ? fma(bsq, xv, boff) : b0sq;
            x[i][w] = fma(amp, z[w], fma(h, drift, xv));
          }
          if (q == (uint32_t)qlast) {
            if (plast < 4) x[i][3] = (R)0;
            if (plast < 3) x[i][2] = (R)0;
            if (plast < 2) x[i][1] = (R)0;
          }
          s += (x[i][0] + x[i][1]) + (x[i][2] + x[i][3]);
        }
      }
      warp_sum_to_shared(sh, s);
      __syncthreads();
      if (warp == 0) {
        if (!group_finish(sh, grp, 1, 0u, 0u)) {
          if (lane == 0) sh.abort = 1;
        } else if (lane == 0) {
          publish_uniforms(sh, a);
        }
      }
      __syncthreads();
      if (sh.abort) return;
    }

    // ---------------- epilogue: store and restrict -----------------------
    if (a.dst != nullptr) {
      R* dst = (R*)a.dst + (size_t)(a.dst_fixed ? 0 : n) * a.pitch;
#pragma unroll
      for (int i = 0; i < NQ; ++i) {
        const int q = qb + tid + i * kTPB;
        if (i < nq && (q != qlast || plast == 4)) {
          Quad<R>::store(dst + 4 * (size_t)q, x[i]);
        } else if (i < nq) {
#pragma unroll
          for (int w = 0; w < 4; ++w)
            if (w < plast) dst[4 * (size_t)q + w] = x[i][w];
        }
      }
    }
    // pass 1: counts and sums per region
    {
      double v[kNV];
#pragma unroll
      for (int k = 0; k < kNV; ++k) v[k] = 0.0;
#pragma unroll
      for (int i = 0; i < NQ; ++i) {
        if (i < nq) {
          const int q = qb + tid + i * kTPB;
          const int valid = q == qlast ? plast : 4;
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            if (w < valid) {
              const double xv = (double)x[i][w];
              if (two && !(x[i][w] < thr)) {
                v[2] += 1.0;
                v[3] += xv;
              } else {
                v[0] += 1.0;
                v[1] += xv;
              }
            }
          }
        }
      }
      warp_reduce_to_shared(sh, v, 4, 0u, 0u);
      __syncthreads();
      if (warp == 0 && !group_finish(sh, grp, 4, 0u, 0u) && lane == 0) sh.abort = 1;
      __syncthreads();
      if (sh.abort) return;
    }
    const double cnt0 = sh.tot[0], cnt1 = sh.tot[2];
    const double mean0 = cnt0 > 0 ? sh.tot[1] / cnt0 : 0.0;
    const double mean1 = cnt1 > 0 ? sh.tot[3] / cnt1 : 0.0;
    const double gmean = (sh.tot[1] + sh.tot[3]) / (double)a.P;
    __syncthreads();
    // pass 2: centred sums and extremes
    {
      double v[kNV];
      v[0] = 0.0; v[1] = 0.0; v[2] = 0.0;
      v[3] = INFINITY; v[4] = -INFINITY; v[5] = INFINITY; v[6] = -INFINITY;
      v[7] = 0.0;
#pragma unroll
      for (int i = 0; i < NQ; ++i) {
        if (i < nq) {
          const int q = qb + tid + i * kTPB;
          const int valid = q == qlast ? plast : 4;
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            if (w < valid) {
              const double xv = (double)x[i][w];
              const double dg = xv - gmean;
              v[2] += dg * dg;
              if (two && !(x[i][w] < thr)) {
                const double d = xv - mean1;
                v[1] += d * d;
                v[5] = fmin(v[5], xv);
                v[6] = fmax(v[6], xv);
              } else {
                const double d = xv - mean0;
                v[0] += d * d;
                v[3] = fmin(v[3], xv);
                v[4] = fmax(v[4], xv);
              }
            }
          }
        }
      }
      const unsigned mn = (1u << 3) | (1u << 5), mx = (1u << 4) | (1u << 6);
      warp_reduce_to_shared(sh, v, 7, mn, mx);
      __syncthreads();
      if (warp == 0 && !group_finish(sh, grp, 7, mn, mx) && lane == 0) sh.abort = 1;
      __syncthreads();
      if (sh.abort) return;
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
}

}  // namespace mmp
