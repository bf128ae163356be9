// driver.cu -- the device-side Parareal driver: coarse moment-ODE sweep,
// iterator and matching parameters, fraction learning and the convergence
// test, all in FP64 (one warp per problem; the sweep over slices is
// sequential by nature, Sec. 3.1).
#include <cmath>

#include "driver.cuh"
#include "mmp_internal.cuh"

namespace mmp {

namespace {

struct Macro {
  double frac[2], mean[2], var[2];
};

__device__ void macro_load(const double* r, Macro& m) {
  m.frac[0] = r[0]; m.mean[0] = r[1]; m.var[0] = r[2];
  m.frac[1] = r[3]; m.mean[1] = r[4]; m.var[1] = r[5];
}

// Global (M, V) of a macro state: Eq. (mixture_of_distributions_mean_variance)
// with variances in place of the printed squares; one region is (M, V).
__device__ void mixture(const DriverArgs& a, const Macro& r, double& M, double& V) {
  if (a.I < 2) {
    M = r.mean[0];
    V = r.var[0];
    return;
  }
  const double m = r.frac[0] * r.mean[0] + r.frac[1] * r.mean[1];
  const double s = r.frac[0] * (r.mean[0] * r.mean[0] + r.var[0]) +
                   r.frac[1] * (r.mean[1] * r.mean[1] + r.var[1]);
  M = m;
  V = s - m * m;
}

__device__ void macro_store(const DriverArgs& a, double* r, const Macro& m) {
  r[0] = m.frac[0]; r[1] = m.mean[0]; r[2] = m.var[0];
  r[3] = m.frac[1]; r[4] = m.mean[1]; r[5] = m.var[1];
  double M, V;
  mixture(a, m, M, V);
  r[6] = M;
  r[7] = V;
}

// Coarse propagator C_n: a moment ODE per region with the fractions frozen
// (Def. 3.2), forward Euler with nc substeps, the mean field M = sum_j P_j m_j
// (the region's own mean when I = 1).  Models (Sec. 2), for the drift
// a(x) = -c3 x^3 + c1 x + kappa M + c0 and diffusion b(x) = B x + BE M + B0:
//   closure (Gaussian-assumed density, expectations in closed form):
//     m' = -c3 (m^3 + 3 m v) + c1 m + kappa M + c0
//     v' = 2 (-3 c3 v (m^2 + v) + c1 v) + B^2 v + (B m + BE M + B0)^2
//   Taylor (Eq. moment_model_class_1): m' = a(m) + a_XX(m) v / 2,
//     v' = (2 a_X(m) + B^2) v + b(m)^2
//   sigma-point (Eq. Gaussian_model_McK_V_SDE with a k-point rule on
//     N(m, v)): m' = E[a], v' = 2 E[(X - m) a] + E[b^2]; k = 2: m -+ sqrt(v),
//     weights 1/2; k = 3: m, m -+ sqrt(3 v), weights 2/3, 1/6, 1/6.
// For c3 = 0 every model is the exact moment ODE of the linear SDE (Lemma 2.1).
__device__ double drift_at(const DriverArgs& a, double x, double M) {
  return a.nc3 * x * x * x + a.c1 * x + a.kappa * M + a.c0;
}
__device__ double diffusion_at(const DriverArgs& a, double x, double M) {
  return a.B * x + a.BE * M + a.B0;
}

__device__ void coarse_rhs(const DriverArgs& a, double m, double v, double M, double& dm, double& dv) {
  const double c3 = -a.nc3;
  if (a.coarse_model == MMP_COARSE_TAYLOR) {
    const double ax = -3.0 * c3 * m * m + a.c1;
    const double axx = -6.0 * c3 * m;
    const double b = diffusion_at(a, m, M);
    dm = drift_at(a, m, M) + 0.5 * axx * v;
    dv = (2.0 * ax + a.B * a.B) * v + b * b;
  } else if (a.coarse_model == MMP_COARSE_SIGMA2 || a.coarse_model == MMP_COARSE_SIGMA3) {
    double xs[3], ws[3];
    int k;
    if (a.coarse_model == MMP_COARSE_SIGMA2) {
      const double d = sqrt(v > 0.0 ? v : 0.0);
      xs[0] = m - d; xs[1] = m + d;
      ws[0] = 0.5; ws[1] = 0.5;
      k = 2;
    } else {
      const double d = sqrt(3.0 * (v > 0.0 ? v : 0.0));
      xs[0] = m; xs[1] = m - d; xs[2] = m + d;
      ws[0] = 2.0 / 3.0; ws[1] = 1.0 / 6.0; ws[2] = 1.0 / 6.0;
      k = 3;
    }
    double ea = 0.0, exa = 0.0, eb2 = 0.0;
    for (int s = 0; s < k; ++s) {
      const double av = drift_at(a, xs[s], M);
      const double bv = diffusion_at(a, xs[s], M);
      ea += ws[s] * av;
      exa += ws[s] * (xs[s] - m) * av;
      eb2 += ws[s] * bv * bv;
    }
    dm = ea;
    dv = 2.0 * exa + eb2;
  } else {
    const double ex3 = m * m * m + 3.0 * m * v;
    const double cov3 = 3.0 * v * (m * m + v);
    const double eb = a.B * m + a.BE * M + a.B0;
    dm = -c3 * ex3 + a.c1 * m + a.kappa * M + a.c0;
    dv = 2.0 * (-c3 * cov3 + a.c1 * v) + a.B * a.B * v + eb * eb;
  }
}

__device__ void coarse(const DriverArgs& a, const Macro& in, Macro& out) {
  out = in;
  for (int s = 0; s < a.nc; ++s) {
    double M = out.mean[0];
    if (a.I > 1) M = out.frac[0] * out.mean[0] + out.frac[1] * out.mean[1];
    double dm[2], dv[2];
    for (int i = 0; i < a.I; ++i) coarse_rhs(a, out.mean[i], out.var[i], M, dm[i], dv[i]);
    for (int i = 0; i < a.I; ++i) {
      out.mean[i] = out.mean[i] + a.hc * dm[i];
      out.var[i] = out.var[i] + a.hc * dv[i];
    }
  }
}

// The transform of the driver's acceptance test, evaluated exactly as the
// fine kernel will apply it (same precision, same rounding of parameters).
__device__ bool stays_in_region(const DriverArgs& a, int i, double extreme, double delta, double sm1,
                                double m) {
  if (a.precision == MMP_MIXED) {
    const float y = apply_affine((float)extreme, (float)delta, (float)sm1, (float)m);
    const float thr = (float)a.thr;
    return i == 0 ? (y < thr) : !(y < thr);
  }
  const double y = apply_affine(extreme, delta, sm1, m);
  return i == 0 ? (y < a.thr) : !(y < a.thr);
}

__device__ void set_aff(double* af, int mode, double p, double q, double r) {
  af[0] = (double)mode;
  af[1] = p;
  af[2] = q;
  af[3] = r;
}

// Matching record for T([mu, sigma], u) on a region with restriction
// (count, m, v): Eq. (multimodal_M); identity for an empty region.
__device__ void matching_record(double* af, double count, double m, double v, double mu, double sigma) {
  if (count <= 0.0 || !(sigma >= 0.0)) {
    set_aff(af, kMatchIdentity, 0.0, 0.0, 0.0);
  } else if (v == 0.0) {
    set_aff(af, kMatchRedraw, mu, sqrt(sigma), 0.0);
  } else {
    set_aff(af, kMatchAffine, mu - m, sqrt(sigma / v) - 1.0, m);
  }
}

// ---------------------------------------------------------------------------
// Learning of the region-0 fraction (Def. 3.4, App. H):
//   P(t) = beta + (p0 - beta) e^{alpha t}
// fitted by Levenberg-Marquardt on the exact slice ends t_1..t_k.  Settings
// (the paper gives none): start from the regression y_{n+1} = r y_n + c,
// damping 1e-3 scaled by diag(J^T J), /10 on success, x10 on failure, at
// most 100 iterations, stop on a relative step below 1e-15 or damping above
// 1e12, then three undamped Gauss-Newton steps; the fit is used only if
// alpha < 0 and 0 <= beta <= 1.
// The sums over points run across the warp (fixed butterfly order), so every
// lane takes the same decisions.
// ---------------------------------------------------------------------------
__device__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__device__ double frac0_at(const DriverArgs& a, int n) {
  // fraction of region 0 at slice end n from the fine outputs (n >= 1) or u0
  const double* st = n == 0 ? a.stats_u0 : a.stats + (size_t)(n - 1) * kStat;
  return st[0] / (double)a.P;
}

__device__ double lsq_cost(const DriverArgs& a, int npts, double p0, double al, double be) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int n = 1 + lane; n <= npts; n += 32) {
    const double t = n * a.dT;
    const double r = frac0_at(a, n) - (be + (p0 - be) * exp(al * t));
    s += r * r;
  }
  return warp_sum(s);
}

__device__ bool lsq_fit(const DriverArgs& a, int npts, double p0, double& alpha, double& beta) {
  const int lane = threadIdx.x & 31;
  if (npts < 2) return false;
  double sx = 0, sy = 0, sxx = 0, sxy = 0;
  for (int n = 1 + lane; n <= npts; n += 32) {
    const double xv = frac0_at(a, n - 1), yv = frac0_at(a, n);
    sx += xv; sy += yv; sxx += xv * xv; sxy += xv * yv;
  }
  sx = warp_sum(sx); sy = warp_sum(sy); sxx = warp_sum(sxx); sxy = warp_sum(sxy);
  const double cnt = (double)npts;
  const double den = sxx - sx * sx / cnt;
  double al = -1.0 / (npts * a.dT);
  double be = frac0_at(a, npts);
  if (den > 0.0) {
    const double r = (sxy - sx * sy / cnt) / den;
    const double c = (sy - r * sx) / cnt;
    if (r > 0.0 && r < 1.0) {
      al = log(r) / a.dT;
      be = c / (1.0 - r);
    }
  }
  double lambda = 1e-3;
  double cost = lsq_cost(a, npts, p0, al, be);
  for (int it = 0; it < 100; ++it) {
    double jaa = 0, jab = 0, jbb = 0, ga = 0, gb = 0;
    for (int n = 1 + lane; n <= npts; n += 32) {
      const double t = n * a.dT;
      const double e = exp(al * t);
      const double f = be + (p0 - be) * e;
      const double r = frac0_at(a, n) - f;
      const double da = (p0 - be) * t * e;
      const double db = 1.0 - e;
      jaa += da * da; jab += da * db; jbb += db * db;
      ga += da * r; gb += db * r;
    }
    jaa = warp_sum(jaa); jab = warp_sum(jab); jbb = warp_sum(jbb);
    ga = warp_sum(ga); gb = warp_sum(gb);
    const double A = jaa * (1.0 + lambda), D = jbb * (1.0 + lambda), Bm = jab;
    const double det = A * D - Bm * Bm;
    if (!(det > 0.0) || !isfinite(det)) {
      lambda *= 10.0;
      if (lambda > 1e12) break;
      continue;
    }
    const double sa = (D * ga - Bm * gb) / det;
    const double sb = (A * gb - Bm * ga) / det;
    const double na = al + sa, nb = be + sb;
    const double ncost = lsq_cost(a, npts, p0, na, nb);
    if (isfinite(ncost) && ncost < cost) {
      al = na; be = nb; cost = ncost;
      lambda /= 10.0;
      const double rel = fmax(fabs(sa) / (fabs(al) + 1e-300), fabs(sb) / (fabs(be) + 1e-300));
      if (rel < 1e-15) break;
    } else {
      lambda *= 10.0;
      if (lambda > 1e12) break;
    }
  }
  // undamped Gauss-Newton refinement to the minimiser (the cost test above
  // cannot resolve the last step once its change is below rounding)
  for (int it = 0; it < 3; ++it) {
    double jaa = 0, jab = 0, jbb = 0, ga = 0, gb = 0;
    for (int n = 1 + lane; n <= npts; n += 32) {
      const double t = n * a.dT;
      const double e = exp(al * t);
      const double r = frac0_at(a, n) - (be + (p0 - be) * e);
      const double da = (p0 - be) * t * e;
      const double db = 1.0 - e;
      jaa += da * da; jab += da * db; jbb += db * db;
      ga += da * r; gb += db * r;
    }
    jaa = warp_sum(jaa); jab = warp_sum(jab); jbb = warp_sum(jbb);
    ga = warp_sum(ga); gb = warp_sum(gb);
    const double det = jaa * jbb - jab * jab;
    if (!(det > 0.0) || !isfinite(det)) break;
    al += (jbb * ga - jab * gb) / det;
    be += (jaa * gb - jab * ga) / det;
  }
  alpha = al;
  beta = be;
  return al < 0.0 && be >= 0.0 && be <= 1.0 && isfinite(al) && isfinite(be);
}

}  // namespace

// One warp per problem.  sweep == 0: lifting (k = 0).  sweep k >= 1: the
// coarse/iterator sweep after fine sweep k, Eq. (mM_parareal_other_k_NEW).
__device__ void driver_body(const DriverArgs& a) {
  const int lane = threadIdx.x & 31;
  const int N = a.N, I = a.I;
  double* ctl = a.ctl;

  if (a.sweep == 0) {
    if (lane != 0) return;
    // rho^0_0 = R(u0); rho^0_{n+1} = C_n(rho^0_n); u^0_n = T(rho^0_n, u0)
    const double* s0 = a.stats_u0;
    Macro r;
    r.frac[0] = s0[0] / (double)a.P; r.mean[0] = s0[1]; r.var[0] = s0[2];
    r.frac[1] = s0[5] / (double)a.P; r.mean[1] = s0[6]; r.var[1] = s0[7];
    if (I < 2) { r.frac[1] = 0.0; r.mean[1] = 0.0; r.var[1] = 0.0; }
    macro_store(a, a.rho, r);
    for (int n = 0; n <= N; ++n) {
      double* af = a.aff + (size_t)n * 2 * kAff;
      for (int i = 0; i < 2; ++i) {
        if (i < I) {
          matching_record(af + i * kAff, s0[i * 5], s0[i * 5 + 1], s0[i * 5 + 2], r.mean[i], r.var[i]);
        } else {
          set_aff(af + i * kAff, kMatchIdentity, 0.0, 0.0, 0.0);
        }
      }
      if (n == N) break;
      Macro nx;
      coarse(a, r, nx);
      double* c = a.cache + (size_t)n * 4;
      c[0] = nx.mean[0]; c[1] = nx.var[0]; c[2] = nx.mean[1]; c[3] = nx.var[1];
      macro_store(a, a.rho + (size_t)(n + 1) * kMom, nx);
      r = nx;
    }
    ctl[0] = 0.0;  // last change
    ctl[1] = 0.0;  // converged
    ctl[2] = 0.0;  // sweeps
    ctl[3] = 0.0;  // done
    ctl[4] = 0.0;  // accepted
    ctl[5] = 0.0;  // rejected
    ctl[6] = 0.0;  // fit alpha
    ctl[7] = 0.0;  // fit beta
    ctl[8] = 0.0;  // fit used
    return;
  }

  const int k = a.sweep;
  // Def. 3.4: fit the fractions of the exact slice ends t_0..t_k
  bool learn = false;
  double alpha = 0.0, beta = 0.0;
  if (a.variant == MMP_LEARNING && I == 2 && k >= 2) {
    const double p0 = frac0_at(a, 0);
    learn = lsq_fit(a, k, p0, alpha, beta);
  }
  if (lane != 0) return;
  const double pk = frac0_at(a, k);

  double change = 0.0;
  int acc = 0, rej = 0;
  bool numeric_bad = false;
  Macro cur;
  macro_load(a.rho, cur);  // rho^{k}_0 = R(u0), unchanged
  for (int n = 0; n < N; ++n) {
    Macro av;
    coarse(a, cur, av);
    const double* b = a.stats + (size_t)n * kStat;
    double* cache = a.cache + (size_t)n * 4;
    double* af = a.aff + (size_t)(n + 1) * 2 * kAff;
    Macro nx;
    for (int i = 0; i < 2; ++i) {
      nx.frac[i] = 0.0; nx.mean[i] = 0.0; nx.var[i] = 0.0;
      set_aff(af + i * kAff, kMatchIdentity, 0.0, 0.0, 0.0);
    }
    for (int i = 0; i < I; ++i) {
      const double cnt = b[i * 5], bm = b[i * 5 + 1], bv = b[i * 5 + 2];
      const double bmin = b[i * 5 + 3], bmax = b[i * 5 + 4];
      if (!(fabs(bm) < INFINITY) || !(bv < INFINITY)) numeric_bad = true;
      if (cnt <= 0.0) {
        // empty region: carry the coarse prediction, move nothing
        nx.mean[i] = av.mean[i];
        nx.var[i] = av.var[i];
        continue;
      }
      // alpha = R(b) + (a - c): a == c returns R(b) exactly (Property 3.3)
      const double am = bm + (av.mean[i] - cache[2 * i]);
      const double avv = bv + (av.var[i] - cache[2 * i + 1]);
      bool accept = avv >= 0.0;
      double delta = 0.0, sm1 = 0.0;
      if (accept && bv > 0.0) {
        delta = am - bm;
        sm1 = sqrt(avv / bv) - 1.0;
      }
      if (accept && a.variant != MMP_UNIMODAL && I > 1) {
        // Def. 3.2: move a region only if no particle leaves it
        if (bv == 0.0) {
          accept = false;
        } else {
          accept = stays_in_region(a, i, i == 0 ? bmax : bmin, delta, sm1, bm);
        }
      }
      if (accept) {
        nx.mean[i] = am;
        nx.var[i] = avv;
        matching_record(af + i * kAff, cnt, bm, bv, am, avv);
        ++acc;
      } else {
        nx.mean[i] = bm;
        nx.var[i] = bv;
        ++rej;
      }
    }
    // fractions come from the fine propagator (Def. 3.2), or from the
    // learned model beyond the exact slices (Def. 3.4)
    for (int i = 0; i < I; ++i) nx.frac[i] = b[i * 5] / (double)a.P;
    if (learn && n + 1 > k) {
      const double p0hat = pk + (pk - beta) * expm1(alpha * (double)(n + 1 - k) * a.dT);
      nx.frac[0] = p0hat;
      nx.frac[1] = 1.0 - p0hat;
    }
    if (I < 2) nx.frac[0] = 1.0;
    cache[0] = av.mean[0]; cache[1] = av.var[0]; cache[2] = av.mean[1]; cache[3] = av.var[1];
    double* rr = a.rho + (size_t)(n + 1) * kMom;
    const double oldM = rr[6], oldV = rr[7];
    macro_store(a, rr, nx);
    change = fmax(change, fmax(fabs(rr[6] - oldM), fabs(rr[7] - oldV)));
    cur = nx;
  }
  if (numeric_bad || !(change < INFINITY)) atomicOr(a.status, kStatusNumeric);
  const bool conv = change < a.tol;
  ctl[0] = change;
  ctl[1] = conv ? 1.0 : 0.0;
  ctl[2] = (double)k;
  ctl[3] = (conv || k >= a.max_sweeps) ? 1.0 : 0.0;
  ctl[4] += acc;
  ctl[5] += rej;
  ctl[6] = alpha;
  ctl[7] = beta;
  ctl[8] = learn ? 1.0 : 0.0;
}

__global__ void __launch_bounds__(32) k_driver(const DriverArgs a) { driver_body(a); }

// Batched form: block b drives problem b if its sweep index is >= 0 this
// round, then copies (change, converged, sweeps, done, status) into
// summary[5 b ..].
__global__ void __launch_bounds__(32) k_driver_batch(const DriverArgs* args, const int* sweep, double* summary,
                                                     int n) {
  const int b = blockIdx.x;
  if (b >= n) return;
  const int k = sweep[b];
  if (k < 0) return;
  DriverArgs a = args[b];
  a.sweep = k;
  driver_body(a);
  __syncwarp();
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) summary[5 * b + i] = a.ctl[i];
    summary[5 * b + 4] = (double)*(volatile unsigned*)a.status;
  }
}

cudaError_t launch_driver(const DriverArgs& args, cudaStream_t stream) {
  k_driver<<<1, 32, 0, stream>>>(args);
  return cudaGetLastError();
}

cudaError_t launch_driver_batch(const DriverArgs* args, const int* sweep, double* summary, int n,
                                cudaStream_t stream) {
  if (n < 1) return cudaSuccess;
  k_driver_batch<<<n, 32, 0, stream>>>(args, sweep, summary, n);
  return cudaGetLastError();
}

}  // namespace mmp
