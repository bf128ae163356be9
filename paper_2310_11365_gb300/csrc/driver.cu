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
  double frac[kMaxRegions], mean[kMaxRegions], var[kMaxRegions];
};

__device__ void macro_zero(Macro& m) {
  for (int i = 0; i < kMaxRegions; ++i) {
    m.frac[i] = 0.0; m.mean[i] = 0.0; m.var[i] = 0.0;
  }
}

__device__ void macro_load(const double* r, Macro& m) {
  for (int i = 0; i < kMaxRegions; ++i) {
    const double* ri = r + mom_region(i);
    m.frac[i] = ri[0]; m.mean[i] = ri[1]; m.var[i] = ri[2];
  }
}

// Global (M, V) of a macro state: Eq. (mixture_of_distributions_mean_variance)
// with variances in place of the printed squares; one region is (M, V).
__device__ void mixture(const DriverArgs& a, const Macro& r, double& M, double& V) {
  if (a.I < 2) {
    M = r.mean[0];
    V = r.var[0];
    return;
  }
  double m = 0.0, s = 0.0;
  for (int i = 0; i < a.I; ++i) m += r.frac[i] * r.mean[i];
  for (int i = 0; i < a.I; ++i) s += r.frac[i] * (r.mean[i] * r.mean[i] + r.var[i]);
  M = m;
  V = s - m * m;
}

// Stores the macro state and its global (M, V) in a moment row; returns (M, V).
__device__ void macro_store(const DriverArgs& a, double* r, const Macro& m, double& M, double& V) {
  for (int i = 0; i < kMaxRegions; ++i) {
    double* ri = r + mom_region(i);
    ri[0] = m.frac[i]; ri[1] = m.mean[i]; ri[2] = m.var[i];
  }
  mixture(a, m, M, V);
  r[kMomM] = M;
  r[kMomV] = V;
  r[14] = 0.0;
  r[15] = 0.0;
}
__device__ void macro_store(const DriverArgs& a, double* r, const Macro& m) {
  double M, V;
  macro_store(a, r, m, M, V);
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
//   Taylor1: the Taylor model without the v term of the mean
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

// Plane rotator (Sec. 5, Eq. SDE_plane_rotator; one region): drift
// K (S cos x - C sin x) - g sin x with S, C the means of sin X, cos X under
// each model's own law, additive noise B0:
//   closure: X ~ N(m, v): S = sin m e^{-v/2}, C = cos m e^{-v/2};
//     m' = K (S C - C S) - g S, and by Stein's lemma
//     v' = 2 v (-K (S^2 + C^2) - g C) + B0^2;
//   Taylor (Eq. moment_model_class_1 at the point mass m: S = sin m,
//     C = cos m): m' = a(m) + a_XX(m) v / 2, v' = 2 a_X(m) v + B0^2, with
//     a_X(m) = -K - g cos m (Eq. plane_rotator_third_order with the sign of
//     its variance term as Eq. moment_model_class_1 gives it); Taylor1
//     without the v term of the mean;
//   sigma-point: the k-point rule for every expectation, S and C included.
__device__ double rotator_drift_at(const DriverArgs& a, double x, double S, double C) {
  return a.K * (S * cos(x) - C * sin(x)) - a.g * sin(x);
}

__device__ void sigma_points(int model, double m, double v, double* xs, double* ws, int& k) {
  if (model == MMP_COARSE_SIGMA2) {
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
}

__device__ void rotator_rhs(const DriverArgs& a, double m, double v, double& dm, double& dv) {
  const double b2 = a.B0 * a.B0;
  if (a.coarse_model == MMP_COARSE_TAYLOR || a.coarse_model == MMP_COARSE_TAYLOR1) {
    const double S = sin(m), C = cos(m);
    const double av = rotator_drift_at(a, m, S, C);
    const double ax = a.K * (-S * sin(m) - C * cos(m)) - a.g * cos(m);
    const double axx = a.K * (-S * cos(m) + C * sin(m)) + a.g * sin(m);
    dm = a.coarse_model == MMP_COARSE_TAYLOR ? av + 0.5 * axx * v : av;
    dv = 2.0 * ax * v + b2;
  } else if (a.coarse_model == MMP_COARSE_SIGMA2 || a.coarse_model == MMP_COARSE_SIGMA3) {
    double xs[3], ws[3];
    int k;
    sigma_points(a.coarse_model, m, v, xs, ws, k);
    double S = 0.0, C = 0.0;
    for (int s = 0; s < k; ++s) {
      S += ws[s] * sin(xs[s]);
      C += ws[s] * cos(xs[s]);
    }
    double ea = 0.0, exa = 0.0;
    for (int s = 0; s < k; ++s) {
      const double av = rotator_drift_at(a, xs[s], S, C);
      ea += ws[s] * av;
      exa += ws[s] * (xs[s] - m) * av;
    }
    dm = ea;
    dv = 2.0 * exa + b2;
  } else {
    const double e = exp(-0.5 * v);
    const double S = sin(m) * e, C = cos(m) * e;
    dm = a.K * (S * C - C * S) - a.g * S;
    dv = 2.0 * v * (-a.K * (S * S + C * C) - a.g * C) + b2;
  }
}

__device__ void coarse_rhs(const DriverArgs& a, double m, double v, double M, double& dm, double& dv) {
  if (a.family == MMP_FAMILY_ROTATOR) {
    rotator_rhs(a, m, v, dm, dv);
    return;
  }
  const double c3 = -a.nc3;
  if (a.coarse_model == MMP_COARSE_TAYLOR || a.coarse_model == MMP_COARSE_TAYLOR1) {
    const double ax = -3.0 * c3 * m * m + a.c1;
    const double axx = -6.0 * c3 * m;
    const double b = diffusion_at(a, m, M);
    dm = drift_at(a, m, M) + (a.coarse_model == MMP_COARSE_TAYLOR ? 0.5 * axx * v : 0.0);
    dv = (2.0 * ax + a.B * a.B) * v + b * b;
  } else if (a.coarse_model == MMP_COARSE_SIGMA2 || a.coarse_model == MMP_COARSE_SIGMA3) {
    double xs[3], ws[3];
    int k;
    sigma_points(a.coarse_model, m, v, xs, ws, k);
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
    if (a.I > 1) {
      M = 0.0;
      for (int i = 0; i < a.I; ++i) M += out.frac[i] * out.mean[i];
    }
    double dm[kMaxRegions], dv[kMaxRegions];
    for (int i = 0; i < a.I; ++i) coarse_rhs(a, out.mean[i], out.var[i], M, dm[i], dv[i]);
    for (int i = 0; i < a.I; ++i) {
      out.mean[i] = out.mean[i] + a.hc * dm[i];
      out.var[i] = out.var[i] + a.hc * dv[i];
    }
  }
}

// Region boundary t_i (i = 1, 2, 3).
__device__ double boundary(const DriverArgs& a, int i) { return i == 1 ? a.thr : (i == 2 ? a.thr2 : a.thr3); }

// Def. 3.2's test that matching region i = [t_i, t_{i+1}) moves no particle
// out of it: the affine map is increasing, so its smallest particle must stay
// at or above t_i and its largest below t_{i+1}.  The transform is evaluated
// exactly as the fine kernel will apply it (same precision, same rounding).
__device__ bool stays_in_region(const DriverArgs& a, int i, double lo, double hi, double delta, double sm1,
                                double m) {
  if (a.precision == MMP_MIXED) {
    bool ok = true;
    if (i > 0) ok = !(apply_affine((float)lo, (float)delta, (float)sm1, (float)m) < (float)boundary(a, i));
    if (ok && i < a.I - 1) ok = apply_affine((float)hi, (float)delta, (float)sm1, (float)m) < (float)boundary(a, i + 1);
    return ok;
  }
  bool ok = true;
  if (i > 0) ok = !(apply_affine(lo, delta, sm1, m) < boundary(a, i));
  if (ok && i < a.I - 1) ok = apply_affine(hi, delta, sm1, m) < boundary(a, i + 1);
  return ok;
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

// ---------------------------------------------------------------------------
// Learning with I >= 3 regions: the rate model of the fractions (Sec. 3.6,
// Eq. generalised_model_multimodal_PFs), dP/dt = A P with rates
// omega_ij >= 0 from D_i to D_j (A_ji = omega_ij, A_ii = -sum_j omega_ij),
// P(t_{n+1}) = Phi P(t_n), Phi = expm(A dT), fitted by least squares to the
// exact fractions of t_0..t_k (k >= I) over the box 0 <= omega <= 20 / dT
// (non-negative rates; beyond omega dT = 20 a region keeps < 2e-9 of its
// mass over a slice, so the slice-end fractions cannot tell faster rates
// apart).  Levenberg-Marquardt on omega with the bounds kept by projection:
// a rate at a bound whose gradient points out of the box is held, the
// others solve (J^T J + mu I) d = J^T r, the new point is the step clipped
// to the box; mu starts at 1e-3 max diag(J^T J) and follows the gain ratio
// rho of actual to predicted decrease (x max(1/3, 1 - (2 rho - 1)^3) after
// a success, x nu after a failure, nu doubling with every failure in a row;
// Madsen, Nielsen and Tingleff 2004, Sec. 3.2).  Converged when the
// predicted decrease is below 1e-15 of the cost, no rate is free or no
// descent is left; otherwise it stops after kRateFitMaxIter iterations or
// 60 failures in a row (the rates, of lower cost than the start, are still
// used).  Start: the one-step regression P_n ~ Phi0 P_{n-1}, omega_ij ~
// Phi0_ji / dT, floored at 1e-3 / (k dT) and capped at 1 / dT.  The
// Jacobian is the derivative of the computed expm (degree-16 Taylor
// polynomial after scaling to norm <= 1/2, then squarings) in each rate's
// direction.
//
// The whole warp runs the fit: lane p computes the directional derivative
// of expm in the direction of rate p, the derivative S_p of every modelled
// fraction, J^T r at p and row p of J^T J, each accumulated over (n, i) in
// the same order as a single pass would; lane 0 runs the sequential parts
// (costs, the damped solve, the decisions).  Everything is IEEE arithmetic
// and sqrt on working arrays in shared memory, in a fixed order, so the fit
// is reproducible bit for bit.
// ---------------------------------------------------------------------------
constexpr int kMaxRates = kMaxRegions * (kMaxRegions - 1);
constexpr int kRateFitMaxIter = 2000;
// sweep staging: slices per chunk, doubles per slice (per region count, mean,
// variance, min, max; the coarse cache; the old global M, V; the fractions)
constexpr int kDrvChunk = 64;
constexpr int kDrvRow = 8 * kMaxRegions + 2;
// the chain's record per slice: accepted flags, coarse prediction (mean,
// variance), new macro state (fraction, mean, variance), per region
constexpr int kOutAcc = 0, kOutAv = kMaxRegions, kOutNx = 3 * kMaxRegions;
constexpr int kDrvOut = 6 * kMaxRegions;

// Working arrays of an expm with its directional derivative: Y, dY, T, dT,
// W, dW, U (16 doubles each); the results are left in T and dT.
constexpr int kExpmWork = 7 * 16;
// Per-rate block: the expm work, then A, dA, the unit vector e, P, Q, S2, S3.
constexpr int kFitLane = kExpmWork + 16 + 16 + kMaxRates + 16;

struct FitShared {
  double lane[kMaxRates][kFitLane];
  double cw[kExpmWork + 16];  // lane 0's expm without derivative, then A
  double S[kMaxRates][4];     // S_p at the current slice end
  double JtJ[kMaxRates * kMaxRates];
  double g[kMaxRates];
  double M[kMaxRates * kMaxRates], L[kMaxRates * kMaxRates];
  double y[kMaxRates], x[kMaxRates], b[kMaxRates];
  double st[kMaxRates], nw[kMaxRates], om[kMaxRates];
  double cp[4], cq[4];
  double Sxx[16], Syx[16], Phi0[16], rhs[4], xr[4];
  int fidx[kMaxRates];
};

__device__ double frac_at(const DriverArgs& a, int n, int i) {
  const double* st = n == 0 ? a.stats_u0 : a.stats + (size_t)(n - 1) * kStat;
  return st[stat_region(i)] / (double)a.P;
}

__device__ void rate_generator(int I, const double* om, double* A) {
  for (int r = 0; r < I * I; ++r) A[r] = 0.0;
  for (int i = 0; i < I; ++i) {
    for (int j = 0; j < I; ++j) {
      if (j == i) continue;
      const double w = om[i * (I - 1) + (j < i ? j : j - 1)];
      A[j * I + i] += w;
      A[i * I + i] -= w;
    }
  }
}

__device__ void mat_mul(int n, const double* X, const double* Y, double* C) {
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += X[i * n + k] * Y[k * n + j];
      C[i * n + j] = s;
    }
  }
}

__device__ void mat_vec(int n, const double* M, const double* x, double* y) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += M[i * n + k] * x[k];
    y[i] = s;
  }
}

// expm(X) (n <= 4) into w + 32 and, if dX is not null, its derivative in
// the direction dX into w + 48, through the same scaling, Horner and
// squaring steps.
__device__ void expm_work(double* w, int n, const double* X, const double* dX) {
  double* Y = w;
  double* dY = w + 16;
  double* T = w + 32;
  double* dT = w + 48;
  double* W = w + 64;
  double* dW = w + 80;
  double* U = w + 96;
  double norm = 0.0;
  for (int j = 0; j < n; ++j) {
    double c = 0.0;
    for (int i = 0; i < n; ++i) c += fabs(X[i * n + j]);
    if (c > norm) norm = c;
  }
  int sq = 0;
  double scale = 1.0;
  while (norm * scale > 0.5 && sq < 60) {
    scale *= 0.5;
    ++sq;
  }
  for (int r = 0; r < n * n; ++r) {
    Y[r] = X[r] * scale;
    dY[r] = dX ? dX[r] * scale : 0.0;
    T[r] = 0.0;
    dT[r] = 0.0;
  }
  for (int i = 0; i < n; ++i) T[i * n + i] = 1.0;
  for (int m = 16; m >= 1; --m) {
    mat_mul(n, Y, T, W);
    if (dX) {
      mat_mul(n, dY, T, dW);
      mat_mul(n, Y, dT, U);
      for (int r = 0; r < n * n; ++r) dT[r] = (dW[r] + U[r]) / (double)m;
    }
    for (int r = 0; r < n * n; ++r) T[r] = W[r] / (double)m;
    for (int i = 0; i < n; ++i) T[i * n + i] += 1.0;
  }
  for (int s = 0; s < sq; ++s) {
    if (dX) {
      mat_mul(n, dT, T, dW);
      mat_mul(n, T, dT, U);
      for (int r = 0; r < n * n; ++r) dT[r] = dW[r] + U[r];
    }
    mat_mul(n, T, T, W);
    for (int r = 0; r < n * n; ++r) T[r] = W[r];
  }
}

// Phi = expm(A(omega) dT) into w + 32 (w: kExpmWork + 16 doubles).
__device__ const double* rate_phi(double* w, int I, const double* om, double dT) {
  double* A = w + kExpmWork;
  rate_generator(I, om, A);
  for (int r = 0; r < I * I; ++r) A[r] *= dT;
  expm_work(w, I, A, nullptr);
  return w + 32;
}

// One lane: the cost sum_n sum_i (fr_{n,i} - (Phi^n P_0)_i)^2 at omega.
__device__ double rate_cost(const DriverArgs& a, FitShared& F, int I, int k, const double* om) {
  const double* Phi = rate_phi(F.cw, I, om, a.dT);
  double* p = F.cp;
  double* q = F.cq;
  for (int i = 0; i < I; ++i) p[i] = frac_at(a, 0, i);
  double s = 0.0;
  for (int n = 1; n <= k; ++n) {
    mat_vec(I, Phi, p, q);
    for (int i = 0; i < I; ++i) {
      p[i] = q[i];
      const double r = frac_at(a, n, i) - p[i];
      s += r * r;
    }
  }
  return s;
}

// Whole warp: J^T J (F.JtJ) and J^T r (F.g) at omega = F.om, with
// J = d model / d omega and r = data - model.  Lane p < I (I - 1) owns rate p.
__device__ void rate_normal_warp(const DriverArgs& a, FitShared& F, int I, int k) {
  const int np = I * (I - 1);
  const int p = threadIdx.x & 31;
  const bool own = p < np;
  double* w = F.lane[own ? p : 0];
  double* A = w + kExpmWork;
  double* dA = A + 16;
  double* e = dA + 16;
  double* P = e + kMaxRates;
  double* Q = P + 4;
  double* S2 = Q + 4;
  double* S3 = S2 + 4;
  const double* Phi = w + 32;
  const double* dPhi = w + 48;
  __syncwarp();
  if (own) {
    rate_generator(I, F.om, A);
    for (int r = 0; r < I * I; ++r) A[r] *= a.dT;
    for (int q = 0; q < kMaxRates; ++q) e[q] = 0.0;
    e[p] = 1.0;
    rate_generator(I, e, dA);
    for (int r = 0; r < I * I; ++r) dA[r] *= a.dT;
    expm_work(w, I, A, dA);
    for (int q = 0; q < np; ++q) F.JtJ[p * np + q] = 0.0;
    F.g[p] = 0.0;
    for (int i = 0; i < I; ++i) {
      P[i] = frac_at(a, 0, i);
      F.S[p][i] = 0.0;
    }
  }
  for (int n = 1; n <= k; ++n) {
    if (own) {
      // S_p <- dPhi_p P + Phi S_p (the derivative of P_n), then P <- Phi P
      mat_vec(I, dPhi, P, S2);
      mat_vec(I, Phi, F.S[p], S3);
      for (int i = 0; i < I; ++i) F.S[p][i] = S2[i] + S3[i];
      mat_vec(I, Phi, P, Q);
      for (int i = 0; i < I; ++i) P[i] = Q[i];
    }
    __syncwarp();
    if (own) {
      for (int i = 0; i < I; ++i) {
        const double r = frac_at(a, n, i) - P[i];
        const double sp = F.S[p][i];
        F.g[p] += sp * r;
        for (int q = 0; q < np; ++q) F.JtJ[p * np + q] += sp * F.S[q][i];
      }
    }
    __syncwarp();
  }
}

// M x = b for symmetric positive definite M (Cholesky, factor in Lf); false if not SPD
__device__ bool spd_solve(double* Lf, double* y, int n, const double* M, const double* b, double* x) {
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = M[i * n + j];
      for (int k = 0; k < j; ++k) s -= Lf[i * n + k] * Lf[j * n + k];
      if (i == j) {
        if (!(s > 0.0) || !isfinite(s)) return false;
        Lf[i * n + i] = sqrt(s);
      } else {
        Lf[i * n + j] = s / Lf[j * n + j];
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= Lf[i * n + k] * y[k];
    y[i] = s / Lf[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < n; ++k) s -= Lf[k * n + i] * x[k];
    x[i] = s / Lf[i * n + i];
  }
  return true;
}

// One lane: the damped step on the free rates (F.st) and its predicted
// decrease; returns the number of free rates, or -1 if the system is not SPD.
__device__ int rate_free_step(FitShared& F, int np, double om_max, double mu, double& pred) {
  int nf = 0;
  for (int p = 0; p < np; ++p) {
    F.st[p] = 0.0;
    const bool held = (F.om[p] == 0.0 && !(F.g[p] > 0.0)) || (F.om[p] == om_max && !(F.g[p] < 0.0));
    if (!held) F.fidx[nf++] = p;
  }
  pred = 0.0;
  if (nf == 0) return 0;
  for (int r = 0; r < nf; ++r) {
    for (int c = 0; c < nf; ++c) F.M[r * nf + c] = F.JtJ[F.fidx[r] * np + F.fidx[c]];
    F.M[r * nf + r] = F.M[r * nf + r] + mu;
    F.b[r] = F.g[F.fidx[r]];
  }
  if (!spd_solve(F.L, F.y, nf, F.M, F.b, F.x)) return -1;
  double s = 0.0;
  for (int r = 0; r < nf; ++r) {
    F.st[F.fidx[r]] = F.x[r];
    s += F.x[r] * (mu * F.x[r] + F.b[r]);
  }
  pred = s;
  return nf;
}

// Whole warp.  Returns 0 (converged), 1 (stopped; rates still used), -1 (k < I)
// or -2 (a rate not finite); the rates are left in F.om.
__device__ int rate_fit(const DriverArgs& a, FitShared& F, int I, int k) {
  const int np = I * (I - 1);
  const int lane = threadIdx.x & 31;
  if (I < 2 || I > kMaxRegions || k < I) return -1;
  const double dT = a.dT;
  const double floor_rate = 1e-3 / ((double)k * dT);
  const double om_max = 20.0 / dT;
  double cost = 0.0, mu = 0.0, nu = 2.0;
  if (lane == 0) {
    for (int r = 0; r < 16; ++r) {
      F.Sxx[r] = 0.0;
      F.Syx[r] = 0.0;
    }
    for (int n = 1; n <= k; ++n)
      for (int p = 0; p < I; ++p)
        for (int q = 0; q < I; ++q) {
          F.Sxx[p * I + q] += frac_at(a, n - 1, p) * frac_at(a, n - 1, q);
          F.Syx[p * I + q] += frac_at(a, n, p) * frac_at(a, n - 1, q);
        }
    bool ok = true;
    for (int p = 0; p < I && ok; ++p) {
      for (int q = 0; q < I; ++q) F.rhs[q] = F.Syx[p * I + q];
      if (!spd_solve(F.L, F.y, I, F.Sxx, F.rhs, F.xr)) {
        ok = false;
      } else {
        for (int q = 0; q < I; ++q) F.Phi0[p * I + q] = F.xr[q];
      }
    }
    for (int i = 0; i < I; ++i)
      for (int j = 0; j < I; ++j) {
        if (j == i) continue;
        const double w = ok ? F.Phi0[j * I + i] / dT : 1.0 / ((double)I * (double)k * dT);
        F.om[i * (I - 1) + (j < i ? j : j - 1)] = isfinite(w) && w > floor_rate ? fmin(w, 1.0 / dT) : floor_rate;
      }
    cost = rate_cost(a, F, I, k, F.om);
  }
  rate_normal_warp(a, F, I, k);
  if (lane == 0) {
    for (int p = 0; p < np; ++p) mu = fmax(mu, F.JtJ[p * np + p]);
    mu = 1e-3 * mu;
  }
  // lane 0 decides; 0 = go on, 1 = accepted (new J^T J needed), 2 = converged, 3 = stopped
  int state = __shfl_sync(0xffffffffu, cost == 0.0 ? 2 : 0, 0);
  for (int it = 0; it < kRateFitMaxIter && state < 2; ++it) {
    int act = 0;
    if (lane == 0) {
      double pred;
      const int nf = rate_free_step(F, np, om_max, mu, pred);
      if (nf == 0) {
        act = 2;  // every rate held at a bound: a stationary point
      } else {
        double ncost = 0.0;
        if (nf > 0) {
          for (int p = 0; p < np; ++p) F.nw[p] = fmin(fmax(F.om[p] + F.st[p], 0.0), om_max);
          ncost = rate_cost(a, F, I, k, F.nw);
        }
        if (nf > 0 && pred > 0.0 && isfinite(ncost) && ncost < cost) {
          const double rho = (cost - ncost) / pred;
          const double t = 2.0 * rho - 1.0;
          for (int p = 0; p < np; ++p) F.om[p] = F.nw[p];
          cost = ncost;
          mu = mu * fmax(1.0 / 3.0, 1.0 - t * t * t);
          nu = 2.0;
          act = (pred < 1e-15 * cost || cost == 0.0) ? 2 : 1;
        } else if (nf > 0 && !(pred > 0.0)) {
          act = 2;  // no descent left on the free rates
        } else {
          mu = mu * nu;
          nu = 2.0 * nu;
          act = nu > 1e18 ? 3 : 0;
        }
      }
    }
    act = __shfl_sync(0xffffffffu, act, 0);
    if (act == 1) rate_normal_warp(a, F, I, k);
    if (act >= 2) state = act;
  }
  __syncwarp();
  int rc = state == 2 ? 0 : 1;
  if (lane == 0) {
    for (int p = 0; p < np; ++p)
      if (!isfinite(F.om[p]) || !(F.om[p] >= 0.0)) rc = -2;
  }
  return __shfl_sync(0xffffffffu, rc, 0);
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
    macro_zero(r);
    for (int i = 0; i < I; ++i) {
      const double* si = s0 + stat_region(i);
      r.frac[i] = si[0] / (double)a.P; r.mean[i] = si[1]; r.var[i] = si[2];
    }
    macro_store(a, a.rho, r);
    for (int n = 0; n <= N; ++n) {
      double* af = a.aff + (size_t)n * kMaxRegions * kAff;
      for (int i = 0; i < kMaxRegions; ++i) {
        if (i < I) {
          const double* si = s0 + stat_region(i);
          matching_record(af + i * kAff, si[0], si[1], si[2], r.mean[i], r.var[i]);
        } else {
          set_aff(af + i * kAff, kMatchIdentity, 0.0, 0.0, 0.0);
        }
      }
      if (n == N) break;
      Macro nx;
      coarse(a, r, nx);
      double* c = a.cache + (size_t)n * 2 * kMaxRegions;
      for (int i = 0; i < kMaxRegions; ++i) {
        c[2 * i] = nx.mean[i];
        c[2 * i + 1] = nx.var[i];
      }
      macro_store(a, a.rho + (size_t)(n + 1) * kMom, nx);
      r = nx;
    }
    ctl[0] = 0.0;  // last change
    ctl[1] = 0.0;  // converged
    ctl[2] = 0.0;  // sweeps
    ctl[3] = 0.0;  // done
    ctl[4] = 0.0;  // accepted
    ctl[5] = 0.0;  // rejected
    ctl[6] = 0.0;  // fit alpha (two regions)
    ctl[7] = 0.0;  // fit beta (two regions)
    ctl[8] = 0.0;  // fit used
    ctl[15] = 0.0;  // copy of the status word after a sweep
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
  // The sweep over a chunk of kDrvChunk slices runs in three phases:
  //   stage (all lanes): the slices' restriction records, coarse cache, old
  //     global moments and fractions (count / P, or the learned two-region
  //     fractions) into shared memory;
  //   chain (lane 0): slice by slice, only what the next slice depends on:
  //     the coarse step, alpha = R(b) + (a - c), acceptance and the new
  //     macro state, recorded per slice;
  //   finish (one lane per slice): matching records, coarse cache, moment
  //     rows with the mixture, and the change, reduced by max over lanes.
  // Each value is the same expression as in a single sequential pass, so
  // the results are the same bit for bit; the FP64 instructions (slow on this
  // chip) off the chain no longer wait for it.
  // The staging arrays double as the rate fit's working memory: the fit
  // ends before the staging starts.
  __shared__ __align__(16) double s_work[kDrvChunk * (kDrvRow + kDrvOut)];
  static_assert(sizeof(FitShared) <= sizeof(s_work), "fit working memory");
  double* s_stage = s_work;
  double* s_out = s_work + kDrvChunk * kDrvRow;
  Macro cur;
  double Phi[16];
  double phat[kMaxRegions];  // extrapolated fractions (I >= 3), from those of t_k
  double change = 0.0;
  int acc = 0, rej = 0;
  bool numeric_bad = false;
  if (a.variant == MMP_LEARNING && I >= 3 && k >= I) {
    // the whole warp fits; lane 0 keeps Phi = expm(A dT) of the fitted rates
    FitShared& F = *reinterpret_cast<FitShared*>(s_work);
    learn = rate_fit(a, F, I, k) >= 0;
    if (learn && lane == 0) {
      const double* ph = rate_phi(F.cw, I, F.om, a.dT);
      for (int r = 0; r < I * I; ++r) Phi[r] = ph[r];
    }
    __syncwarp();
  }
  if (lane == 0) {
    for (int i = 0; i < I; ++i) phat[i] = frac_at(a, k, i);
    macro_load(a.rho, cur);  // rho^{k}_0 = R(u0), unchanged
  }
  const bool learn2 = learn && I == 2;  // known to every lane (the two-region fit is warp-wide)
  const double pk = frac0_at(a, k);
  for (int c0 = 0; c0 < N; c0 += kDrvChunk) {
    const int cn = min(kDrvChunk, N - c0);
    __syncwarp();
    for (int idx = lane; idx < cn * kDrvRow; idx += 32) {
      const int n = c0 + idx / kDrvRow;
      const int f = idx % kDrvRow;
      double v;
      if (f < 5 * kMaxRegions) {
        v = a.stats[(size_t)n * kStat + stat_region(f / 5) + f % 5];
      } else if (f < 7 * kMaxRegions) {
        v = a.cache[(size_t)n * 2 * kMaxRegions + (f - 5 * kMaxRegions)];
      } else if (f < 7 * kMaxRegions + 2) {
        v = a.rho[(size_t)(n + 1) * kMom + (f == 7 * kMaxRegions ? kMomM : kMomV)];
      } else {
        // fractions of slice end n + 1: from the fine propagator (Def. 3.2), or
        // learned beyond the exact slices (Def. 3.4, two regions)
        const int i = f - (7 * kMaxRegions + 2);
        v = a.stats[(size_t)n * kStat + stat_region(i)] / (double)a.P;
        if (learn2 && n + 1 > k && i < 2) {
          const double p0hat = pk + (pk - beta) * expm1(alpha * (double)(n + 1 - k) * a.dT);
          v = i == 0 ? p0hat : 1.0 - p0hat;
        }
      }
      s_stage[idx] = v;
    }
    __syncwarp();
    if (lane == 0) {
      for (int n = c0; n < c0 + cn; ++n) {
        const double* row = s_stage + (size_t)(n - c0) * kDrvRow;
        const double* cache_old = row + 5 * kMaxRegions;
        const double* frac = row + 7 * kMaxRegions + 2;
        double* out = s_out + (size_t)(n - c0) * kDrvOut;
        Macro av;
        coarse(a, cur, av);
        Macro nx;
        macro_zero(nx);
        for (int i = 0; i < I; ++i) {
          const double* bi = row + 5 * i;
          const double cnt = bi[0], bm = bi[1], bv = bi[2];
          const double bmin = bi[3], bmax = bi[4];
          out[kOutAcc + i] = 0.0;
          if (!(fabs(bm) < INFINITY) || !(bv < INFINITY)) numeric_bad = true;
          if (cnt <= 0.0) {
            // empty region: carry the coarse prediction, move nothing
            nx.mean[i] = av.mean[i];
            nx.var[i] = av.var[i];
            continue;
          }
          // alpha = R(b) + (a - c): a == c returns R(b) exactly (Property 3.3)
          const double am = bm + (av.mean[i] - cache_old[2 * i]);
          const double avv = bv + (av.var[i] - cache_old[2 * i + 1]);
          bool accept = avv >= 0.0;
          if (accept && a.variant != MMP_UNIMODAL && I > 1) {
            // Def. 3.2: move a region only if no particle leaves it
            if (bv == 0.0) {
              accept = false;
            } else {
              const double delta = am - bm;
              const double sm1 = sqrt(avv / bv) - 1.0;
              accept = stays_in_region(a, i, bmin, bmax, delta, sm1, bm);
            }
          }
          if (accept) {
            nx.mean[i] = am;
            nx.var[i] = avv;
            out[kOutAcc + i] = 1.0;
            ++acc;
          } else {
            nx.mean[i] = bm;
            nx.var[i] = bv;
            ++rej;
          }
        }
        for (int i = 0; i < I; ++i) nx.frac[i] = frac[i];
        if (learn && I >= 3 && n + 1 > k) {
          double q[kMaxRegions];
          mat_vec(I, Phi, phat, q);
          for (int i = 0; i < I; ++i) {
            phat[i] = q[i];
            nx.frac[i] = q[i];
          }
        }
        if (I < 2) nx.frac[0] = 1.0;
        for (int i = 0; i < kMaxRegions; ++i) {
          out[kOutAv + 2 * i] = av.mean[i];
          out[kOutAv + 2 * i + 1] = av.var[i];
          out[kOutNx + 3 * i] = nx.frac[i];
          out[kOutNx + 3 * i + 1] = nx.mean[i];
          out[kOutNx + 3 * i + 2] = nx.var[i];
        }
        cur = nx;
      }
    }
    __syncwarp();
    for (int j = lane; j < cn; j += 32) {
      const int n = c0 + j;
      const double* row = s_stage + (size_t)j * kDrvRow;
      const double* out = s_out + (size_t)j * kDrvOut;
      double* af = a.aff + (size_t)(n + 1) * kMaxRegions * kAff;
      for (int i = 0; i < kMaxRegions; ++i) {
        if (i < I && out[kOutAcc + i] != 0.0) {
          const double* bi = row + 5 * i;
          matching_record(af + i * kAff, bi[0], bi[1], bi[2], out[kOutNx + 3 * i + 1], out[kOutNx + 3 * i + 2]);
        } else {
          set_aff(af + i * kAff, kMatchIdentity, 0.0, 0.0, 0.0);
        }
      }
      double* cache = a.cache + (size_t)n * 2 * kMaxRegions;
      Macro nx;
      for (int i = 0; i < kMaxRegions; ++i) {
        cache[2 * i] = out[kOutAv + 2 * i];
        cache[2 * i + 1] = out[kOutAv + 2 * i + 1];
        nx.frac[i] = out[kOutNx + 3 * i];
        nx.mean[i] = out[kOutNx + 3 * i + 1];
        nx.var[i] = out[kOutNx + 3 * i + 2];
      }
      const double oldM = row[7 * kMaxRegions], oldV = row[7 * kMaxRegions + 1];
      double M, V;
      macro_store(a, a.rho + (size_t)(n + 1) * kMom, nx, M, V);
      change = fmax(change, fmax(fabs(M - oldM), fabs(V - oldV)));
    }
  }
  // the change is a maximum over slices: any order gives the same value
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) change = fmax(change, __shfl_xor_sync(0xffffffffu, change, off));
  if (lane != 0) return;
  if (numeric_bad || !(change < INFINITY)) atomicOr(a.status, kStatusNumeric);
  ctl[15] = (double)*(volatile unsigned*)a.status;  // the status word, for one read of ctl by the host
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
