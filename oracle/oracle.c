/*
 * oracle.c -- plain FP64 CPU oracle for MC-moments micro-macro Parareal
 * (arXiv 2310.11365).  TEST INFRASTRUCTURE ONLY: see oracle.h.
 *
 * Each function names the part of the paper it restates.  Readings of
 * places where the paper is silent or garbled are marked "reading:".
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * Philox-4x32-10, from its published definition (Salmon et al., SC'11,
 * "Parallel random numbers: as easy as 1, 2, 3"): ten rounds of the
 * 4x32 S-box with multipliers M0, M1 and the key bumped by the Weyl
 * constants W0, W1 between rounds.
 * ---------------------------------------------------------------------- */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* u = ((o >> 9) + 1/2) 2^-23, strictly inside (0, 1). */
double orc_uniform(uint32_t word) {
  return ((double)(word >> 9) + 0.5) * ldexp(1.0, -23);
}

/* Box-Muller on two uniforms. */
static void box_muller(double ua, double ub, double* z0, double* z1) {
  const double two_pi = 6.283185307179586476925286766559;
  double r = sqrt(-2.0 * log(ua));
  *z0 = r * cos(two_pi * ub);
  *z1 = r * sin(two_pi * ub);
}

/* The four normals of one Philox call, for particles 4q .. 4q+3. */
static void normals4(const orc_problem* pr, int tag, uint32_t j, uint32_t n, uint32_t q, double z[4]) {
  uint32_t key[2] = {(uint32_t)(pr->seed & 0xffffffffu), (uint32_t)(pr->seed >> 32)};
  uint32_t ctr[4] = {q, j, n | ((uint32_t)tag << 24), pr->problem_tag};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  box_muller(orc_uniform(o[0]), orc_uniform(o[1]), &z[0], &z[1]);
  box_muller(orc_uniform(o[2]), orc_uniform(o[3]), &z[2], &z[3]);
}

double orc_normal(const orc_problem* pr, int tag, uint32_t j, uint32_t n, long long p) {
  double z[4];
  normals4(pr, tag, j, n, (uint32_t)(p / 4), z);
  return z[p % 4];
}

/* The plane rotator's shift modulo 2 pi (Sec. 5, Example "Unimodal plane
 * rotator": applied to every particle in each time step).
 * reading: the interval is [-pi, pi], not the printed [0, 2 pi].  The printed
 * drift -sin x has its stable point at 0 = 2 pi, the end of [0, 2 pi], so an
 * ensemble shifted there piles up at both ends (mean near pi, variance near
 * pi^2) instead of being the unimodal distribution the example describes;
 * centred on the stable point it is unimodal and the iteration reaches the
 * statistical error in a few sweeps, as the example reports.
 * reading: the initial ensemble is shifted as well, so that every slice end,
 * t_0 included, holds particles in [-pi, pi]. */
static const double PI = 3.141592653589793238462643383280;
static const double TWO_PI = 6.283185307179586476925286766559;

double orc_wrap(double x) {
  return x - TWO_PI * floor((x + PI) / TWO_PI);
}

void orc_initial(const orc_problem* pr, double* u0) {
  for (long long p = 0; p < pr->P; ++p) {
    u0[p] = pr->m0 + pr->s0 * orc_normal(pr, 1, 0, 0, p);
    if (pr->family == ORC_FAMILY_ROTATOR) u0[p] = orc_wrap(u0[p]);
  }
}

/* ------------------------------------------------------------------------
 * Fine propagator F_n: Euler-Maruyama for the particle system, Sec. 1.2
 * Eq. (Euler_Maruyama), Ito (Sec. 1.1).
 * reading: the printed scheme drops the "X_n +" term; the update is
 *   X_{j+1} = X_j + a(X_j, m_j) h + b(X_j, m_j) sqrt(h) xi_j
 * with m_j the mean of the ensemble before the step.
 * reading: the slice length T/N need not be a multiple of dt; the slice is
 * cut into n_f = ceil(T/(N dt) - 1e-9) equal steps h = T/(N n_f).
 * ---------------------------------------------------------------------- */
int orc_fine_steps(const orc_problem* pr) {
  double dT = pr->T / pr->N;
  int nf = (int)ceil(dT / pr->dt - 1e-9);
  return nf < 1 ? 1 : nf;
}

double orc_fine_h(const orc_problem* pr) {
  return (pr->T / pr->N) / orc_fine_steps(pr);
}

/* a(x, m, s) with s = E[X^2]; the term -q2 x s is the second-moment
 * coupling of the polynomial-drift example (App. C), zero elsewhere */
static double drift(const orc_problem* pr, double x, double m, double s) {
  return -pr->c3 * x * x * x + (pr->c1 - pr->q2 * s) * x + pr->kappa * m + pr->c0;
}

static double diffusion(const orc_problem* pr, double x, double m) {
  return pr->B * x + pr->BE * m + pr->B0;
}

static double ensemble_mean(const double* u, long long P) {
  double s = 0.0;
  for (long long p = 0; p < P; ++p) s += u[p];
  return s / (double)P;
}

/* E[X^2] of the ensemble (the second raw moment) */
static double ensemble_second_moment(const double* u, long long P) {
  double s = 0.0;
  for (long long p = 0; p < P; ++p) s += u[p] * u[p];
  return s / (double)P;
}

/* Plane rotator: (K/P) sum_q sin(X_q - x) = K (S cos x - C sin x) by the
 * difference formula for the sine, with S, C the ensemble means of sin X and
 * cos X; the pinning term -g sin x. */
static double rotator_drift(const orc_problem* pr, double x, double S, double C) {
  return pr->K * (S * cos(x) - C * sin(x)) - pr->g * sin(x);
}

static void ensemble_sin_cos(const double* u, long long P, double* S, double* C) {
  double s = 0.0, c = 0.0;
  for (long long p = 0; p < P; ++p) {
    s += sin(u[p]);
    c += cos(u[p]);
  }
  *S = s / (double)P;
  *C = c / (double)P;
}

void orc_fine(const orc_problem* pr, int n, const double* u_in, double* u_out, double* means) {
  const long long P = pr->P;
  const int nf = orc_fine_steps(pr);
  const double h = orc_fine_h(pr);
  const double sqrt_h = sqrt(h);
  double* x = (double*)malloc(sizeof(double) * (size_t)P);
  double* y = (double*)malloc(sizeof(double) * (size_t)P);
  memcpy(x, u_in, sizeof(double) * (size_t)P);
  const int rotator = pr->family == ORC_FAMILY_ROTATOR;
  for (int j = 0; j < nf; ++j) {
    double m = ensemble_mean(x, P);
    if (means) means[j] = m;
    double S = 0.0, C = 0.0;
    if (rotator) ensemble_sin_cos(x, P, &S, &C);
    const double s2 = pr->q2 != 0.0 ? ensemble_second_moment(x, P) : 0.0;
    for (long long q = 0; 4 * q < P; ++q) {
      double z[4];
      normals4(pr, 0, (uint32_t)j, (uint32_t)n, (uint32_t)q, z);
      for (int w = 0; w < 4 && 4 * q + w < P; ++w) {
        long long p = 4 * q + w;
        if (rotator) {
          y[p] = orc_wrap(x[p] + rotator_drift(pr, x[p], S, C) * h + pr->B0 * sqrt_h * z[w]);
        } else {
          y[p] = x[p] + drift(pr, x[p], m, s2) * h + diffusion(pr, x[p], m) * sqrt_h * z[w];
        }
      }
    }
    double* t = x; x = y; y = t;
  }
  if (means) means[nf] = ensemble_mean(x, P);
  memcpy(u_out, x, sizeof(double) * (size_t)P);
  free(x);
  free(y);
}

/* ------------------------------------------------------------------------
 * Restriction.  Unimodal: S(u) = [E u, V u] (Sec. 3.4).  Multimodal:
 * Eq. (multimodal_R), per region D_i the fraction, mean and variance.
 * reading: variances are population variances (1/n_i), which makes the
 * mixture identity exact and keeps Lemma 3.1.
 * reading: the regions are consecutive intervals of the real line split at
 * t_1 < t_2 < t_3: D_0 = {x < t_1}, D_i = {t_i <= x < t_{i+1}} and
 * D_{I-1} = {x >= t_{I-1}}; with I = 2 this is D_0 = {x < thr}, D_1 = {x >= thr}.
 * ---------------------------------------------------------------------- */
int orc_region(const orc_problem* pr, double x) {
  const int I = pr->n_regions;
  if (I < 2 || x < pr->threshold) return 0;
  if (I < 3 || x < pr->threshold2) return 1;
  if (I < 4 || x < pr->threshold3) return 2;
  return 3;
}

/* lower boundary t_i of region i >= 1 */
static double region_lower(const orc_problem* pr, int i) {
  return i == 1 ? pr->threshold : (i == 2 ? pr->threshold2 : pr->threshold3);
}

void orc_restrict(const orc_problem* pr, const double* u, orc_stats* st) {
  const long long P = pr->P;
  memset(st, 0, sizeof(*st));
  double sum[ORC_MAX_REGIONS] = {0};
  for (int i = 0; i < ORC_MAX_REGIONS; ++i) {
    st->min[i] = INFINITY;
    st->max[i] = -INFINITY;
  }
  for (long long p = 0; p < P; ++p) {
    int i = orc_region(pr, u[p]);
    st->count[i] += 1;
    sum[i] += u[p];
    if (u[p] < st->min[i]) st->min[i] = u[p];
    if (u[p] > st->max[i]) st->max[i] = u[p];
  }
  for (int i = 0; i < ORC_MAX_REGIONS; ++i)
    st->mean[i] = st->count[i] > 0 ? sum[i] / (double)st->count[i] : 0.0;
  double ss[ORC_MAX_REGIONS] = {0};
  for (long long p = 0; p < P; ++p) {
    int i = orc_region(pr, u[p]);
    double d = u[p] - st->mean[i];
    ss[i] += d * d;
  }
  for (int i = 0; i < ORC_MAX_REGIONS; ++i)
    st->var[i] = st->count[i] > 0 ? ss[i] / (double)st->count[i] : 0.0;
  st->gmean = ensemble_mean(u, P);
  double g = 0.0;
  for (long long p = 0; p < P; ++p) g += (u[p] - st->gmean) * (u[p] - st->gmean);
  st->gvar = g / (double)P;
}

/* Global mean and variance of a macro state, Sec. 2.2
 * Eq. (mixture_of_distributions_mean_variance).
 * reading: the printed Sigma^2, Sigma_i^2 are variances:
 *   M = sum_i P_i M_i,  V = sum_i P_i (M_i^2 + V_i) - M^2.
 * With one region the state is (M, V) itself. */
void orc_mixture(const orc_problem* pr, const orc_macro* r, double* M, double* V) {
  if (pr->n_regions < 2) {
    *M = r->mean[0];
    *V = r->var[0];
    return;
  }
  double m = 0.0, s = 0.0;
  for (int i = 0; i < pr->n_regions; ++i) m += r->frac[i] * r->mean[i];
  for (int i = 0; i < pr->n_regions; ++i) s += r->frac[i] * (r->mean[i] * r->mean[i] + r->var[i]);
  *M = m;
  *V = s - m * m;
}

/* Matching T([mu, sigma], u), Sec. 3.4 Eq. (multimodal_M), applied to the
 * particles of each selected region.
 * reading: the affine branch is evaluated as
 *   x + (mu - E u) + (sqrt(sigma / V u) - 1)(x - E u),
 * algebraically the printed sqrt(sigma/V u)(x - E u) + mu, but the identity
 * T(S u, u) = u (Lemma 3.1) then holds bit for bit.
 * reading: the redraw branch (V u = 0) uses tag-2 draws with j = region and
 * n = target slice, so it repeats in every iteration. */
void orc_match(const orc_problem* pr, int n, const double* mu, const double* sigma,
               const int* do_region, const orc_stats* st_u, const double* u, double* u_out) {
  const long long P = pr->P;
  for (long long p = 0; p < P; ++p) {
    int i = orc_region(pr, u[p]);
    double x = u[p];
    if (do_region[i]) {
      double m = st_u->mean[i];
      double v = st_u->var[i];
      if (v == 0.0) {
        x = mu[i] + sqrt(sigma[i]) * orc_normal(pr, 2, (uint32_t)i, (uint32_t)n, p);
      } else {
        double s = sqrt(sigma[i] / v);
        x = x + (mu[i] - m) + (s - 1.0) * (x - m);
      }
    }
    u_out[p] = x;
  }
}

/* ------------------------------------------------------------------------
 * Coarse propagator C_n: moment ODE per region, Sec. 2.1-2.2.
 * reading: the printed variance equations (2 E[a] + E[b^2], and the
 * Gaussian model's "2 int a p + int b p") drop the centring and the square;
 * by Ito, dV/dt = 2 E[(X - M) a] + E[b^2].  Under the Gaussian assumption of
 * Eq. (Gaussian_model_McK_V_SDE) with polynomial drift the integrals are
 * closed-form: E[X^3] = m^3 + 3 m v and Cov(X, X^3) = 3 v (m^2 + v), so per
 * region i, with the mean field M = sum_j P_j m_j held by the frozen
 * fractions (Def. 3.2: the coarse propagator does not move P_i):
 *   dm_i/dt = -c3 (m_i^3 + 3 m_i v_i) + c1 m_i + kappa M + c0
 *   dv_i/dt = 2 (-3 c3 v_i (m_i^2 + v_i) + c1 v_i) + B^2 v_i + (B m_i + BE M + B0)^2
 * For c3 = 0 this is the Taylor model of Eq. (moment_model_class_1), exact
 * for linear SDEs (Lemma 2.1).
 * reading: the paper integrates with adaptive Tsit5; here forward Euler
 * with n_c = ceil(T/(N coarse_h) - 1e-9) equal substeps.
 * ---------------------------------------------------------------------- */
int orc_coarse_steps(const orc_problem* pr) {
  double dT = pr->T / pr->N;
  int nc = (int)ceil(dT / pr->coarse_h - 1e-9);
  return nc < 1 ? 1 : nc;
}

/* Right-hand side of the coarse moment ODE of each region i, the mean field
 * M being the mixture mean (the region's own mean when I = 1).
 *   closure: dm = E[a], dv = 2 Cov(X, a) + E[b^2] under N(m, v), in closed
 *            form for the cubic drift (E X^3 = m^3 + 3 m v,
 *            Cov(X, X^3) = 3 v (m^2 + v));
 *   Taylor:  dm = a(m) + a_XX(m) v / 2, dv = (2 a_X(m) + b_X^2) v + b(m)^2
 *            (Eq. moment_model_class_1; the same model without its Sigma^2
 *            term for this drift);
 *   Taylor1: the Taylor model without its Sigma term in the mean,
 *            dm = a(m);
 *   sigma-point: the expectations of Eq. Gaussian_model_McK_V_SDE by a
 *            k-point rule on N(m, v): k = 2: m -+ sqrt(v), weights 1/2;
 *            k = 3: m, m -+ sqrt(3 v), weights 2/3, 1/6, 1/6. */
static void sigma_points(int model, double m, double v, double* xs, double* ws, int* k) {
  if (model == ORC_COARSE_SIGMA2) {
    double d = sqrt(v > 0.0 ? v : 0.0);
    xs[0] = m - d; xs[1] = m + d;
    ws[0] = 0.5; ws[1] = 0.5;
    *k = 2;
  } else {
    double d = sqrt(3.0 * (v > 0.0 ? v : 0.0));
    xs[0] = m; xs[1] = m - d; xs[2] = m + d;
    ws[0] = 2.0 / 3.0; ws[1] = 1.0 / 6.0; ws[2] = 1.0 / 6.0;
    *k = 3;
  }
}

/* Coarse moment ODE of the plane rotator (one region), the mean-field means
 * S = E[sin X], C = E[cos X] taken under each model's own law:
 *   closure: X ~ N(m, v): E sin X = sin m e^{-v/2}, E cos X = cos m e^{-v/2};
 *            dm = E[a] = K (S C - C S) - g S, and by Stein's lemma
 *            E[(X - m) f(X)] = v E[f'(X)]:
 *            dv = 2 v E[a_X] + B0^2 = 2 v (-K (S^2 + C^2) - g C) + B0^2;
 *   Taylor:  the point mass at m (S = sin m, C = cos m) and the derivatives
 *            of a at m: dm = a(m) + a_XX(m) v / 2 = -g sin m + g sin m v / 2,
 *            dv = 2 a_X(m) v + B0^2 = 2 (-K - g cos m) v + B0^2, which is
 *            Eq. plane_rotator_third_order for g = 1;
 *            reading: that equation's variance line prints
 *            -2 (-K - cos M) Sigma, a growing variance; Eq.
 *            moment_model_class_1 gives +2 a_X Sigma with a_X = -K - cos M;
 *   Taylor1: the same without the Sigma term of the mean (the paper's first
 *            coarse solver of this example);
 *   sigma-point: the k-point rule for every expectation, S and C included. */
static void rotator_rhs(const orc_problem* pr, double m, double v, double* dm, double* dv) {
  const double b2 = pr->B0 * pr->B0;
  if (pr->coarse_model == ORC_COARSE_TAYLOR || pr->coarse_model == ORC_COARSE_TAYLOR1) {
    const double S = sin(m), C = cos(m);
    const double a = rotator_drift(pr, m, S, C);
    const double ax = pr->K * (-S * sin(m) - C * cos(m)) - pr->g * cos(m);
    const double axx = pr->K * (-S * cos(m) + C * sin(m)) + pr->g * sin(m);
    *dm = pr->coarse_model == ORC_COARSE_TAYLOR ? a + 0.5 * axx * v : a;
    *dv = 2.0 * ax * v + b2;
  } else if (pr->coarse_model == ORC_COARSE_SIGMA2 || pr->coarse_model == ORC_COARSE_SIGMA3) {
    double xs[3], ws[3];
    int k;
    sigma_points(pr->coarse_model, m, v, xs, ws, &k);
    double S = 0.0, C = 0.0;
    for (int s = 0; s < k; ++s) {
      S += ws[s] * sin(xs[s]);
      C += ws[s] * cos(xs[s]);
    }
    double ea = 0.0, exa = 0.0;
    for (int s = 0; s < k; ++s) {
      const double a = rotator_drift(pr, xs[s], S, C);
      ea += ws[s] * a;
      exa += ws[s] * (xs[s] - m) * a;
    }
    *dm = ea;
    *dv = 2.0 * exa + b2;
  } else {
    const double e = exp(-0.5 * v);
    const double S = sin(m) * e, C = cos(m) * e;
    *dm = pr->K * (S * C - C * S) - pr->g * S;
    *dv = 2.0 * v * (-pr->K * (S * S + C * C) - pr->g * C) + b2;
  }
}

void orc_coarse_rhs(const orc_problem* pr, const orc_macro* r, double* dm, double* dv) {
  if (pr->family == ORC_FAMILY_ROTATOR) {
    rotator_rhs(pr, r->mean[0], r->var[0], &dm[0], &dv[0]);
    return;
  }
  const int I = pr->n_regions < 2 ? 1 : pr->n_regions;
  /* the mean field: the mixture mean M, and (second-moment coupling only)
   * the mixture second moment S2 = sum_i P_i (M_i^2 + Sigma_i) */
  double M = 0.0, S2 = 0.0;
  if (I == 1) {
    M = r->mean[0];
    S2 = r->mean[0] * r->mean[0] + r->var[0];
  } else {
    for (int i = 0; i < I; ++i) {
      M += r->frac[i] * r->mean[i];
      S2 += r->frac[i] * (r->mean[i] * r->mean[i] + r->var[i]);
    }
  }
  if (pr->q2 == 0.0) S2 = 0.0;
  /* with the coupling the drift is linear in x with coefficient c1 - q2 S2 */
  const double c1e = pr->c1 - pr->q2 * S2;
  for (int i = 0; i < I; ++i) {
    double m = r->mean[i], v = r->var[i];
    if (pr->coarse_model == ORC_COARSE_TAYLOR || pr->coarse_model == ORC_COARSE_TAYLOR1) {
      double ax = -3.0 * pr->c3 * m * m + c1e;
      double axx = -6.0 * pr->c3 * m;
      double b = diffusion(pr, m, M);
      dm[i] = drift(pr, m, M, S2) + (pr->coarse_model == ORC_COARSE_TAYLOR ? 0.5 * axx * v : 0.0);
      dv[i] = (2.0 * ax + pr->B * pr->B) * v + b * b;
    } else if (pr->coarse_model == ORC_COARSE_SIGMA2 || pr->coarse_model == ORC_COARSE_SIGMA3) {
      double xs[3], ws[3];
      int k;
      sigma_points(pr->coarse_model, m, v, xs, ws, &k);
      double ea = 0.0, exa = 0.0, eb2 = 0.0;
      for (int s = 0; s < k; ++s) {
        double a = drift(pr, xs[s], M, S2);
        double b = diffusion(pr, xs[s], M);
        ea += ws[s] * a;
        exa += ws[s] * (xs[s] - m) * a;
        eb2 += ws[s] * b * b;
      }
      dm[i] = ea;
      dv[i] = 2.0 * exa + eb2;
    } else {
      double ex3 = m * m * m + 3.0 * m * v;
      double cov3 = 3.0 * v * (m * m + v);
      double eb = pr->B * m + pr->BE * M + pr->B0;
      dm[i] = -pr->c3 * ex3 + c1e * m + pr->kappa * M + pr->c0;
      dv[i] = 2.0 * (-pr->c3 * cov3 + c1e * v) + pr->B * pr->B * v + eb * eb;
    }
  }
}
void orc_coarse(const orc_problem* pr, const orc_macro* in, orc_macro* out) {
  const int I = pr->n_regions < 2 ? 1 : pr->n_regions;
  const int nc = orc_coarse_steps(pr);
  const double hc = (pr->T / pr->N) / nc;
  orc_macro r = *in;
  for (int s = 0; s < nc; ++s) {
    double dm[ORC_MAX_REGIONS], dv[ORC_MAX_REGIONS];
    orc_coarse_rhs(pr, &r, dm, dv);
    for (int i = 0; i < I; ++i) {
      r.mean[i] = r.mean[i] + hc * dm[i];
      r.var[i] = r.var[i] + hc * dv[i];
    }
  }
  *out = r;
}

/* ------------------------------------------------------------------------
 * Learning of the particle fractions, Sec. 3.6 Def. 3.4 and App. H.
 * reading: the two-state model of App. H,
 *   P(t) = beta + (P(0) - beta) e^{alpha t},
 * fitted to the fractions of region D_0 at the exact slice ends t_1..t_k
 * (with P(0) known) by Levenberg-Marquardt; the paper leaves the LM
 * settings unstated ("implemented in." has no reference), so: start from a
 * one-step linear regression y_{n+1} = r y_n + c (r = e^{alpha dT},
 * beta = c / (1 - r)); damping lambda_0 = 1e-3 scaled by diag(J^T J),
 * /10 on an accepted step, x10 on a rejected one; at most 100 iterations;
 * stop when the accepted step is below 1e-15 relative or lambda > 1e12,
 * then three undamped Gauss-Newton steps to land on the minimiser to
 * rounding level.
 * The fit is rejected (no learning this sweep) unless alpha < 0 and
 * 0 <= beta <= 1.
 * ---------------------------------------------------------------------- */
static double lsq_cost(int n_pts, const double* t, const double* y, double p0, double a, double b) {
  double s = 0.0;
  for (int n = 0; n < n_pts; ++n) {
    double r = y[n] - (b + (p0 - b) * exp(a * t[n]));
    s += r * r;
  }
  return s;
}

int orc_lsq_fit(int n_pts, const double* t, const double* y, double p0, double dT,
                double* alpha, double* beta) {
  if (n_pts < 2) return -1;
  /* initial guess: regress y_{n+1} on y_n over the sequence p0, y_0.. */
  double sx = 0, sy = 0, sxx = 0, sxy = 0;
  for (int n = 0; n < n_pts; ++n) {
    double xv = n == 0 ? p0 : y[n - 1];
    double yv = y[n];
    sx += xv; sy += yv; sxx += xv * xv; sxy += xv * yv;
  }
  double cnt = (double)n_pts;
  double den = sxx - sx * sx / cnt;
  double a = -1.0 / t[n_pts - 1];
  double b = y[n_pts - 1];
  if (den > 0.0) {
    double r = (sxy - sx * sy / cnt) / den;
    double c = (sy - r * sx) / cnt;
    if (r > 0.0 && r < 1.0) {
      a = log(r) / dT;
      b = c / (1.0 - r);
    }
  }
  double lambda = 1e-3;
  double cost = lsq_cost(n_pts, t, y, p0, a, b);
  for (int it = 0; it < 100; ++it) {
    double jaa = 0, jab = 0, jbb = 0, ga = 0, gb = 0;
    for (int n = 0; n < n_pts; ++n) {
      double e = exp(a * t[n]);
      double f = b + (p0 - b) * e;
      double r = y[n] - f;
      double da = (p0 - b) * t[n] * e; /* d f / d alpha */
      double db = 1.0 - e;             /* d f / d beta */
      jaa += da * da; jab += da * db; jbb += db * db;
      ga += da * r; gb += db * r;
    }
    double A = jaa * (1.0 + lambda), D = jbb * (1.0 + lambda), Bm = jab;
    double det = A * D - Bm * Bm;
    if (!(det > 0.0) || !isfinite(det)) {
      lambda *= 10.0;
      if (lambda > 1e12) break;
      continue;
    }
    double step_a = (D * ga - Bm * gb) / det;
    double step_b = (A * gb - Bm * ga) / det;
    double na = a + step_a, nb = b + step_b;
    double ncost = lsq_cost(n_pts, t, y, p0, na, nb);
    if (isfinite(ncost) && ncost < cost) {
      a = na; b = nb; cost = ncost;
      lambda /= 10.0;
      double rel = fmax(fabs(step_a) / (fabs(a) + 1e-300), fabs(step_b) / (fabs(b) + 1e-300));
      if (rel < 1e-15) break;
    } else {
      lambda *= 10.0;
      if (lambda > 1e12) break;
    }
  }
  /* near the minimiser the cost stops resolving the remaining step (its
   * change falls below rounding), so finish with undamped Gauss-Newton steps,
   * which converge to the minimiser to rounding level */
  for (int it = 0; it < 3; ++it) {
    double jaa = 0, jab = 0, jbb = 0, ga = 0, gb = 0;
    for (int n = 0; n < n_pts; ++n) {
      double e = exp(a * t[n]);
      double r = y[n] - (b + (p0 - b) * e);
      double da = (p0 - b) * t[n] * e;
      double db = 1.0 - e;
      jaa += da * da; jab += da * db; jbb += db * db;
      ga += da * r; gb += db * r;
    }
    double det = jaa * jbb - jab * jab;
    if (!(det > 0.0) || !isfinite(det)) break;
    a += (jbb * ga - jab * gb) / det;
    b += (jaa * gb - jab * ga) / det;
  }
  *alpha = a;
  *beta = b;
  if (!(a < 0.0) || !(b >= 0.0) || !(b <= 1.0) || !isfinite(a) || !isfinite(b)) return -2;
  return 0;
}

/* H(P_k, m, theta) of Def. 3.4 (App. H form): beta + (P_k - beta) e^{alpha t},
 * written P_k + (P_k - beta) expm1(alpha t) so that t = 0 returns P_k. */
double orc_extrapolate(double p_k, double alpha, double beta, double dt_ahead) {
  return p_k + (p_k - beta) * expm1(alpha * dt_ahead);
}

/* ------------------------------------------------------------------------
 * The general model of the particle fractions, Sec. 3.6
 * Eq. (generalised_model_multimodal_PFs): dP/dt = A P, where omega_ij >= 0
 * is the rate from region D_i to D_j (i != j), A_ji = omega_ij and
 * A_ii = -sum_{j != i} omega_ij (columns sum to zero, so sum_i P_i is kept).
 * Over one slice P(t_{n+1}) = Phi P(t_n) with Phi = expm(A dT).
 * reading (the paper fits theta = {omega_ij} by Levenberg-Marquardt, with
 * H_i(P_k, m, theta) = (expm(A m dT) P_k)_i, and gives no further detail):
 * with I >= 3 regions all I fractions of the exact slice ends t_0..t_k are
 * fitted (P(t_0) fixed).  The rates are exit rates, so the fit runs on
 * theta_ij with omega_ij = theta_ij^2 (every rate stays >= 0, Phi stays a
 * stochastic matrix and the extrapolated fractions stay in [0, 1] with sum
 * 1; an unconstrained fit of a handful of noisy fractions drives some rates
 * negative; the square keeps the fit free of transcendental functions, so
 * that it is reproducible bit for bit).  Start: the one-step regression
 * P_n ~ Phi0 P_{n-1} (least squares over n = 1..k) with Phi0 ~ I + A dT,
 * i.e. omega_ij ~ Phi0_ji / dT, floored at 1e-3 / (k dT).  The Jacobian is
 * the exact derivative of the computed expm (forward mode through the
 * Taylor polynomial and the squarings) times 2 theta.  Damping and stopping
 * as in the two-region fit above, with each step of theta_ij capped at twice
 * max(|theta_ij|, sqrt(floor)); then up to three Gauss-Newton steps, each
 * kept only if it does not raise the cost.  The fit is used only from k >= I
 * (the k I residuals minus the k fixed sums outnumber the I (I - 1) rates)
 * and only if every rate is finite.  With I = 2 the App. H form above is
 * this model with alpha = -(omega_01 + omega_10),
 * beta = omega_10 / (omega_01 + omega_10).
 * ---------------------------------------------------------------------- */
void orc_rate_generator(int I, const double* om, double* A) {
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

/* C = X Y for n x n row-major matrices (sums over k in increasing order) */
static void matmul(int n, const double* X, const double* Y, double* C) {
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += X[i * n + k] * Y[k * n + j];
      C[i * n + j] = s;
    }
  }
}

void orc_expm(int n, const double* X, const double* dX, double* E, double* dE) {
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
  double Y[64], dY[64], T[64], dT[64], W[64], dW[64];
  for (int r = 0; r < n * n; ++r) {
    Y[r] = X[r] * scale;
    dY[r] = dX ? dX[r] * scale : 0.0;
    T[r] = 0.0;
    dT[r] = 0.0;
  }
  for (int i = 0; i < n; ++i) T[i * n + i] = 1.0;
  /* Horner: T <- I + Y T / m for m = 16 .. 1 */
  for (int m = 16; m >= 1; --m) {
    matmul(n, Y, T, W);
    if (dX) {
      double U[64];
      matmul(n, dY, T, dW);
      matmul(n, Y, dT, U);
      for (int r = 0; r < n * n; ++r) dT[r] = (dW[r] + U[r]) / (double)m;
    }
    for (int r = 0; r < n * n; ++r) T[r] = W[r] / (double)m;
    for (int i = 0; i < n; ++i) T[i * n + i] += 1.0;
  }
  for (int s = 0; s < sq; ++s) {
    if (dX) {
      double U[64];
      matmul(n, dT, T, dW);
      matmul(n, T, dT, U);
      for (int r = 0; r < n * n; ++r) dT[r] = dW[r] + U[r];
    }
    matmul(n, T, T, W);
    for (int r = 0; r < n * n; ++r) T[r] = W[r];
  }
  for (int r = 0; r < n * n; ++r) {
    E[r] = T[r];
    if (dE) dE[r] = dT[r];
  }
}

static void matvec(int n, const double* M, const double* x, double* y) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += M[i * n + k] * x[k];
    y[i] = s;
  }
}

static void rate_phi(int I, const double* om, double dT, double* Phi) {
  double A[16];
  orc_rate_generator(I, om, A);
  for (int r = 0; r < I * I; ++r) A[r] *= dT;
  orc_expm(I, A, NULL, Phi, NULL);
}

static double rate_cost(int I, int k, const double* fr, double dT, const double* om) {
  double Phi[16], p[4], q[4];
  rate_phi(I, om, dT, Phi);
  for (int i = 0; i < I; ++i) p[i] = fr[i];
  double s = 0.0;
  for (int n = 1; n <= k; ++n) {
    matvec(I, Phi, p, q);
    for (int i = 0; i < I; ++i) {
      p[i] = q[i];
      const double r = fr[n * I + i] - p[i];
      s += r * r;
    }
  }
  return s;
}

/* Normal equations of the fit at omega: JtJ [np x np] and g = J^T r, with
 * J = d(model)/d(omega) and r = data - model. */
static void rate_normal(int I, int k, const double* fr, double dT, const double* om, double* JtJ, double* g) {
  const int np = I * (I - 1);
  double A[16], Phi[16], dPhi[12][16];
  orc_rate_generator(I, om, A);
  for (int r = 0; r < I * I; ++r) A[r] *= dT;
  for (int p = 0; p < np; ++p) {
    double e[12] = {0.0}, dA[16];
    e[p] = 1.0;
    orc_rate_generator(I, e, dA);
    for (int r = 0; r < I * I; ++r) dA[r] *= dT;
    orc_expm(I, A, dA, Phi, dPhi[p]);
  }
  if (np == 0) orc_expm(I, A, NULL, Phi, NULL);
  for (int r = 0; r < np * np; ++r) JtJ[r] = 0.0;
  for (int p = 0; p < np; ++p) g[p] = 0.0;
  double P[4], Q[4], S[12][4], S2[4], S3[4];
  for (int i = 0; i < I; ++i) P[i] = fr[i];
  for (int p = 0; p < np; ++p)
    for (int i = 0; i < I; ++i) S[p][i] = 0.0;
  for (int n = 1; n <= k; ++n) {
    /* S_p <- dPhi_p P + Phi S_p (the derivative of P_n), then P <- Phi P */
    for (int p = 0; p < np; ++p) {
      matvec(I, dPhi[p], P, S2);
      matvec(I, Phi, S[p], S3);
      for (int i = 0; i < I; ++i) S[p][i] = S2[i] + S3[i];
    }
    matvec(I, Phi, P, Q);
    for (int i = 0; i < I; ++i) P[i] = Q[i];
    for (int i = 0; i < I; ++i) {
      const double r = fr[n * I + i] - P[i];
      for (int p = 0; p < np; ++p) {
        g[p] += S[p][i] * r;
        for (int q = 0; q < np; ++q) JtJ[p * np + q] += S[p][i] * S[q][i];
      }
    }
  }
}

/* Solve M x = b for a symmetric positive definite M (Cholesky); 0 on success */
static int spd_solve(int n, const double* M, const double* b, double* x) {
  double L[144];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = M[i * n + j];
      for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      if (i == j) {
        if (!(s > 0.0) || !isfinite(s)) return -1;
        L[i * n + i] = sqrt(s);
      } else {
        L[i * n + j] = s / L[j * n + j];
      }
    }
  }
  double y[12];
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
    y[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
  return 0;
}

/* The rates are non-negative (they are transition rates between regions),
 * and a rate far above 1 / dT is indistinguishable from a faster one: a
 * region left at rate omega keeps a share e^{-omega dT} of its mass over one
 * slice, below 2e-9 once omega dT >= 20, so the slice-end fractions cannot
 * tell such rates apart and the cost is flat there.  The fit is therefore
 * the least-squares minimiser of rate_cost over the box
 * 0 <= omega <= omega_max = 20 / dT, found by Levenberg-Marquardt on omega
 * with the bounds kept by projection: in every iteration a rate is held when
 * it sits at a bound and the cost would fall only if it crossed it (J^T r
 * pointing out of the box); the other ("free") rates take the damped
 * Gauss-Newton step (J^T J + mu I) d = J^T r, and the new point is the step
 * clipped to the box.  The damping mu follows the gain
 * ratio rho = (actual decrease) / (decrease predicted by the linear model):
 * after a step with rho > 0 it is multiplied by max(1/3, 1 - (2 rho - 1)^3),
 * after a failed one by nu, which doubles with every failure in a row
 * (Madsen, Nielsen and Tingleff, "Methods for non-linear least squares
 * problems", 2004, Sec. 3.2). */
static int rate_free_step(int np, const double* om, double om_max, const double* JtJ, const double* g,
                          double mu, double* step, double* pred) {
  int fr_idx[12], nf = 0;
  for (int p = 0; p < np; ++p) {
    step[p] = 0.0;
    const int held = (om[p] == 0.0 && !(g[p] > 0.0)) || (om[p] == om_max && !(g[p] < 0.0));
    if (!held) fr_idx[nf++] = p;
  }
  *pred = 0.0;
  if (nf == 0) return 0;
  double M[144], b[12], x[12];
  for (int a = 0; a < nf; ++a) {
    for (int c = 0; c < nf; ++c) M[a * nf + c] = JtJ[fr_idx[a] * np + fr_idx[c]];
    M[a * nf + a] = M[a * nf + a] + mu;
    b[a] = g[fr_idx[a]];
  }
  if (spd_solve(nf, M, b, x) != 0) return -1;
  /* predicted decrease of the cost: d^T (mu d + g) over the free rates */
  double s = 0.0;
  for (int a = 0; a < nf; ++a) {
    step[fr_idx[a]] = x[a];
    s += x[a] * (mu * x[a] + b[a]);
  }
  *pred = s;
  return nf;
}

int orc_rate_fit(int I, int k, const double* fr, double dT, double* om) {
  const int np = I * (I - 1);
  if (I < 2 || I > 4 || k < I) return -1;
  /* initial rates: the one-step regression P_n ~ Phi0 P_{n-1} (least squares
   * over n = 1..k), Phi0 ~ I + A dT, so omega_ij ~ Phi0_ji / dT, floored at
   * a small positive rate and capped at 1 / dT (a start among much faster
   * rates lies where the cost is flat and leaves the iteration nothing to
   * follow); equal rates 1 / (I k dT) if the regression is singular */
  const double floor_rate = 1e-3 / ((double)k * dT);
  const double om_max = 20.0 / dT;
  {
    double Sxx[16] = {0.0}, Syx[16] = {0.0};
    for (int n = 1; n <= k; ++n)
      for (int a = 0; a < I; ++a)
        for (int b = 0; b < I; ++b) {
          Sxx[a * I + b] += fr[(n - 1) * I + a] * fr[(n - 1) * I + b];
          Syx[a * I + b] += fr[n * I + a] * fr[(n - 1) * I + b];
        }
    int ok = 1;
    double Phi0[16];
    for (int a = 0; a < I && ok; ++a) {
      /* row a of Phi0 solves Sxx x = (row a of Syx) (Sxx is symmetric) */
      double rhs[4], x[4];
      for (int b = 0; b < I; ++b) rhs[b] = Syx[a * I + b];
      if (spd_solve(I, Sxx, rhs, x) != 0) {
        ok = 0;
      } else {
        for (int b = 0; b < I; ++b) Phi0[a * I + b] = x[b];
      }
    }
    for (int i = 0; i < I; ++i)
      for (int j = 0; j < I; ++j) {
        if (j == i) continue;
        const double w = ok ? Phi0[j * I + i] / dT : 1.0 / ((double)I * (double)k * dT);
        om[i * (I - 1) + (j < i ? j : j - 1)] = isfinite(w) && w > floor_rate ? fmin(w, 1.0 / dT) : floor_rate;
      }
  }
  double JtJ[144], g[12], st[12], nw[12];
  double cost = rate_cost(I, k, fr, dT, om);
  rate_normal(I, k, fr, dT, om, JtJ, g);
  double mu = 0.0, nu = 2.0;
  for (int p = 0; p < np; ++p) mu = fmax(mu, JtJ[p * np + p]);
  mu = 1e-3 * mu;
  int converged = cost == 0.0;
  for (int it = 0; it < ORC_RATE_FIT_MAX_ITER && !converged; ++it) {
    double pred;
    const int nf = rate_free_step(np, om, om_max, JtJ, g, mu, st, &pred);
    if (nf == 0) { /* every rate held at a bound: a stationary point */
      converged = 1;
      break;
    }
    double ncost = 0.0;
    if (nf > 0) {
      for (int p = 0; p < np; ++p) nw[p] = fmin(fmax(om[p] + st[p], 0.0), om_max);
      ncost = rate_cost(I, k, fr, dT, nw);
    }
    if (nf > 0 && pred > 0.0 && isfinite(ncost) && ncost < cost) {
      const double rho = (cost - ncost) / pred;
      const double t = 2.0 * rho - 1.0;
      for (int p = 0; p < np; ++p) om[p] = nw[p];
      cost = ncost;
      rate_normal(I, k, fr, dT, om, JtJ, g);
      mu = mu * fmax(1.0 / 3.0, 1.0 - t * t * t);
      nu = 2.0;
      if (pred < 1e-15 * cost || cost == 0.0) converged = 1; /* the model promises nothing more */
    } else {
      if (nf > 0 && !(pred > 0.0)) { /* no descent left on the free rates */
        converged = 1;
        break;
      }
      mu = mu * nu;
      nu = 2.0 * nu;
      if (nu > 1e18) break;
    }
  }
  for (int p = 0; p < np; ++p)
    if (!isfinite(om[p]) || !(om[p] >= 0.0)) return -2;
  return converged ? 0 : 1;
}

void orc_rate_propagate(int I, const double* om, double dT, const double* p_in, int m, double* p_out) {
  double Phi[16], p[4], q[4];
  rate_phi(I, om, dT, Phi);
  for (int i = 0; i < I; ++i) p[i] = p_in[i];
  for (int s = 0; s < m; ++s) {
    matvec(I, Phi, p, q);
    for (int i = 0; i < I; ++i) p[i] = q[i];
  }
  for (int i = 0; i < I; ++i) p_out[i] = p[i];
}

/* ------------------------------------------------------------------------
 * Classical Parareal, Sec. 3.1 Eq. (original_parareal), with the noisy fine
 * propagator of Lemma 4.1: F(u) = Fm u + Fa + eps.
 * ---------------------------------------------------------------------- */
void orc_parareal_scalar(int N, int K, double u0, double Fm, double Fa, double Gm, double Ga,
                         const double* noise, double* out) {
  const int W = N + 1;
  out[0] = u0;
  for (int n = 0; n < N; ++n) out[n + 1] = Gm * out[n] + Ga;
  for (int k = 1; k <= K; ++k) {
    double* cur = out + (size_t)k * W;
    const double* prev = out + (size_t)(k - 1) * W;
    cur[0] = u0;
    for (int n = 0; n < N; ++n) {
      double fine = Fm * prev[n] + Fa + (noise ? noise[(size_t)k * W + n + 1] : 0.0);
      double g_new = Gm * cur[n] + Ga;
      double g_old = Gm * prev[n] + Ga;
      cur[n + 1] = g_new + fine - g_old;
    }
  }
}

/* ------------------------------------------------------------------------
 * MC-moments Parareal: the generalised iteration Eq. (mM_parareal_other_k_NEW)
 * with the operators of Def. 3.1 (unimodal), Def. 3.2 (multimodal) and
 * Def. 3.4 (learning).
 * ---------------------------------------------------------------------- */
static void macro_from_stats(const orc_problem* pr, const orc_stats* st, orc_macro* r) {
  memset(r, 0, sizeof(*r));
  const int I = pr->n_regions < 2 ? 1 : pr->n_regions;
  for (int i = 0; i < I; ++i) {
    r->frac[i] = (double)st->count[i] / (double)pr->P;
    r->mean[i] = st->mean[i];
    r->var[i] = st->var[i];
  }
}

/* Lifting L(rho) = T(rho, u0) per region, Def. 3.1/3.2.
 * reading: a region of u0 with no particles is left alone; a negative
 * coarse variance (which T cannot reach) leaves the region untouched. */
static void lift(const orc_problem* pr, int n, const orc_macro* rho, const orc_stats* st0,
                 const double* u0, double* out) {
  const int I = pr->n_regions < 2 ? 1 : pr->n_regions;
  int doit[ORC_MAX_REGIONS] = {0};
  double mu[ORC_MAX_REGIONS] = {0}, sg[ORC_MAX_REGIONS] = {0};
  for (int i = 0; i < I; ++i) {
    doit[i] = st0->count[i] > 0 && rho->var[i] >= 0.0;
    mu[i] = rho->mean[i];
    sg[i] = rho->var[i];
  }
  orc_match(pr, n, mu, sg, doit, st0, u0, out);
}

static double transformed(double x, double mu, double sigma, double m, double v) {
  double s = sqrt(sigma / v);
  return x + (mu - m) + (s - 1.0) * (x - m);
}

int orc_parareal(const orc_problem* pr, const double* u0_in, double* hist, orc_macro* macro_out,
                 double* parts_out, orc_result* res) {
  const int N = pr->N;
  const long long P = pr->P;
  const int I = pr->n_regions < 2 ? 1 : pr->n_regions;
  const int multimodal = pr->variant != ORC_UNIMODAL && I > 1;
  const int learning = pr->variant == ORC_LEARNING && I >= 2;
  const double dT = pr->T / N;
  int K = pr->max_iter < N ? pr->max_iter : N;
  if (K < 1) K = 1;
  if (pr->family == ORC_FAMILY_ROTATOR && I > 1) return -1;

  double* u0 = (double*)malloc(sizeof(double) * (size_t)P);
  if (u0_in) memcpy(u0, u0_in, sizeof(double) * (size_t)P);
  else orc_initial(pr, u0);

  double* U = (double*)malloc(sizeof(double) * (size_t)P * (N + 1));      /* u^k_n */
  double* Unew = (double*)malloc(sizeof(double) * (size_t)P * (N + 1));   /* u^{k+1}_n */
  double* Bf = (double*)malloc(sizeof(double) * (size_t)P * N);           /* F_n(u^k_n) */
  orc_macro* rho = (orc_macro*)calloc((size_t)N + 1, sizeof(orc_macro));
  orc_macro* rho_new = (orc_macro*)calloc((size_t)N + 1, sizeof(orc_macro));
  orc_macro* cache = (orc_macro*)calloc((size_t)N, sizeof(orc_macro));    /* C_n(rho^k_n) */
  orc_stats* rst = (orc_stats*)calloc((size_t)N, sizeof(orc_stats));
  double* frac0 = (double*)calloc((size_t)N + 1, sizeof(double));
  double* tpts = (double*)calloc((size_t)N + 1, sizeof(double));

  /* k = 0: rho^0_0 = R(u0); rho^0_{n+1} = C_n(rho^0_n); u^0_n = L(rho^0_n). */
  orc_stats st0;
  orc_restrict(pr, u0, &st0);
  macro_from_stats(pr, &st0, &rho[0]);
  for (int n = 0; n < N; ++n) {
    orc_coarse(pr, &rho[n], &rho[n + 1]);
    cache[n] = rho[n + 1];
  }
  memcpy(U, u0, sizeof(double) * (size_t)P);
  for (int n = 1; n <= N; ++n) lift(pr, n, &rho[n], &st0, u0, U + (size_t)n * P);
  if (hist) {
    for (int n = 0; n <= N; ++n) orc_mixture(pr, &rho[n], &hist[2 * n], &hist[2 * n + 1]);
  }

  orc_result r = {0, 0, 0.0, 0, 0};
  for (int k = 1; k <= K; ++k) {
    /* the fine propagator on every slice (parallel in the paper) */
    for (int n = 0; n < N; ++n) {
      orc_fine(pr, n, U + (size_t)n * P, Bf + (size_t)n * P, NULL);
      orc_restrict(pr, Bf + (size_t)n * P, &rst[n]);
    }
    /* fractions of the new iterate come from the fine propagator (Def. 3.2) */
    double* fr = (double*)malloc(sizeof(double) * (size_t)(N + 1) * ORC_MAX_REGIONS);
    for (int i = 0; i < I; ++i) fr[i] = rho[0].frac[i];
    for (int n = 0; n < N; ++n)
      for (int i = 0; i < I; ++i) fr[(n + 1) * ORC_MAX_REGIONS + i] = (double)rst[n].count[i] / (double)P;
    /* learning (Def. 3.4): after sweep k the slice ends t_0..t_k are exact;
     * fit on them and extrapolate the fractions beyond t_k. */
    if (learning && I >= 3 && k >= I) {
      /* the general rate model on all fractions (Eq. generalised_model_multimodal_PFs) */
      double* frk = (double*)malloc(sizeof(double) * (size_t)(k + 1) * I);
      double om[12];
      for (int n = 0; n <= k; ++n)
        for (int i = 0; i < I; ++i) frk[n * I + i] = fr[n * ORC_MAX_REGIONS + i];
      if (orc_rate_fit(I, k, frk, dT, om) >= 0) {
        for (int n = k + 1; n <= N; ++n)
          orc_rate_propagate(I, om, dT, fr + (size_t)(n - 1) * ORC_MAX_REGIONS, 1, fr + (size_t)n * ORC_MAX_REGIONS);
      }
      free(frk);
    }
    if (learning && I == 2 && k >= 2) {
      for (int n = 0; n <= k; ++n) {
        frac0[n] = fr[n * ORC_MAX_REGIONS + 0];
        tpts[n] = n * dT;
      }
      double al, be;
      if (orc_lsq_fit(k, tpts + 1, frac0 + 1, frac0[0], dT, &al, &be) == 0) {
        double pk = frac0[k];
        for (int n = k + 1; n <= N; ++n) {
          double p0hat = orc_extrapolate(pk, al, be, (n - k) * dT);
          fr[n * ORC_MAX_REGIONS + 0] = p0hat;
          fr[n * ORC_MAX_REGIONS + 1] = 1.0 - p0hat;
        }
      }
    }

    rho_new[0] = rho[0];
    memcpy(Unew, u0, sizeof(double) * (size_t)P);
    for (int n = 0; n < N; ++n) {
      for (int i = 0; i < I; ++i) rho_new[n].frac[i] = fr[n * ORC_MAX_REGIONS + i];
      orc_macro a;
      orc_coarse(pr, &rho_new[n], &a);
      const orc_stats* b = &rst[n];
      orc_macro nxt;
      memset(&nxt, 0, sizeof(nxt));
      int doit[ORC_MAX_REGIONS] = {0};
      double mu[ORC_MAX_REGIONS] = {0}, sg[ORC_MAX_REGIONS] = {0};
      for (int i = 0; i < I; ++i) {
        if (b->count[i] == 0) {
          /* reading (Def. 3.2/3.4): an empty region carries the coarse
           * prediction and moves no particle */
          nxt.mean[i] = a.mean[i];
          nxt.var[i] = a.var[i];
          continue;
        }
        /* alpha = a + R(b) - c, evaluated as R(b) + (a - c) so that a == c
         * gives R(b) exactly (Property 3.3 bit for bit) */
        double am = b->mean[i] + (a.mean[i] - cache[n].mean[i]);
        double av = b->var[i] + (a.var[i] - cache[n].var[i]);
        int accept = av >= 0.0;
        if (multimodal && accept) {
          /* Def. 3.2: accept only if T leaves the fractions unchanged;
           * T is monotone, so test the extreme particle of the region.
           * reading: a region with V = 0 (redraw branch) is not moved. */
          if (b->var[i] == 0.0) {
            accept = 0;
          } else {
            /* D_i = [t_i, t_{i+1}): the smallest particle stays at or above
             * t_i, the largest below t_{i+1} */
            if (i > 0)
              accept = transformed(b->min[i], am, av, b->mean[i], b->var[i]) >= region_lower(pr, i);
            if (accept && i < I - 1)
              accept = transformed(b->max[i], am, av, b->mean[i], b->var[i]) < region_lower(pr, i + 1);
          }
        }
        if (accept) {
          nxt.mean[i] = am;
          nxt.var[i] = av;
          doit[i] = 1;
          mu[i] = am;
          sg[i] = av;
          r.accepted_total++;
        } else {
          nxt.mean[i] = b->mean[i];
          nxt.var[i] = b->var[i];
          r.rejected_total++;
        }
      }
      for (int i = 0; i < I; ++i) nxt.frac[i] = fr[(n + 1) * ORC_MAX_REGIONS + i];
      rho_new[n + 1] = nxt;
      orc_match(pr, n + 1, mu, sg, doit, b, Bf + (size_t)n * P, Unew + (size_t)(n + 1) * P);
      cache[n] = a;
    }
    free(fr);

    double change = 0.0;
    for (int n = 0; n <= N; ++n) {
      double M1, V1, M0, V0;
      orc_mixture(pr, &rho_new[n], &M1, &V1);
      orc_mixture(pr, &rho[n], &M0, &V0);
      change = fmax(change, fmax(fabs(M1 - M0), fabs(V1 - V0)));
      if (hist) {
        hist[((size_t)k * (N + 1) + n) * 2] = M1;
        hist[((size_t)k * (N + 1) + n) * 2 + 1] = V1;
      }
    }
    memcpy(rho, rho_new, sizeof(orc_macro) * (size_t)(N + 1));
    double* t = U; U = Unew; Unew = t;
    r.sweeps = k;
    r.last_change = change;
    if (change < pr->tol) {
      r.converged = 1;
      break;
    }
  }
  if (r.sweeps == N) r.converged = 1;
  if (macro_out) memcpy(macro_out, rho, sizeof(orc_macro) * (size_t)(N + 1));
  if (parts_out) memcpy(parts_out, U, sizeof(double) * (size_t)P * (N + 1));
  if (res) *res = r;
  free(u0); free(U); free(Unew); free(Bf); free(rho); free(rho_new); free(cache); free(rst);
  free(frac0); free(tpts);
  return 0;
}

void orc_fine_serial(const orc_problem* pr, const double* u0_in, orc_stats* stats, double* parts) {
  const long long P = pr->P;
  const int N = pr->N;
  double* u = (double*)malloc(sizeof(double) * (size_t)P);
  double* v = (double*)malloc(sizeof(double) * (size_t)P);
  if (u0_in) memcpy(u, u0_in, sizeof(double) * (size_t)P);
  else orc_initial(pr, u);
  for (int n = 0; n <= N; ++n) {
    if (stats) orc_restrict(pr, u, &stats[n]);
    if (parts) memcpy(parts + (size_t)n * P, u, sizeof(double) * (size_t)P);
    if (n == N) break;
    orc_fine(pr, n, u, v, NULL);
    double* t = u; u = v; v = t;
  }
  free(u);
  free(v);
}

/* ------------------------------------------------------------------------
 * Adjoint of the serial fine propagator F_{N-1} o ... o F_0 (the limit the
 * Parareal iteration reproduces, Property 3.3).  Reverse-mode
 * differentiation of the Euler-Maruyama recursion of Sec. 1.2,
 *   x_{j+1,p} = x_{j,p} + h a(x_{j,p}, m_j) + sqrt(h) b(x_{j,p}, m_j) xi_{j,p},
 * with the mean field m_j = (1/P) sum_q x_{j,q}, a = -c3 x^3 + c1 x + kappa m + c0
 * and b = B x + BE m + B0:
 *   d x_{j+1,p} / d x_{j,q} = delta_pq (1 + h a_x(x_{j,p}) + sqrt(h) B xi_{j,p})
 *                             + (h kappa + sqrt(h) BE xi_{j,p}) / P,
 *   a_x(x) = -3 c3 x^2 + c1,
 * so with lambda_j = dL/dx_j, S_j = sum_p lambda_{j+1,p} and
 * Z_j = sum_p lambda_{j+1,p} xi_{j,p}:
 *   lambda_{j,q} = lambda_{j+1,q} (1 + h a_x(x_{j,q}) + sqrt(h) B xi_{j,q})
 *                  + (h kappa S_j + sqrt(h) BE Z_j) / P + [loss at x_j]
 * and the explicit parameter derivatives of step j are
 *   d/dc3 = -h x^3, d/dc1 = h x, d/dkappa = h m_j, d/dc0 = h,
 *   d/dB0 = sqrt(h) xi, d/dB = sqrt(h) x xi, d/dBE = sqrt(h) m_j xi.
 * The loss at slice end n injects gm/P + gv (2/P)(x - M_n)
 * (dV/dx_q = (2/P)(x_q - M) for the population variance).
 * ---------------------------------------------------------------------- */
int orc_adjoint(const orc_problem* pr, const double* u0_in, const double* gm, const double* gv,
                double grad[ORC_N_THETA], double* moments) {
  if (pr->family == ORC_FAMILY_ROTATOR || pr->q2 != 0.0) return -1;
  const long long P = pr->P;
  const int N = pr->N;
  const int nf = orc_fine_steps(pr);
  const double h = orc_fine_h(pr);
  const double sqrt_h = sqrt(h);
  const long long J = (long long)N * nf;
  double* X = (double*)malloc(sizeof(double) * (size_t)P * (size_t)(J + 1));
  double* m = (double*)malloc(sizeof(double) * (size_t)(J + 1));
  double* lam = (double*)calloc((size_t)P, sizeof(double));
  double* Mn = (double*)malloc(sizeof(double) * (size_t)(N + 1));
  double* Vn = (double*)malloc(sizeof(double) * (size_t)(N + 1));
  if (u0_in) memcpy(X, u0_in, sizeof(double) * (size_t)P);
  else orc_initial(pr, X);
  /* forward: the serial fine run, keeping every state and mean */
  for (long long j = 0; j < J; ++j) {
    const double* x = X + (size_t)j * P;
    double* y = X + (size_t)(j + 1) * P;
    m[j] = ensemble_mean(x, P);
    const int n = (int)(j / nf), js = (int)(j % nf);
    for (long long p = 0; p < P; ++p) {
      double xi = orc_normal(pr, 0, (uint32_t)js, (uint32_t)n, p);
      y[p] = x[p] + drift(pr, x[p], m[j], 0.0) * h + diffusion(pr, x[p], m[j]) * sqrt_h * xi;
    }
  }
  m[J] = ensemble_mean(X + (size_t)J * P, P);
  for (int n = 0; n <= N; ++n) {
    const double* x = X + (size_t)n * nf * P;
    double mm = ensemble_mean(x, P), vv = 0.0;
    for (long long p = 0; p < P; ++p) vv += (x[p] - mm) * (x[p] - mm);
    Mn[n] = mm;
    Vn[n] = vv / (double)P;
    if (moments) {
      moments[2 * n] = Mn[n];
      moments[2 * n + 1] = Vn[n];
    }
  }
  /* reverse */
  for (int k = 0; k < ORC_N_THETA; ++k) grad[k] = 0.0;
  for (long long j = J - 1; j >= 0; --j) {
    if ((j + 1) % nf == 0) {
      const int n = (int)((j + 1) / nf);
      const double* x1 = X + (size_t)(j + 1) * P;
      for (long long p = 0; p < P; ++p)
        lam[p] += gm[n - 1] / (double)P + gv[n - 1] * (2.0 / (double)P) * (x1[p] - Mn[n]);
    }
    const double* x = X + (size_t)j * P;
    const int n = (int)(j / nf), js = (int)(j % nf);
    double S = 0.0, Z = 0.0;
    for (long long p = 0; p < P; ++p) {
      const double xv = x[p];
      const double xi = orc_normal(pr, 0, (uint32_t)js, (uint32_t)n, p);
      grad[0] += lam[p] * (-h * xv * xv * xv);
      grad[1] += lam[p] * (h * xv);
      grad[2] += lam[p] * (h * m[j]);
      grad[3] += lam[p] * h;
      grad[4] += lam[p] * (sqrt_h * xi);
      grad[5] += lam[p] * (sqrt_h * xv * xi);
      grad[6] += lam[p] * (sqrt_h * m[j] * xi);
      S += lam[p];
      Z += lam[p] * xi;
    }
    const double shift = (h * pr->kappa * S + sqrt_h * pr->BE * Z) / (double)P;
    for (long long p = 0; p < P; ++p) {
      const double xv = x[p];
      const double xi = orc_normal(pr, 0, (uint32_t)js, (uint32_t)n, p);
      const double ax = -3.0 * pr->c3 * xv * xv + pr->c1;
      lam[p] = lam[p] * (1.0 + h * ax + sqrt_h * pr->B * xi) + shift;
    }
  }
  free(X); free(m); free(lam); free(Mn); free(Vn);
  return 0;
}

int orc_adjoint_loss(const orc_problem* pr, const double* u0_in, const double* m_tgt,
                     const double* v_tgt, double grad[ORC_N_THETA], double* loss) {
  if (pr->family == ORC_FAMILY_ROTATOR) return -1;
  const int N = pr->N;
  double* mom = (double*)malloc(sizeof(double) * 2 * (size_t)(N + 1));
  double* gm = (double*)calloc((size_t)N, sizeof(double));
  double* gv = (double*)calloc((size_t)N, sizeof(double));
  /* the moments first (a zero-cotangent pass), then the cotangents of L */
  int rc = orc_adjoint(pr, u0_in, gm, gv, grad, mom);
  if (rc == 0) {
    double L = 0.0;
    for (int n = 1; n <= N; ++n) {
      const double dm = mom[2 * n] - m_tgt[n - 1], dv = mom[2 * n + 1] - v_tgt[n - 1];
      L += dm * dm + dv * dv;
      gm[n - 1] = 2.0 * dm;
      gv[n - 1] = 2.0 * dv;
    }
    if (loss) *loss = L;
    rc = orc_adjoint(pr, u0_in, gm, gv, grad, NULL);
  }
  free(mom); free(gm); free(gv);
  return rc;
}
