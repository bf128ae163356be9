/*
 * oracle.h -- plain FP64 CPU oracle for MC-moments micro-macro Parareal
 * (Bossuyt, Vandewalle, Samaey, arXiv 2310.11365).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or execute this code: only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py use it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Everything is written for clarity, not speed: one thread, double
 * precision, no blocking or fusion beyond what the paper states.
 *
 * Pins (tests/test_oracle_*.py): every function here is checked against
 * something other than itself -- closed forms, exact sample-path
 * identities, quadrature, brute force on tiny ensembles, invariants such as
 * Lemma 3.1 and Property 3.3, the classical Parareal recursion, and the
 * outcomes the paper states for its setups.  Parity unpinned: the values of
 * whole nonlinear runs (orc_parareal on the cubic, double-well and rotator
 * models at full size), for which the paper prints no numbers (its figures
 * are not in the text); they rest on the pinned parts and the invariants.
 *
 * The model family (Sec. 2.1, Eq. SDE_class_1 with f(x) = x):
 *   drift      a(x, m) = -c3 x^3 + c1 x + kappa m + c0
 *   diffusion  b(x, m) = B x + BE m + B0
 * where m = E[X] is the ensemble mean.  The linear McKean-Vlasov SDE of
 * Lemma 2.1 is c3 = 0; the cubic and double-well drifts of Sec. 5.3 are
 * c3 > 0 with additive noise (B = BE = 0).  One more term, -q2 x E[X^2]
 * (q2 = 0 otherwise), couples the drift to the ensemble's second moment:
 * the polynomial-drift example of App. C, dX = (alpha X + E[X] - X E[X^2]) dt
 * + X dW, is c1 = alpha, kappa = 1, q2 = 1, B = 1.  In every coarse model the
 * term acts as the linear coefficient c1 - q2 S with S = V + M^2 of the
 * law (the mixture's with several regions).  The adjoint does not take it.
 *
 * A second family, the plane rotator of Sec. 5 (Example "Unimodal plane
 * rotator", Eq. SDE_plane_rotator), has the drift
 *   a(x) = (K/P) sum_q sin(X_q - x) - g sin x = K (S cos x - C sin x) - g sin x
 * with S, C the ensemble means of sin X and cos X (the particle itself
 * included, sin 0 = 0), g = 1 in the paper, additive noise b = B0 =
 * sqrt(2 k_B T), and every particle shifted modulo 2 pi into [-pi, pi]
 * (x - 2 pi floor((x + pi) / 2 pi)) after each Euler-Maruyama step and in
 * the initial ensemble (the paper prints [0, 2 pi]; see orc_wrap).  It has
 * one region and no adjoint here.
 *
 * Random numbers (Property 3.3 needs the same draws in every iteration):
 * Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *   key     = (seed mod 2^32, seed div 2^32)
 *   counter = (p div 4, j, n | tag << 24, problem_tag)
 * word w of the output belongs to particle 4 (p div 4) + w.  A word o is
 * mapped to the uniform u = ((o >> 9) + 1/2) 2^-23 and the pairs (w0, w1),
 * (w2, w3) go through Box-Muller: z = sqrt(-2 ln u_a) (cos 2 pi u_b,
 * sin 2 pi u_b).  Tags: 0 = Euler-Maruyama noise at fine step j of slice n;
 * 1 = initial ensemble X0 = m0 + s0 z (j = 0, n = 0); 2 = the redraw branch
 * of the matching T when V[u] = 0 (j = region, n = slice).
 */
#ifndef MMP_ORACLE_H
#define MMP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_REGIONS 4

enum { ORC_UNIMODAL = 0, ORC_MULTIMODAL = 1, ORC_LEARNING = 2 };
enum { ORC_FAMILY_POLY = 0, ORC_FAMILY_ROTATOR = 1 };

typedef struct {
  double c3, c1, kappa, c0;   /* drift coefficients */
  double B, BE, B0;           /* diffusion coefficients */
  double m0, s0;              /* p0 = N(m0, s0^2) */
  double T;                   /* horizon */
  int N;                      /* Parareal slices */
  double dt;                  /* requested fine step */
  long long P;                /* particles */
  double coarse_h;            /* largest coarse step */
  int n_regions;              /* 1 .. ORC_MAX_REGIONS */
  double threshold;           /* t_1: D_0 = {x < t_1}, D_1 = {t_1 <= x (< t_2)}, ... */
  int variant;                /* ORC_UNIMODAL / ORC_MULTIMODAL / ORC_LEARNING */
  uint64_t seed;
  uint32_t problem_tag;
  double tol;                 /* stop when max_n |d(M,V)| < tol */
  int max_iter;               /* at most this many fine sweeps (<= N) */
  int coarse_model;           /* ORC_COARSE_CLOSURE / _TAYLOR / _SIGMA2 / _SIGMA3 */
  double threshold2, threshold3;  /* t_2, t_3 (n_regions 3, 4): D_2 = {t_2 <= x (< t_3)}, D_3 = {x >= t_3} */
  int family;                 /* ORC_FAMILY_POLY / ORC_FAMILY_ROTATOR */
  double K, g;                /* plane rotator: coupling K, pinning g (c3..c0, B, BE unused) */
  double q2;                  /* second-moment coupling: the drift gets -q2 x E[X^2] (App. C) */
} orc_problem;

/* Coarse moment models (Sec. 2): the Gaussian closure (expectations of the
 * polynomial coefficients under N(M, Sigma) in closed form), the Taylor
 * model (Eq. moment_model_class_1), and the Gaussian-assumed density
 * (Eq. Gaussian_model_McK_V_SDE) with a 2- or 3-point sigma-point rule. */
#define ORC_COARSE_CLOSURE 0
#define ORC_COARSE_TAYLOR 1
#define ORC_COARSE_SIGMA2 2
#define ORC_COARSE_SIGMA3 3
/* The Taylor model without the Sigma term of the mean, dM = a(M) (the first
 * coarse model of the plane-rotator example). */
#define ORC_COARSE_TAYLOR1 4

/* Restriction of one ensemble (Eq. multimodal_R plus the extremes needed by
 * the "fractions unchanged" test of Def. 3.2). */
typedef struct {
  long long count[ORC_MAX_REGIONS];
  double mean[ORC_MAX_REGIONS];
  double var[ORC_MAX_REGIONS];     /* population variance, 1/n_i */
  double min[ORC_MAX_REGIONS];
  double max[ORC_MAX_REGIONS];
  double gmean, gvar;              /* whole-ensemble mean / population var */
} orc_stats;

/* Macro state rho = (P_i, M_i, Sigma_i), i < I (Def. 3.2). */
typedef struct {
  double frac[ORC_MAX_REGIONS];
  double mean[ORC_MAX_REGIONS];
  double var[ORC_MAX_REGIONS];
} orc_macro;

/* -- random numbers ------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t word);
/* the normal drawn for particle p under (tag, j, n) */
double orc_normal(const orc_problem* pr, int tag, uint32_t j, uint32_t n, long long p);
/* X0 = m0 + s0 z, tag 1 */
void orc_initial(const orc_problem* pr, double* u0);

/* x shifted modulo 2 pi into [-pi, pi] (plane rotator) */
double orc_wrap(double x);

/* -- fine propagator (Eq. Euler_Maruyama) -------------------------------- */
int orc_fine_steps(const orc_problem* pr);
double orc_fine_h(const orc_problem* pr);
/* u_out = F_n(u_in); if means != NULL it receives the n_f + 1 ensemble
 * means m_0 .. m_{n_f} seen by the mean-field term. */
void orc_fine(const orc_problem* pr, int n, const double* u_in, double* u_out, double* means);

/* -- restriction and matching (Sec. 3.4) --------------------------------- */
int orc_region(const orc_problem* pr, double x);
void orc_restrict(const orc_problem* pr, const double* u, orc_stats* st);
void orc_mixture(const orc_problem* pr, const orc_macro* r, double* M, double* V);
/* u_out = T([mu_i, sigma_i], u) applied in every region i with do_region[i]
 * != 0; other regions are copied.  n is the slice index of the target, used
 * only by the V[u] = 0 redraw branch. */
void orc_match(const orc_problem* pr, int n, const double* mu, const double* sigma,
               const int* do_region, const orc_stats* st_u, const double* u, double* u_out);

/* -- coarse propagator (Sec. 2, Gaussian closure, forward Euler) -------- */
int orc_coarse_steps(const orc_problem* pr);
void orc_coarse_rhs(const orc_problem* pr, const orc_macro* r, double* dm, double* dv);
void orc_coarse(const orc_problem* pr, const orc_macro* in, orc_macro* out);

/* -- learning of particle fractions (Sec. 3.6, App. H) ------------------ */
/* Fit P(t) = beta + (p0 - beta) e^{alpha t} to (t_n, y_n), n = 1..n_pts,
 * with P(0) = p0 fixed.  Returns 0 on success. */
int orc_lsq_fit(int n_pts, const double* t, const double* y, double p0, double dT,
                double* alpha, double* beta);
double orc_extrapolate(double p_k, double alpha, double beta, double dt_ahead);

/* The general model of the fractions (Eq. generalised_model_multimodal_PFs):
 * dP/dt = A P with the rates omega_ij >= 0 (i != j) from D_i to D_j,
 * A_ji = omega_ij, A_ii = -sum_{j != i} omega_ij.  omega is stored as
 * omega[i (I-1) + (j < i ? j : j - 1)], I (I-1) values. */
void orc_rate_generator(int I, const double* omega, double* A);
/* E = expm(X) for an n x n row-major X (n <= 8), by scaling and squaring
 * with a degree-16 Taylor polynomial; if dX is not NULL, dE receives the
 * derivative of that computation in the direction dX. */
void orc_expm(int n, const double* X, const double* dX, double* E, double* dE);
/* Fit omega to the fractions fr[n I + i] at t_n = n dT, n = 0..k (fr at
 * t_0 fixed): a least-squares minimiser over the box 0 <= omega <= 20 / dT,
 * by Levenberg-Marquardt on omega with the bounds kept by projection, from
 * the one-step regression (see oracle.c).  Returns 0 when the iteration
 * converged, 1 when it stopped after ORC_RATE_FIT_MAX_ITER iterations or
 * could not reduce the damping further (the rates are then a point of lower
 * cost than the start, still used), -1 if k < I, -2 if a rate is not
 * finite. */
#define ORC_RATE_FIT_MAX_ITER 2000
int orc_rate_fit(int I, int k, const double* fr, double dT, double* omega);
/* p_out = expm(A m dT) p_in as m steps of Phi = expm(A dT). */
void orc_rate_propagate(int I, const double* omega, double dT, const double* p_in, int m, double* p_out);

/* -- Parareal ------------------------------------------------------------ */
/* Generic iteration of Eq. mM_parareal_other_k_NEW for classical scalar
 * Parareal (R = M = L = identity): iterates u^k_n, k = 0..K, stored in
 * out[k * (N+1) + n].  F and G are scalar linear maps u -> Fm u + Fa,
 * noise[k * (N+1) + n] is added to F(u^{k-1}_{n-1}) (Lemma 4.1). */
void orc_parareal_scalar(int N, int K, double u0, double Fm, double Fa, double Gm, double Ga,
                         const double* noise, double* out);

typedef struct {
  int sweeps;               /* fine sweeps done */
  int converged;
  double last_change;
  int accepted_total;       /* matching accepted (regions x slices, summed) */
  int rejected_total;
} orc_result;

/* Full MC-moments Parareal (Defs. 3.1, 3.2, 3.4).  Outputs, all optional:
 *   hist     [(max_iter+1)][N+1][2]   global (M, V) of rho^k_n, k = 0..sweeps
 *   macro    [N+1]                    final rho^K_n
 *   parts    [(N+1) * P]              final particle iterates u^K_n
 *   u0_in    optional user initial ensemble (NULL: tag-1 Philox draws) */
int orc_parareal(const orc_problem* pr, const double* u0_in, double* hist, orc_macro* macro,
                 double* parts, orc_result* res);
/* orc_parareal returns 0, or -1 for a plane rotator with more than one region. */

/* Serial reference u_{n+1} = F_n(u_n): stats[n] = R(u_n), n = 0..N;
 * parts (optional) [(N+1) * P]. */
void orc_fine_serial(const orc_problem* pr, const double* u0_in, orc_stats* stats, double* parts);

/* -- adjoint of the serial fine propagator ------------------------------ */
#define ORC_N_THETA 7
/* Gradient of L = sum_{n=1..N} gm[n-1] M_n + gv[n-1] V_n, where (M_n, V_n)
 * are the mean and population variance of the serial fine run at slice end
 * n, with respect to theta = (c3, c1, kappa, c0, B0, B, BE), by the discrete
 * adjoint of the Euler-Maruyama recursion on the same draws (additive,
 * state-proportional and mean-field diffusion alike).  Stores the whole
 * trajectory (P (N n_f + 1) doubles).  moments (optional) receives
 * (M_n, V_n), n = 0..N.  Returns 0, or -1 for the plane rotator. */
int orc_adjoint(const orc_problem* pr, const double* u0_in, const double* gm, const double* gv,
                double grad[ORC_N_THETA], double* moments);
/* L = sum_n (M_n - m_tgt[n-1])^2 + (V_n - v_tgt[n-1])^2 and its gradient. */
int orc_adjoint_loss(const orc_problem* pr, const double* u0_in, const double* m_tgt,
                     const double* v_tgt, double grad[ORC_N_THETA], double* loss);

#ifdef __cplusplus
}
#endif
#endif
