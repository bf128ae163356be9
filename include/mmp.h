/*
 * mmp.h -- C-ABI of the GB300 (sm_103a) MC-moments micro-macro Parareal
 * library libmmp.so (Bossuyt, Vandewalle, Samaey, arXiv 2310.11365).
 *
 * The library runs the data-parallel hot path of the method on one GPU:
 * the Euler-Maruyama fine propagator of a P-particle mean-field ensemble
 * (Sec. 1.2 Eq. Euler_Maruyama) for all Parareal slices at once, fused with
 * the restriction (Sec. 3.4, Eq. multimodal_R) and the matching
 * (Eq. multimodal_M), and the sequential coarse moment-ODE sweep with the
 * Parareal iterator (Eq. mM_parareal_other_k_NEW, Defs. 3.1, 3.2, 3.4).
 *
 * Conventions for every call:
 *  - return value: MMP_OK (0) or a negative MMP_ERR_* code; mmp_strerror()
 *    names it.  Arguments are checked on the host before any launch.
 *  - memory: the library allocates no device memory.  The caller passes one
 *    device workspace (size from mmp_workspace_size) and owns it; the
 *    context only records pointers.  Every device workspace (context,
 *    adjoint, autotune) starts on a 256-byte boundary, as cudaMalloc's and
 *    PyTorch's allocations do; a NULL, misaligned or too small workspace is
 *    MMP_ERR_WORKSPACE, returned before any device work.  Host pointers
 *    passed in are read or written before the call returns.
 *  - streams: `stream` is a cudaStream_t (passed as void*); all device work
 *    of a context is issued on it, in order.  Calls documented as
 *    "synchronising" wait for that stream before they return.
 *  - layout: particle ensembles are contiguous arrays of P values, double
 *    (MMP_FP64) or float (MMP_MIXED), 16-byte aligned.
 */
#ifndef MMP_H
#define MMP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MMP_OK 0
#define MMP_ERR_INVALID_ARG (-1) /* a descriptor or argument is out of range  */
#define MMP_ERR_WORKSPACE (-2)   /* workspace missing, misaligned or too small */
#define MMP_ERR_UNSUPPORTED (-3) /* valid but not supported (e.g. too large)   */
#define MMP_ERR_CUDA (-4)        /* a CUDA call failed (see mmp_last_cuda_error) */
#define MMP_ERR_NUMERIC (-5)     /* device saw NaN/Inf or a negative variance   */
#define MMP_ERR_TIMEOUT (-6)     /* a bounded device-side wait gave up          */
#define MMP_ERR_STATE (-7)       /* call out of order (e.g. iterate before lift) */

/* Precision of the particle state.  MMP_FP64: particles, draws and all
 * moments in double.  MMP_MIXED: particles and their normal draws in float;
 * per-step means, restriction moments, the coarse ODE, the Parareal
 * correction, matching parameters and the fraction fit stay in double. */
#define MMP_FP64 0
#define MMP_MIXED 1

/* Parareal variant: Def. 3.1 (one region), Def. 3.2 (per region, with the
 * fractions-unchanged test), Def. 3.4 (Def. 3.2 plus learned fractions:
 * with two regions the fraction of region 0 follows App. H's
 * P(t) = beta + (P(0) - beta) e^{alpha t}; with three or four, all fractions
 * follow dP/dt = A P of Sec. 3.6, the rates fitted by Levenberg-Marquardt on
 * the exact slice ends t_0..t_k, from sweep k = n_regions on). */
#define MMP_UNIMODAL 0
#define MMP_MULTIMODAL 1
#define MMP_LEARNING 2

/* Problem statement (Sec. 1.1 Eq. general_McKean_Vlasov restricted to the
 * class of Eq. SDE_class_1 with f(x) = x):
 *   dX = a(X, E[X]) dt + b(X, E[X]) dW,  X(0) ~ N(m0, s0^2)
 *   a(x, m) = -c3 x^3 + c1 x + kappa m + c0
 *   b(x, m) = B x + BE m + B0
 * (family MMP_FAMILY_POLY), or the plane rotator of Sec. 5 (Example
 * "Unimodal plane rotator", Eq. SDE_plane_rotator; family
 * MMP_FAMILY_ROTATOR):
 *   a(x) = (K/P) sum_q sin(X_q - x) - g sin x = K (S cos x - C sin x) - g sin x,
 *   b = B0,
 * with S, C the ensemble means of sin X and cos X, every particle shifted
 * modulo 2 pi into [-pi, pi] (x - 2 pi floor((x + pi) / (2 pi))) after each
 * Euler-Maruyama step and in the initial ensemble; c3, c1, kappa, c0 are
 * unused and B, BE must be 0; one region.
 * on [0, T] cut into N Parareal slices; each slice takes
 * n_f = ceil(T/(N dt) - 1e-9) Euler-Maruyama steps of h = T/(N n_f).
 * The coarse propagator is the Gaussian-closure moment ODE per region
 * (exact for c3 = 0, Lemma 2.1) integrated by forward Euler with
 * n_c = ceil(T/(N coarse_h) - 1e-9) substeps.  With I = n_regions > 1 the
 * regions are consecutive intervals split at t_1 = threshold < t_2 =
 * threshold2 < t_3 = threshold3 (the first I - 1 of them):
 * D_0 = {x < t_1}, D_i = {t_i <= x < t_{i+1}}, D_{I-1} = {x >= t_{I-1}}.
 * Random numbers: Philox-4x32-10 with key (seed mod 2^32, seed div 2^32)
 * and counter (p div 4, step, slice | tag << 24, problem_tag). */
typedef struct {
  double c3, c1, kappa, c0;  /* drift coefficients                           */
  double B, BE, B0;          /* diffusion coefficients                       */
  double m0, s0;             /* initial law N(m0, s0^2)                      */
  double T;                  /* horizon, > 0                                  */
  int N;                     /* slices, 1..65535                              */
  double dt;                 /* requested fine step, > 0                      */
  long long P;               /* particles, 1 .. 2^31 - 8                      */
  double coarse_h;           /* largest coarse step, > 0                      */
  int n_regions;             /* 1 .. MMP_MAX_REGIONS                          */
  double threshold;          /* t_1, the first region boundary (n_regions > 1)  */
  int variant;               /* MMP_UNIMODAL / MMP_MULTIMODAL / MMP_LEARNING  */
  int precision;             /* MMP_FP64 / MMP_MIXED                          */
  unsigned long long seed;
  unsigned int problem_tag;
  double tol;                /* stop when max_n max(|dM|,|dV|) < tol          */
  int max_iter;              /* at most this many fine sweeps; <= 0 means N   */
  int coarse_model;          /* MMP_COARSE_CLOSURE (0) / _TAYLOR / _SIGMA2 / _SIGMA3 */
  double threshold2;         /* t_2 (n_regions >= 3), > t_1                   */
  double threshold3;         /* t_3 (n_regions = 4), > t_2                    */
  int family;                /* MMP_FAMILY_POLY (0) / MMP_FAMILY_ROTATOR      */
  double K, g;               /* plane rotator: coupling K, pinning g          */
} mmp_problem_desc;

/* Drift families. */
#define MMP_FAMILY_POLY 0
#define MMP_FAMILY_ROTATOR 1

/* Largest n_regions. */
#define MMP_MAX_REGIONS 4

/* Coarse moment models (Sec. 2), each integrated by forward Euler per
 * region with the fractions frozen:
 *   CLOSURE: Gaussian-assumed density with the expectations of the
 *            polynomial drift and diffusion in closed form;
 *   TAYLOR:  the Taylor-expansion model, Eq. moment_model_class_1
 *            (dM = a(M) + a_XX(M) Sigma / 2, dSigma = (2 a_X + b_X^2) Sigma + b^2);
 *   SIGMA2 / SIGMA3: Gaussian-assumed density, Eq. Gaussian_model_McK_V_SDE,
 *            with a 2- or 3-point sigma-point rule;
 *   TAYLOR1: the Taylor model without the Sigma term of the mean,
 *            dM = a(M) (the plane-rotator example's first coarse solver).
 * For the plane rotator the closure takes S = sin M e^{-Sigma/2},
 * C = cos M e^{-Sigma/2} under N(M, Sigma) and Stein's lemma for the
 * variance (dM = -g S, dSigma = 2 Sigma (-K (S^2 + C^2) - g C) + B0^2);
 * the Taylor models take the point mass at M (a_X(M) = -K - g cos M); the
 * sigma-point rules take every expectation, S and C included, from their
 * points. */
#define MMP_COARSE_CLOSURE 0
#define MMP_COARSE_TAYLOR 1
#define MMP_COARSE_SIGMA2 2
#define MMP_COARSE_SIGMA3 3
#define MMP_COARSE_TAYLOR1 4

typedef struct mmp_ctx mmp_ctx;

/* Number of doubles per slice in the moments returned by mmp_get_moments:
 * frac_0, mean_0, var_0, frac_1, mean_1, var_1, M, V, frac_2, mean_2,
 * var_2, frac_3, mean_3, var_3, 0, 0 (the regions past n_regions zero).
 * Region i's triple starts at MMP_MOMENT_REGION(i). */
#define MMP_MOMENT_STRIDE 16
#define MMP_MOMENT_REGION(i) ((i) < 2 ? 3 * (i) : 3 * (i) + 2)
/* Number of doubles per ensemble in restriction records (mmp_fine_serial,
 * mmp_fine, mmp_fine_static): count_0, mean_0, var_0, min_0, max_0,
 * count_1, .., max_1, mean, var, region_flips, input_mean, 0, 0, then
 * count_2, .., max_2, count_3, .., max_3, and six zeros.  Region i's
 * five values start at MMP_STAT_REGION(i). */
#define MMP_STAT_STRIDE 32
#define MMP_STAT_REGION(i) ((i) < 2 ? 5 * (i) : 5 * (i) + 6)

const char* mmp_strerror(int code);
/* Version of the C-ABI: 101 adds up to four regions (threshold2, threshold3;
 * 16-double moment rows, 32-double restriction records), seven-coefficient
 * adjoints (mmp_set_params' n_theta, mmp_adjoint); 102 adds the drift
 * family (family, K, g: the plane rotator) and MMP_COARSE_TAYLOR1.
 * Checkpoints (mmp_get_state) restore only into the same version. */
#define MMP_VERSION 102
int mmp_version(void);
/* Last CUDA error code seen by the library in this process (0 if none). */
int mmp_last_cuda_error(void);

/* Bytes of device workspace needed for n_problems problems. */
int mmp_workspace_size(const mmp_problem_desc* descs, int n_problems, size_t* bytes);

/* Create a context over caller-owned device workspace.  Validates every
 * descriptor, plans the launch shape of the fine kernel per problem and
 * draws the initial ensembles X0 = m0 + s0 z (tag-1 draws) on `stream`.
 * Asynchronous.  The context (a small host object) is freed by
 * mmp_destroy; the workspace stays the caller's. */
int mmp_create(mmp_ctx** ctx, const mmp_problem_desc* descs, int n_problems, void* workspace,
               size_t workspace_bytes, void* stream);
int mmp_destroy(mmp_ctx* ctx);

/* Replace problem `prob`'s initial ensemble by P values (double for
 * MMP_FP64, float for MMP_MIXED) at `u0`, a host pointer if from_host != 0
 * else a device pointer.  Copies before returning (host) or on the stream. */
int mmp_set_initial(mmp_ctx* ctx, int prob, const void* u0, int from_host);

/* Iteration k = 0 (Eq. mM_parareal_0 / generalised form): restriction of
 * u0, sequential coarse sweep rho^0_{n+1} = C_n(rho^0_n) and lifting
 * parameters L(rho) = T(rho, u0).  Asynchronous. */
int mmp_lift(mmp_ctx* ctx);

/* Up to n_iter fine sweeps, each followed by the coarse/iterator sweep
 * (Eq. mM_parareal_other_k_NEW).  Slices already exact (Property 3.3) are
 * not recomputed.  Synchronising: reads each problem's convergence word
 * after every sweep; *all_converged (optional) is set when every problem
 * met its tolerance or reached max_iter. */
int mmp_iterate(mmp_ctx* ctx, int n_iter, int* all_converged);

/* mmp_lift followed by mmp_iterate until every problem stops.
 * Synchronising.  *sweeps_out (optional): the largest sweep count. */
int mmp_run(mmp_ctx* ctx, int* sweeps_out);

/* Per-problem state after the last sweep.  Synchronising.
 * dev_err: device status word (0 or an MMP_ERR_* code). */
int mmp_status(mmp_ctx* ctx, int prob, int* sweeps, int* converged, double* last_change,
               int* dev_err);

/* Macro state rho^K_n, n = 0..N, to host memory `out`
 * [(N+1) * MMP_MOMENT_STRIDE].  Synchronising. */
int mmp_get_moments(mmp_ctx* ctx, int prob, double* out);

/* Particle iterate u^K_n of slice end n (0..N), i.e. the matched fine
 * output, P values to `dst` (host if to_host != 0, else device).
 * Synchronising when to_host. */
int mmp_get_particles(mmp_ctx* ctx, int prob, int n, void* dst, int to_host);

/* Serial reference u_{n+1} = F_n(u_n) from the same u0 and the same
 * draws, for slices 0 .. n_end-1 (n_end <= 0 or > N means N); restriction
 * records of u_0..u_{n_end} to host `stats_out` [(n_end+1) * MMP_STAT_STRIDE]
 * (may be NULL).  If parts_dev is not NULL it receives u_{n_end} (device).
 * Uses the same launch shape as the Parareal sweeps, so the first k slice
 * ends after k sweeps match it bit for bit.  Synchronising. */
int mmp_fine_serial(mmp_ctx* ctx, int prob, int n_end, double* stats_out, void* parts_dev);

/* Launch shape chosen for problem `prob`: quads of 4 particles held per
 * thread, CTAs per slice (one group barrier spans them), the largest number
 * of slices one launch runs concurrently, and whether the particles live in
 * shared memory (1) or registers (0) between steps.  Any pointer may be
 * NULL. */
int mmp_get_plan(mmp_ctx* ctx, int prob, int* quads_per_thread, int* ctas_per_slice,
                 int* max_concurrent_slices, int* particles_in_shared);

/* Replace problem `prob`'s drift and diffusion coefficients by
 * theta = (c3, c1, kappa, c0, B0) (n_theta = 5; B and BE unchanged) or
 * (c3, c1, kappa, c0, B0, B, BE) (n_theta = 7); host doubles, finite, else
 * MMP_ERR_INVALID_ARG.  The launch shape does not depend on them, so nothing
 * is re-planned.  Making B or BE nonzero (or both zero) switches the fine
 * kernel between its additive-noise and general forms: MMP_ERR_UNSUPPORTED
 * (nothing changed) in a batched context or if the other form does not fit
 * the problem's launch shape.  A recorded adjoint forward run is
 * invalidated. */
int mmp_set_params(mmp_ctx* ctx, int prob, const double* theta, int n_theta);

/* Adjoint of the serial fine propagator F_{N-1} o ... o F_0 (the run the
 * Parareal iteration converges to exactly, Property 3.3).  The paper has no
 * adjoint; this is the reverse mode of its Euler-Maruyama recursion
 * (Sec. 1.2) with drift a = -c3 x^3 + c1 x + kappa m + c0 and diffusion
 * b = B x + BE m + B0, mean-field coupling included, for calibrating the
 * model coefficients to moment targets.
 *
 * mmp_adjoint_workspace_size: bytes of caller-owned device workspace for a
 * checkpoint every `ckpt_every` fine steps: one particle row per checkpoint,
 * 3 recorded values per step, two buffers of ckpt_every + 1 state rows and
 * two of ckpt_every draw rows (the reverse sweep replays the next segment
 * into the second buffers while it reverses one; the draw rows are used
 * with B or BE nonzero, additive noise regenerating its draws; the size
 * does not depend on the form).
 *
 * mmp_adjoint_forward: runs the serial fine propagation from u0 with the
 * current coefficients, recording checkpoints and per-step mean-field values
 * into `ws`; writes the slice-end moments (M_n, V_n), n = 0..N, to host
 * `moments_out` [(N+1) * 2] (may be NULL).  Synchronising.
 *
 * mmp_adjoint_backward: given cotangents gm[n-1] = dL/dM_n, gv[n-1] = dL/dV_n
 * for n = 1..N (host, N doubles each), writes
 * dL/d(c3, c1, kappa, c0, B0, B, BE) to host `grad_out` [MMP_N_THETA]
 * (the derivatives in B and BE are those at the current values, zero
 * included).  Needs the workspace of the last forward run of this problem
 * (else MMP_ERR_STATE).  Each segment of ckpt_every steps is recomputed
 * from its checkpoint with the same draws and reversed with one group
 * exchange of the adjoint per step (one sum for additive noise; with B or
 * BE nonzero also the sums that form Z_j = sum_p lambda_{j+1,p} xi_{j,p}).
 * Synchronising. */
#define MMP_N_THETA 7
int mmp_adjoint_workspace_size(mmp_ctx* ctx, int prob, int ckpt_every, size_t* bytes);
int mmp_adjoint_forward(mmp_ctx* ctx, int prob, int ckpt_every, void* ws, size_t ws_bytes,
                        double* moments_out);
int mmp_adjoint_backward(mmp_ctx* ctx, int prob, const double* gm, const double* gv, void* ws,
                         size_t ws_bytes, double* grad_out);

/* The loss L = sum_{n=1..N} (M_n - m_tgt[n-1])^2 + (V_n - v_tgt[n-1])^2 of
 * the serial fine run's slice-end moments and its gradient in one call:
 * mmp_adjoint_forward, the cotangents 2 (M_n - m_tgt), 2 (V_n - v_tgt) on the
 * host, then mmp_adjoint_backward.  m_tgt, v_tgt: host, N doubles each;
 * grad_out: host, MMP_N_THETA doubles; loss: host, may be NULL.  The same
 * workspace rules and errors as the two calls.  Synchronising. */
int mmp_adjoint(mmp_ctx* ctx, int prob, const double* m_tgt, const double* v_tgt, int ckpt_every, void* ws,
                size_t ws_bytes, double* grad_out, double* loss);

/* Device-time accounting.  With timing on, the library records CUDA
 * events on the context stream around every fine-kernel launch and reads
 * them at its synchronisation points.  mmp_timing reports, since the last
 * reset: fine-kernel milliseconds and launches, the particle-steps those
 * launches performed, and the number of other library kernel launches
 * (driver, initial ensemble).  Any output pointer may be NULL. */
int mmp_set_timing(mmp_ctx* ctx, int on);
int mmp_timing(mmp_ctx* ctx, int reset, double* fine_ms, long long* fine_launches,
               double* fine_particle_steps, long long* other_launches);

/* Checkpoint and resume of a run (for instance across a process restart).
 * The state is the contents of the context's workspace (particle buffers,
 * macro states, matching records, control blocks) and each problem's host
 * view of the iteration (sweeps done, finished, last change, which buffer
 * holds each slice's latest output).  mmp_state_size gives its bytes;
 * mmp_get_state writes it to host memory `dst` (caller-owned, that many
 * bytes); mmp_set_state restores it from host memory `src` (that many bytes)
 * into a context created with the same
 * problem descriptions and the same launch plans, at any workspace address:
 * the next mmp_iterate continues exactly as the saved context would have,
 * bit for bit.  Adjoint recordings are not part of the state.  Both
 * synchronise.  Errors: MMP_ERR_INVALID_ARG (NULL), MMP_ERR_STATE (the blob
 * belongs to other problems, plans or library version, or holds an iteration
 * state no run reaches; the context is then left unchanged), MMP_ERR_CUDA.  The
 * paper has no counterpart (a property of this library). */
int mmp_state_size(mmp_ctx* ctx, size_t* bytes);
int mmp_get_state(mmp_ctx* ctx, void* dst);
int mmp_set_state(mmp_ctx* ctx, const void* src);

/* Batched sweeps of a context with several problems (one cooperative
 * launch per sweep over every unconverged problem's slices; the task list
 * is built on the device, so sweeps run back to back).  batched (may be
 * NULL) = 1 if the context batches its problems; graph (may be NULL) = 1
 * if its sweeps replay from a captured CUDA graph (known after the first
 * mmp_iterate; 0 when MMP_BATCH_GRAPH=0 or the runtime refused the
 * capture, in which case the same work is enqueued directly). */
int mmp_batch_info(mmp_ctx* ctx, int* batched, int* graph);

/* Measured launch shapes.  The planner chooses the fine kernel's quads
 * per thread (4 particles each; this fixes the CTAs per slice G =
 * ceil(ceil(P/4) / (256 nq)) and the slices resident at once) from a cost
 * model; mmp_autotune measures instead.  For each candidate count
 * (`candidates`, n_candidates entries; NULL: every count 1..32 for mixed,
 * 1..16 for FP64) it times, with CUDA events after one warm-up launch, a
 * fine launch of *desc's model and P with probe_steps Euler-Maruyama steps
 * per slice (0: min(n_f, 64)) from the problem's seeded initial ensemble,
 * over max(N, two full waves of resident slices) slices, i.e. the
 * throughput with the GPU full, on `stream` (synchronising).  best_nq receives the fastest candidate;
 * rates (may be NULL; n_candidates entries, or 32 / 16 for NULL
 * candidates) the particle-steps per second of each (0 for a candidate that
 * does not fit).  `workspace` (device, mmp_autotune_workspace_size bytes,
 * caller-owned) holds the ensemble and the exchange scratch.  Errors:
 * MMP_ERR_INVALID_ARG, MMP_ERR_WORKSPACE, MMP_ERR_UNSUPPORTED (no
 * candidate fits), MMP_ERR_TIMEOUT, MMP_ERR_CUDA.
 *
 * mmp_set_tuning adds a process-wide entry: problems of `precision` with
 * p_lo <= P <= p_hi are planned with the largest reachable count of at most
 * quads_per_thread (later entries win; MMP_FINE_NQ still overrides).
 * quads_per_thread = 0 removes every entry of that precision.  Contexts
 * created afterwards use the table for single problems whose N slices fill
 * the resident CTAs at that count (otherwise the cost model, which favours
 * more CTAs per slice, decides).
 *
 * mmp_set_batch_nq sets the cap on quads per thread of batched contexts of
 * `precision` created afterwards (each problem takes the most quads per
 * thread up to the cap; 0 restores the default 26 mixed / 13 FP64;
 * MMP_BATCH_NQ still overrides).  The batched kernel sizes its shared
 * memory for the largest count in the batch, so the cap also fixes its
 * occupancy; the Python helper tune.tune_batch measures it on a sample of
 * the batch.  The paper has no counterpart (a property of this library). */
int mmp_autotune_workspace_size(const mmp_problem_desc* desc, size_t* bytes);
int mmp_autotune(const mmp_problem_desc* desc, const int* candidates, int n_candidates, int probe_steps,
                 void* workspace, size_t bytes, void* stream, int* best_nq, double* rates);
int mmp_set_tuning(int precision, long long p_lo, long long p_hi, int quads_per_thread);
int mmp_set_batch_nq(int precision, int quads_per_thread);

/* One fine propagation F_n of an explicit ensemble (no matching):
 * reads P values at u_in (device), writes F_n(u_in) to u_out (device,
 * may not alias u_in) and its restriction record to stats_out (host,
 * MMP_STAT_STRIDE doubles, may be NULL).  `n` is the slice index used
 * for the draws.  Synchronising. */
int mmp_fine(mmp_ctx* ctx, int prob, int n, const void* u_in, void* u_out, double* stats_out);

/* Philox-4x32-10 on n counters: ctr (device, 4n uint32), key (host, 2
 * uint32) -> out (device, 4n uint32).  Asynchronous on `stream`. */
int mmp_philox(const unsigned int* ctr, const unsigned int* key, unsigned int* out, long long n,
               void* stream);

/* The normals the fine propagator uses for (tag, step j, slice n):
 * out[p] for p < count (device, double or float per `precision`, aligned
 * to its element; count <= 2^34; tag < 256; n < 2^24, else
 * MMP_ERR_INVALID_ARG).  Asynchronous on `stream`. */
int mmp_normals(const mmp_problem_desc* desc, int tag, unsigned int j, unsigned int n,
                long long count, void* out, void* stream);

/* Counters of the device-side iteration of problem `prob` (the paper has
 * no counterpart; for diagnosing convergence): out[0] regions accepted by
 * the iterator (Defs. 3.1, 3.2), summed over slices and sweeps since the
 * lift; out[1] regions rejected; out[2] 1 if the last sweep used learned
 * fractions (Def. 3.4); out[3], out[4] the two-region fit (alpha, beta) of
 * that sweep; out[5] the change max_n max(|dM|, |dV|) of that sweep.  out:
 * host, 6 doubles.  Synchronising. */
int mmp_sweep_info(mmp_ctx* ctx, int prob, double* out);

/* Throughput of fused multiply-adds on this device in FP64 (precision
 * MMP_FP64) or FP32 (MMP_MIXED), in TFLOP/s (2 flops per FMA): one launch of
 * 4 CTAs per SM whose threads run 8 independent FMA chains, timed with CUDA
 * events after a warm-up launch.  The plain FP64 form is measured against
 * it (the paper has no counterpart).  ws: device, 256-byte aligned, 8 bytes
 * at least (a sink the kernel never writes in practice).  Synchronising. */
int mmp_probe_fma(int precision, void* ws, size_t ws_bytes, void* stream, double* tflops);

/* Throughput, in particle-steps/s, of the fine step's arithmetic without the
 * cross-CTA exchange of the mean: the mixed-precision additive-noise
 * Euler-Maruyama step (Eq. Euler_Maruyama with the draws of Philox-4x32-10
 * and Box-Muller, the per-step sum of the particles) evaluated by the same
 * device functions as the fine kernel, two 256-thread CTAs per SM, on
 * particles that stay on chip for every step.  form 0: 4 quads (16
 * particles) per thread in registers, no synchronisation; form 1: 26 quads
 * per thread in shared memory, the fine kernel's layout, with a warp
 * butterfly and a CTA barrier every step.  One launch of about 2.5e10
 * particle-steps timed with CUDA events after a warm-up launch; the fused
 * fine kernel's step loop is measured against it (the paper has no
 * counterpart).  ws: device, 256-byte aligned, 8 bytes at least (a sink the
 * kernel never writes in practice).  MMP_ERR_INVALID_ARG for another form
 * or a null result pointer.  Synchronising. */
int mmp_probe_step(int form, void* ws, size_t ws_bytes, void* stream, double* particle_steps_per_s);

/* One problem's slices on several GPUs.  Within a Parareal iteration the
 * fine propagations of the slices are independent (Sec. 3.1: the parallel
 * step of Parareal), so the slices can be split into contiguous blocks, one
 * per GPU (rank), each rank holding a context over the whole problem.  A
 * sweep k (Eq. mM_parareal_other_k_NEW) then runs in two phases:
 *
 * mmp_sweep_fine: the fine propagations F_n(u^{k-1}_n), matching fused, of
 *   the slices n in [max(k - 1, n_lo), n_hi) (slices before k - 1 are exact,
 *   Property 3.3).  Slice n reads the fine output of slice n - 1 of sweep
 *   k - 1, so a rank whose block starts at n_lo >= k needs that row from the
 *   previous rank first (mmp_set_output).  Asynchronous.  Not for batched
 *   contexts (MMP_ERR_UNSUPPORTED); MMP_ERR_STATE before mmp_lift, after the
 *   problem stopped, or when a fine phase already waits for its driver.
 * mmp_sweep_coarse: the driver of sweep k (the sequential coarse sweep, the
 *   iterator, the matching records, the convergence test) over all N slices,
 *   from the restriction records of all of them, which must therefore be in
 *   place (mmp_set_records).  On every rank the same inputs give the same
 *   results bit for bit.  *done (optional) = 1 when the problem stopped.
 *   Synchronising; returns a device-side error like mmp_iterate.
 * mmp_get_records / mmp_set_records: restriction records of the fine
 *   outputs of slices [n_lo, n_hi) (MMP_STAT_STRIDE doubles each, host
 *   memory), to gather them on every rank between the phases.  Synchronising.
 * mmp_get_output / mmp_set_output: the P values of the fine output of slice
 *   n written by the latest fine phase (dst / src in host memory if to_host /
 *   from_host, else device memory; host copies synchronise).  After sweep k
 *   the rank that propagated slice n_hi - 1 sends it to the rank whose block
 *   starts at n_hi, which sets it before its fine phase of sweep k + 1.
 *   MMP_ERR_STATE before the first fine phase.
 * mmp_iterate is refused (MMP_ERR_STATE) while a fine phase waits for its
 * driver, and so is mmp_get_state. */
int mmp_sweep_fine(mmp_ctx* ctx, int prob, int n_lo, int n_hi);
int mmp_sweep_coarse(mmp_ctx* ctx, int prob, int* done);
int mmp_get_records(mmp_ctx* ctx, int prob, int n_lo, int n_hi, double* out);
int mmp_set_records(mmp_ctx* ctx, int prob, int n_lo, int n_hi, const double* in);
int mmp_get_output(mmp_ctx* ctx, int prob, int n, void* dst, int to_host);
int mmp_set_output(mmp_ctx* ctx, int prob, int n, const void* src, int from_host);

/* Self-test of the failure detection of the fine kernel's group exchange
 * (the paper has no counterpart; a property of the library).  Launches one
 * CTA of a group of G CTAs on `stream`; it runs the kernel's own group
 * reduction (channel 0: records behind release/acquire epoch flags, as the
 * restriction and FP64 particles use; channel 1: the tagged 8-byte step
 * words of float particles), but no peer ever publishes, so with G >= 2
 * every bounded wait runs out after limit_ms milliseconds, sets the timeout
 * bit (1) of the status word and lets the kernel return; nothing faults or
 * hangs, and the device stays usable.  ws: device scratch, 256-byte
 * aligned, at least G * 548 + 4 bytes (publication slots, step words, epoch
 * flags, status word), caller-owned.  Synchronising.  *status_out (may be
 * NULL) receives the status word.  Returns MMP_ERR_TIMEOUT when the wait ran
 * out (G >= 2), MMP_OK when nothing had to be waited for (G = 1);
 * MMP_ERR_INVALID_ARG for a channel other than 0 or 1, G outside 1..1024 or
 * limit_ms outside [1, 10000]; MMP_ERR_WORKSPACE for a NULL, misaligned or
 * short ws. */
int mmp_probe_wait(int channel, int G, double limit_ms, void* ws, size_t ws_bytes, void* stream,
                   unsigned* status_out);

/* One fine propagation F_n of an explicit ensemble, like mmp_fine, for
 * callers that cannot allocate device memory where they call it: code
 * inside a host application or framework that owns the GPU's memory through
 * its own allocator and gives plugins no way to reserve more, and
 * latency-bound loops in which a cudaMalloc or cudaFree (which can
 * synchronise the whole device) is not acceptable.  They own their
 * ensembles; what they cannot provide is the scratch of the kernel's
 * cross-CTA mean reduction.  The paper has no counterpart; this is a
 * property of the library.
 *
 * No context, no workspace, no allocation: that scratch is one fixed array
 * inside libmmp.so (about 650 KB of device memory, held on every GPU that
 * loads the library until the process exits), serving at most
 * MMP_STATIC_MAX_CTAS CTAs per slice; larger problems (above roughly 9.9e6
 * float or 4.9e6 double particles, depending on the launch shape) return
 * MMP_ERR_UNSUPPORTED before any device work.  The first call on a device
 * looks up the array's device address (once per device, kept for the life
 * of the process); make that first call before any stream capture.  After a
 * cudaDeviceReset the kept address is stale: resetting a device while this
 * entry point is in use is not supported.
 *
 * desc      problem (only one slice is propagated; n in 0..N-1 selects the
 *           draws)
 * u_in      device, P values (double for MMP_FP64, float for MMP_MIXED),
 *           16-byte aligned; u_out device, P values, must not alias u_in
 * stats_dev device, MMP_STAT_STRIDE doubles or NULL: the restriction of
 *           F_n(u_in); element 14 receives the device status bits
 *           (0 = ok, 1 = a bounded wait gave up, 2 = non-finite result).
 *           This is the only place device-side errors are reported: with
 *           stats_dev NULL a timed-out or non-finite propagation is not
 *           seen by the caller.
 * stream    cudaStream_t; asynchronous.
 * Every call shares the array and leaves its contents behind: the call
 * clears what must start at zero, and calls that overlap on the GPU (on
 * different streams, or from different host threads) race on it. */
#define MMP_STATIC_MAX_CTAS 1216
int mmp_fine_static(const mmp_problem_desc* desc, int n, const void* u_in, void* u_out,
                    double* stats_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif
