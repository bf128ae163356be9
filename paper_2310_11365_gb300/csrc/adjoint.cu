// adjoint.cu -- reverse-mode derivative of the serial fine propagator
// F_{N-1} o ... o F_0 (the Euler-Maruyama particle system of Sec. 1.2 with
// the mean field m_j = (1/P) sum_q x_{j,q}) with respect to the model
// coefficients (c3, c1, kappa, c0, B0), for cotangents on the slice-end
// means and population variances.
//
// With lambda_j = dL/dx_j:
//   lambda_{j,q} = lambda_{j+1,q} (1 + h a_x(x_{j,q})) + (h kappa / P) sum_p lambda_{j+1,p}
//                  + [slice-end loss at x_j],  a_x(x) = -3 c3 x^2 + c1,
//   dL/dc3 = -h sum_{j,p} lambda_{j+1,p} x_{j,p}^3,  dL/dc1 = h sum lambda_{j+1} x_j,
//   dL/dkappa = h sum_j m_j S_j,  dL/dc0 = h sum_j S_j,  S_j = sum_p lambda_{j+1,p},
//   dL/dB0 = sqrt(h) sum lambda_{j+1} xi_j,
// and a cotangent (gm, gv) on (M_n, V_n) injects gm/P + gv (2/P)(x - M_n).
//
// The forward run (the fine kernel with recording on) leaves a particle
// checkpoint every c steps and the per-step uniforms it used (the mean m_j,
// the common shift d_j = h (kappa m_j + c0) and the noise amplitude).  Per segment,
// in reverse: each thread recomputes its own particles over the c steps from
// the checkpoint (no reduction is needed: the means are recorded), storing
// states and draws, then sweeps backward with one group sum per step, in
// the shift form that lets that sum run one step behind the sweep (below).
// The replay evaluates the step exactly as the forward kernel did, so it
// reproduces the forward states.
#include <cmath>

#include "adjoint.cuh"
#include "fine_kernel.cuh"

namespace mmp {

template <typename R>
__global__ void __launch_bounds__(kTPB, 2) k_adjoint(const AdjointArgs a) {
  __shared__ GroupShared sh;
  const int G = a.G;
  const int g = blockIdx.x;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int qb = (int)(((long long)a.Q * g) / G);
  const int qe = (int)(((long long)a.Q * (g + 1)) / G);
  const int span = qe - qb - tid;
  const int nq = span <= 0 ? 0 : min(a.nq, (span + kTPB - 1) / kTPB);
  const int qlast = a.Q - 1;
  const int plast = (int)(a.P - 4LL * qlast);

  Group grp;
  grp.part = a.partials;
  grp.flags = a.flags;
  grp.tags = a.tags;
  grp.status = a.status;
  grp.limit_ns = a.wait_limit_ns;
  grp.G = G;
  grp.g = g;
  grp.epoch = 0;
  grp.tight_polls = G <= a.sms ? kTightPolls : 0;
  if (tid == 0) sh.abort = 0;

  QuadStore<R, 0> lam;  // lambda of this thread's quads, in shared memory
  lam.bind();
  for (int i = 0; i < nq; ++i) {
    const R zero[4] = {0, 0, 0, 0};
    lam.put(i, zero);
  }

  // coefficients rounded once per CTA (keeps FP64 conversions out of the loops)
  if (sizeof(R) == 4 && tid == 0) {
    sh.cf[0] = (float)a.h;
    sh.cf[1] = (float)a.nc3;
    sh.cf[2] = (float)a.c1;
    sh.cf[3] = (float)(a.kappa * a.h / (double)a.P);
    sh.cf[4] = (float)a.sqrt_h;
    sh.cf[5] = (float)(a.h * a.nc3);
    sh.cf[6] = (float)(a.h * a.c1);
  }
  __syncthreads();
  const bool fl = sizeof(R) == 4;
  const R h = fl ? (R)sh.cf[0] : (R)a.h;
  const R nc3 = fl ? (R)sh.cf[1] : (R)a.nc3;
  const R c1 = fl ? (R)sh.cf[2] : (R)a.c1;
  const R kh_p = fl ? (R)sh.cf[3] : (R)(a.kappa * a.h / (double)a.P);
  const R sqh = fl ? (R)sh.cf[4] : (R)a.sqrt_h;
  const R hn3 = fl ? (R)sh.cf[5] : (R)(a.h * a.nc3);  // as the forward rounds them
  const R hc1 = fl ? (R)sh.cf[6] : (R)(a.h * a.c1);
  const R* uni = (const R*)a.uni;
  R* segx = (R*)a.segx;
  R* segz = (R*)a.segz;

  Acc<R> acc3, acc1, accb;         // -h x^3, h x, sqrt(h) xi terms
  double acc_k = 0.0, acc_c0 = 0.0;  // h m_j S_j, h S_j (thread 0 of CTA 0)
  R s_next = (R)0;                   // pending shift s_{j+1} of lambda_{j+1}

  auto zero_tail = [&](int q, R v[4]) {
    if (q == qlast) {
      if (plast < 4) v[3] = (R)0;
      if (plast < 3) v[2] = (R)0;
      if (plast < 2) v[1] = (R)0;
    }
  };
  // slice-end cotangent at global step j (a multiple of nf, j >= 1)
  auto inject = [&](long long j, int q, const R x[4], R l[4]) {
    const int n = (int)(j / a.nf);
    const double M = a.mom[(size_t)n * kStat + 10];
    const R ca = (R)(a.gm[n - 1] / (double)a.P);
    const R cb = (R)(2.0 * a.gv[n - 1] / (double)a.P);
    const R Mr = (R)M;
#pragma unroll
    for (int w = 0; w < 4; ++w) l[w] += ca + cb * (x[w] - Mr);
    zero_tail(q, l);
  };

  for (int seg = a.n_seg - 1; seg >= 0; --seg) {
    const long long j0 = (long long)seg * a.c;
    const long long j1 = min(a.J, j0 + a.c);
    const int L = (int)(j1 - j0);
    // ---- replay the segment from its checkpoint (thread-private) --------
    const R* ck = (const R*)a.ckpt + (size_t)seg * a.pitch;
    for (int i = 0; i < nq; ++i) {
      const int q = qb + tid + i * kTPB;
      R x[4];
      Quad<R>::load(ck + 4 * (size_t)q, x);
      for (int jj = 0; jj < L; ++jj) {
        const long long j = j0 + jj;
        Quad<R>::store(segx + (size_t)jj * a.pitch + 4 * (size_t)q, x);
        R nr[2], c[2], sn[2];
        normals4_polar<R>(philox4x32_10(rng_counter((uint32_t)q, (uint32_t)(j % a.nf), (uint32_t)(j / a.nf), 0u,
                                                    a.ptag), a.key0, a.key1), nr, c, sn);
        const R z[4] = {mulR(nr[0], c[0]), mulR(nr[0], sn[0]), mulR(nr[1], c[1]), mulR(nr[1], sn[1])};
        Quad<R>::store(segz + (size_t)jj * a.pitch + 4 * (size_t)q, z);
        const R d = uni[3 * j + 1];    // h (kappa m_j + c0) as the forward used it
        const R amp = uni[3 * j + 2];  // B0 sqrt(h) as the forward used it
        em_partial_pair(x[0], x[1], nr[0], c[0], sn[0], hn3, hc1, amp);
        em_partial_pair(x[2], x[3], nr[1], c[1], sn[1], hn3, hc1, amp);
#pragma unroll
        for (int w = 0; w < 4; ++w) x[w] = addR(x[w], d);
        zero_tail(q, x);
      }
      Quad<R>::store(segx + (size_t)L * a.pitch + 4 * (size_t)q, x);
    }
    // ---- backward through the segment ----------------------------------
    // Shift form of the reverse recursion: lambda_j = mu_j + s_j with
    //   mu_j = lambda_{j+1} (1 + h a_x(x_j)) [+ slice-end injection at x_j],
    //   s_j  = (h kappa / P) S_j,  S_j = sum lambda_{j+1} = sum mu_{j+1} + P s_{j+1},
    // so the group sum of mu_j published at the end of reverse step j is
    // first needed at the end of step j - 1 (the exchange is one step
    // behind, as in the forward).  `lam` holds mu, `s_next` the pending shift.
    if (j1 == a.J) {
      // lambda_J: the last slice end's injection alone (s_J = 0); its sum is epoch 0
      R part = (R)0;
      for (int i = 0; i < nq; ++i) {
        const int q = qb + tid + i * kTPB;
        R x[4], l[4] = {0, 0, 0, 0};
        Quad<R>::load(segx + (size_t)L * a.pitch + 4 * (size_t)q, x);
        inject(a.J, q, x, l);
        lam.put(i, l);
        part = addR(part, addR(addR(l[0], l[1]), addR(l[2], l[3])));
      }
      step_sum_warp<R>(sh, 1, part);
      __syncthreads();
      if (warp == 0) {
        const typename StepSum<R>::T cta = step_sum_cta<R>(sh, 1);
        if (lane == 0) StepSum<R>::publish(grp, 0u, cta);
      }
      grp.epoch = 1u;
    }
    for (int jj = L - 1; jj >= 0; --jj) {
      const long long j = j0 + jj;
      const unsigned ej = (unsigned)(a.J - j);  // epoch of sum mu_j
      const bool end_j = j > 0 && j % a.nf == 0;
      R part = (R)0, p3 = (R)0, p1 = (R)0, pb = (R)0;
      for (int i = 0; i < nq; ++i) {
        const int q = qb + tid + i * kTPB;
        R l[4], x[4], z[4];
        lam.get(i, l);
        Quad<R>::load(segx + (size_t)jj * a.pitch + 4 * (size_t)q, x);
        Quad<R>::load(segz + (size_t)jj * a.pitch + 4 * (size_t)q, z);
#pragma unroll
        for (int w = 0; w < 4; ++w) l[w] = addR(l[w], s_next);  // lambda_{j+1}
        zero_tail(q, l);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          // step j's parameter partials, then mu_j
          p3 -= l[w] * x[w] * x[w] * x[w];
          p1 += l[w] * x[w];
          pb += l[w] * z[w];
          const R ax = fmaR((R)3 * nc3, x[w] * x[w], c1);  // -3 c3 x^2 + c1
          l[w] = mulR(l[w], fmaR(h, ax, (R)1));
        }
        if (end_j) inject(j, q, x, l);
        zero_tail(q, l);
        lam.put(i, l);
        part = addR(part, addR(addR(l[0], l[1]), addR(l[2], l[3])));
      }
      acc3.add(h * p3);
      acc1.add(h * p1);
      accb.add(sqh * pb);
      // warp 0 reads sum mu_{j+1} (epoch ej - 1, published a step ago) before
      // the barrier and publishes sum mu_j (epoch ej) after it
      step_sum_warp<R>(sh, jj & 1, part);
      if (warp == 0) {
        typename StepSum<R>::T sum;
        const bool ok = StepSum<R>::fetch(grp, ej - 1u, sum);
        if (lane == 0) {
          StepSum<R>::gsum(sh, jj & 1) = sum;
          if (!ok) sh.abort = 1;
        }
      }
      __syncthreads();
      if (sh.abort) return;
      const typename StepSum<R>::T sm = StepSum<R>::gsum(sh, jj & 1);
      double S_d;
      R S;
      if constexpr (sizeof(R) == 4) {
        S = addR(addR(sm.x, sm.y), mulR((R)a.P, s_next));
        S_d = (double)sm.x + (double)sm.y + (double)a.P * (double)s_next;
      } else {
        S = addR(sm, mulR((R)a.P, s_next));
        S_d = S;
      }
      if (g == 0 && tid == 0) {
        acc_k += a.h * (double)uni[3 * j] * S_d;
        acc_c0 += a.h * S_d;
      }
      s_next = mulR(kh_p, S);  // s_j, pending on lambda_j
      if (warp == 0) {
        const typename StepSum<R>::T cta = step_sum_cta<R>(sh, jj & 1);
        if (lane == 0) StepSum<R>::publish(grp, ej, cta);
      }
      grp.epoch = ej + 1u;
    }
  }
  // ---- reduce the parameter partials over the group (FP64) -------------
  {
    double v[5] = {acc3.get(), acc1.get(), acc_k, acc_c0, accb.get()};
    warp_reduce_to_shared<5>(sh, v, 0u, 0u);
    __syncthreads();
    if (sh.abort) return;
    const unsigned e = grp.epoch++;
    if (warp == 0 && !group_finish<5>(sh, grp, e, 0u, 0u) && lane == 0) sh.abort = 1;
    __syncthreads();
    if (sh.abort) return;
    if (g == 0 && tid == 0) {
      for (int k = 0; k < 5; ++k) a.grad[k] = sh.tot[k];
      if (!(fabs(sh.tot[0]) < INFINITY) || !(fabs(sh.tot[4]) < INFINITY)) atomicOr(a.status, kStatusNumeric);
    }
  }
}

const void* adjoint_kernel(int precision) {
  return precision == MMP_MIXED ? (const void*)k_adjoint<float> : (const void*)k_adjoint<double>;
}

size_t adjoint_smem_bytes(int precision, int nq) {
  return (size_t)nq * kTPB * 4 * (precision == MMP_MIXED ? sizeof(float) : sizeof(double));
}

cudaError_t launch_adjoint(int precision, const AdjointArgs& args, cudaStream_t stream) {
  AdjointArgs copy = args;
  void* params[] = {&copy};
  return cudaLaunchCooperativeKernel(adjoint_kernel(precision), dim3(args.G), dim3(kTPB), params,
                                     adjoint_smem_bytes(precision, args.nq), stream);
}

}  // namespace mmp
