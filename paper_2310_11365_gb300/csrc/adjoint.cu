// adjoint.cu -- reverse-mode derivative of the serial fine propagator
// F_{N-1} o ... o F_0 (the Euler-Maruyama particle system of Sec. 1.2,
//   x_{j+1} = x_j + h a(x_j, m_j) + sqrt(h) b(x_j, m_j) xi_j,
//   a = -c3 x^3 + c1 x + kappa m + c0,  b = B x + BE m + B0,
// with the mean field m_j = (1/P) sum_q x_{j,q}) with respect to the model
// coefficients (c3, c1, kappa, c0, B0, B, BE), for cotangents on the
// slice-end means and population variances.
//
// With lambda_j = dL/dx_j, S_j = sum_p lambda_{j+1,p}, Z_j = sum_p lambda_{j+1,p} xi_{j,p}:
//   lambda_{j,q} = lambda_{j+1,q} (1 + h a_x(x_{j,q}) + sqrt(h) B xi_{j,q})
//                  + (h kappa S_j + sqrt(h) BE Z_j) / P + [slice-end loss at x_j],
//   a_x(x) = -3 c3 x^2 + c1,
//   dL/dc3 = -h sum_{j,p} lambda_{j+1,p} x_{j,p}^3,  dL/dc1 = h sum lambda_{j+1} x_j,
//   dL/dkappa = h sum_j m_j S_j,  dL/dc0 = h sum_j S_j,
//   dL/dB0 = sqrt(h) sum lambda_{j+1} xi_j,  dL/dB = sqrt(h) sum lambda_{j+1} x_j xi_j,
//   dL/dBE = sqrt(h) sum_j m_j Z_j,
// and a cotangent (gm, gv) on (M_n, V_n) injects gm/P + gv (2/P)(x - M_n).
//
// The forward run (the fine kernel with recording on) leaves a particle
// checkpoint every c steps and the per-step uniforms it used (the mean m_j
// and the two mean-dependent terms of the step).  Per segment, in reverse:
// each thread recomputes its own particles over the c steps from the
// checkpoint (no reduction is needed: the means are recorded), storing
// states (and, with state- or mean-dependent diffusion, draws; with
// additive noise the backward step regenerates its draws from Philox, which
// costs less than reading them back), then sweeps backward with one group
// exchange per step,
// in the shift form that lets that exchange run one step behind the sweep
// (below).  The replay evaluates the step exactly as the forward kernel did,
// so it reproduces the forward states.
#include <cmath>

#include "adjoint.cuh"
#include "fine_kernel.cuh"

namespace mmp {


// MULT false: additive diffusion (B = BE = 0), the forward's shift form;
// the per-step exchange is the group sum of mu (one value).
// MULT true: general diffusion; the shift of lambda_j also needs Z_j, so
// the exchange carries three sums (below) as FP64 records.
// TPB threads per CTA, one CTA per SM: the whole GPU holds one slice's
// particles, a few quads per thread, and the warps of the one CTA hide
// the latency of the loads of the replayed states.
template <typename R, bool MULT, int TPB>
__global__ void __launch_bounds__(TPB, 1) k_adjoint(const AdjointArgs a) {
  constexpr int NW = TPB / 32;
  __shared__ GroupSharedT<NW> sh;
  __shared__ double mred[2][NW][3];      // general form: per-warp partials, by exchange parity
  __shared__ double mtot[2][3];          // general form: group sums, by exchange parity
  const int G = a.G;
  const int g = blockIdx.x;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int qb = (int)(((long long)a.Q * g) / G);
  const int qe = (int)(((long long)a.Q * (g + 1)) / G);
  const int span = qe - qb - tid;
  const int nq = span <= 0 ? 0 : min(a.nq, (span + TPB - 1) / TPB);
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

  QuadStore<R, 0, TPB> lam;  // mu of this thread's quads, in shared memory
  lam.bind();
  for (int i = 0; i < nq; ++i) {
    const R zero[4] = {0, 0, 0, 0};
    lam.put(i, zero);
  }

  // coefficients rounded once per CTA (keeps FP64 conversions out of the
  // loops), each exactly as the forward kernel rounds it
  if (sizeof(R) == 4 && tid == 0) {
    sh.cf[0] = (float)a.h;
    sh.cf[1] = (float)a.nc3;
    sh.cf[2] = (float)a.c1;
    sh.cf[3] = (float)(a.kappa * a.h / (double)a.P);
    sh.cf[4] = (float)a.sqrt_h;
    sh.cf[5] = (float)(a.h * a.nc3);
    sh.cf[6] = (float)(a.h * a.c1);
    sh.cf[7] = (float)(a.B * a.sqrt_h);
  }
  __syncthreads();
  const bool fl = sizeof(R) == 4;
  const R h = fl ? (R)sh.cf[0] : (R)a.h;
  const R nc3 = fl ? (R)sh.cf[1] : (R)a.nc3;
  const R c1 = fl ? (R)sh.cf[2] : (R)a.c1;
  const R kh_p = fl ? (R)sh.cf[3] : (R)(a.kappa * a.h / (double)a.P);
  const R sqh = fl ? (R)sh.cf[4] : (R)a.sqrt_h;
  const R hn3 = fl ? (R)sh.cf[5] : (R)(a.h * a.nc3);
  const R hc1 = fl ? (R)sh.cf[6] : (R)(a.h * a.c1);
  const R bsq = fl ? (R)sh.cf[7] : (R)(a.B * a.sqrt_h);  // B sqrt(h), the state-proportional amplitude
  const R* uni = (const R*)a.uni;
  R* segx = (R*)a.segx;
  R* segz = (R*)a.segz;

  Acc<R> acc3, acc1, accb, accB, accBE;  // -h x^3, h x, sqrt(h) xi, sqrt(h) x xi, sqrt(h) m xi terms
  double acc_k = 0.0, acc_c0 = 0.0;      // h m_j S_j, h S_j (thread 0 of CTA 0)
  R s_next = (R)0;                       // pending shift s_{j+1} of lambda_{j+1}
  int par = 0;                           // exchange parity: alternates with every exchange

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
  // the draws of global step j for quad q as the additive form's step uses
  // them, radius times cosine or sine (lanes past P zeroed)
  auto polar_draws = [&](long long j, int q, R z[4]) {
    R nr[2], c[2], sn[2];
    normals4_polar<R>(philox4x32_10(rng_counter((uint32_t)q, (uint32_t)(j % a.nf), (uint32_t)(j / a.nf), 0u,
                                                a.ptag), a.key0, a.key1), nr, c, sn);
    z[0] = mulR(nr[0], c[0]);
    z[1] = mulR(nr[0], sn[0]);
    z[2] = mulR(nr[1], c[1]);
    z[3] = mulR(nr[1], sn[1]);
    zero_tail(q, z);
  };
  // the draws of global step j for quad q (lanes past P zeroed)
  auto draws = [&](long long j, int q, R z[4]) {
    normals4<R>(philox4x32_10(rng_counter((uint32_t)q, (uint32_t)(j % a.nf), (uint32_t)(j / a.nf), 0u, a.ptag),
                              a.key0, a.key1), z);
    zero_tail(q, z);
  };
  // General form: the exchange of reverse step j carries, for the step
  // before it, sum mu_j, sum_p mu_{j,p} xi_{j-1,p} and sum_p xi_{j-1,p}; the
  // reader forms S_{j-1} = sum mu_j + P s_j and Z_{j-1} = sum mu_j xi_{j-1} + s_j sum xi_{j-1}.
  // Per warp: butterfly, lane 0 stores the warp's three partials.
  auto mult_warp = [&](double v0, double v1, double v2) {
    double v[3] = {v0, v1, v2};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 3; ++k) mred[par][warp][k] = v[k];
    }
  };
  // warp 0, after the barrier: the CTA's partials (warps in index order) as record epoch e
  auto mult_publish = [&](unsigned e) {
    double v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = lane < NW ? mred[par][lane][k] : 0.0;
#pragma unroll
    for (int off = NW / 2; off > 0; off >>= 1) {
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    }
    if (lane == 0) group_publish(grp, e, v, 3);
  };
  // warp 0, before the barrier: bounded wait for record epoch e of every CTA,
  // the sums (CTAs in a fixed order) into mtot[par]
  auto mult_fetch = [&](unsigned e) {
    const bool ok = group_wait(grp, e);
    double v[3] = {0.0, 0.0, 0.0};
    if (ok) {
      for (int c = lane; c < G; c += 32) {
        const double* s = group_slot(grp, c, e);
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] += __ldcg(s + k);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 3; ++k) mtot[par][k] = v[k];
      if (!ok) sh.abort = 1;
    }
  };

  // Two buffers of a segment's replayed states (and, for the general form,
  // its draws).  While the group reverses segment s (reading buffer s & 1),
  // warps 1.. replay segment s - 1 into the other, one step per reverse
  // step, in the time warp 0 waits for the peers' sums; only the last
  // segment is replayed on its own.  The replayed values are those of a
  // replay done before the reverse sweep (each quad's steps run in order
  // through the same arithmetic); a replayed quad is carried from step to
  // step through its row of the buffer.
  auto buf = [&](int sg) -> R* { return segx + (size_t)(sg & 1) * (size_t)(a.c + 1) * (size_t)a.pitch; };
  auto bufz = [&](int sg) -> R* { return segz + (size_t)(sg & 1) * (size_t)a.c * (size_t)a.pitch; };
  const int n_rep = TPB - 32;  // replay threads (warps 1..)
  const int rt = tid - 32;     // this thread's replay index (negative in warp 0)
  // x at global step j -> x at step j + 1, as the forward stepped it; the
  // general form also stores the step's draws at zdst
  auto replay_step = [&](int q, long long j, R x[4], R* zdst) {
    const uint4 o = philox4x32_10(
        rng_counter((uint32_t)q, (uint32_t)(j % a.nf), (uint32_t)(j / a.nf), 0u, a.ptag), a.key0, a.key1);
    if constexpr (MULT) {
      // x + h (nc3 x^3 + c1 x + kappa m_j + c0) + (B sqrt(h) x + (BE m_j + B0) sqrt(h)) xi,
      // rounded as the forward's general form rounds it
      R z[4];
      normals4<R>(o, z);
      zero_tail(q, z);
      Quad<R>::store(zdst + 4 * (size_t)q, z);
      const R base = uni[3 * j + 1];  // kappa m_j + c0 as the forward used it
      const R boff = uni[3 * j + 2];  // (BE m_j + B0) sqrt(h) as the forward used it
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const R xv = x[w];
        const R drift = fmaR(fmaR(nc3, mulR(xv, xv), c1), xv, base);
        const R amp = fmaR(bsq, xv, boff);
        x[w] = fmaR(amp, z[w], fmaR(h, drift, xv));
      }
    } else {
      // the draws are not stored: the reverse sweep regenerates them
      R nr[2], c[2], sn[2];
      normals4_polar<R>(o, nr, c, sn);
      const R d = uni[3 * j + 1];    // h (kappa m_j + c0) as the forward used it
      const R amp = uni[3 * j + 2];  // B0 sqrt(h) as the forward used it
      em_partial_pair(x[0], x[1], nr[0], c[0], sn[0], hn3, hc1, amp);
      em_partial_pair(x[2], x[3], nr[1], c[1], sn[1], hn3, hc1, amp);
#pragma unroll
      for (int w = 0; w < 4; ++w) x[w] = addR(x[w], d);
    }
    zero_tail(q, x);
  };
  // warps 1..: step r of segment sr for this thread's replay quads (rows r,
  // from the checkpoint at r = 0, and r + 1 of its state buffer; draw row r)
  auto replay_rows = [&](int sr, int r) {
    if (rt < 0) return;
    R* bx = buf(sr);
    R* bz = bufz(sr) + (size_t)r * a.pitch;
    const R* ckr = (const R*)a.ckpt + (size_t)sr * a.pitch;
    const long long jr = (long long)sr * a.c + r;
    for (int q = qb + rt; q < qe; q += n_rep) {
      R x[4];
      if (r == 0) {
        Quad<R>::load(ckr + 4 * (size_t)q, x);
        Quad<R>::store(bx + 4 * (size_t)q, x);
      } else {
        Quad<R>::load(bx + (size_t)r * a.pitch + 4 * (size_t)q, x);
      }
      replay_step(q, jr, x, bz);
      Quad<R>::store(bx + (size_t)(r + 1) * a.pitch + 4 * (size_t)q, x);
    }
  };

  for (int seg = a.n_seg - 1; seg >= 0; --seg) {
    const long long j0 = (long long)seg * a.c;
    const long long j1 = min(a.J, j0 + a.c);
    const int L = (int)(j1 - j0);
    R* const bxs = buf(seg);   // this segment's replayed states
    R* const bzs = bufz(seg);  // and draws (general form)
    // ---- the last segment: replayed on its own (warps 1..) ---------------
    if (seg == a.n_seg - 1) {
      const R* ck = (const R*)a.ckpt + (size_t)seg * a.pitch;
      if (rt >= 0) {
        for (int q = qb + rt; q < qe; q += n_rep) {
          R x[4];
          Quad<R>::load(ck + 4 * (size_t)q, x);
          for (int jj = 0; jj < L; ++jj) {
            Quad<R>::store(bxs + (size_t)jj * a.pitch + 4 * (size_t)q, x);
            replay_step(q, j0 + jj, x, bzs + (size_t)jj * a.pitch);
          }
          Quad<R>::store(bxs + (size_t)L * a.pitch + 4 * (size_t)q, x);
        }
      }
      __syncthreads();  // the rows are read by other threads than their writers
    }
    // ---- backward through the segment ----------------------------------
    // Shift form of the reverse recursion: lambda_j = mu_j + s_j with
    //   mu_j = lambda_{j+1} (1 + h a_x(x_j) + sqrt(h) B xi_j) [+ slice-end injection at x_j],
    //   s_j  = (h kappa S_j + sqrt(h) BE Z_j) / P,  S_j = sum mu_{j+1} + P s_{j+1},
    //   Z_j  = sum mu_{j+1} xi_j + s_{j+1} sum xi_j,
    // so the group sums of mu_j published at the end of reverse step j are
    // first needed at the end of step j - 1 (the exchange is one step
    // behind, as in the forward).  `lam` holds mu, `s_next` the pending shift.
    if (j1 == a.J) {
      // lambda_J: the last slice end's injection alone (s_J = 0); its sums are epoch 0
      R part = (R)0, pz = (R)0, zs = (R)0;
      for (int i = 0; i < nq; ++i) {
        const int q = qb + tid + i * TPB;
        R x[4], l[4] = {0, 0, 0, 0};
        Quad<R>::load(bxs + (size_t)L * a.pitch + 4 * (size_t)q, x);
        inject(a.J, q, x, l);
        lam.put(i, l);
        part = addR(part, addR(addR(l[0], l[1]), addR(l[2], l[3])));
        if constexpr (MULT) {
          R zp[4];
          Quad<R>::load(bzs + (size_t)(L - 1) * a.pitch + 4 * (size_t)q, zp);
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            pz = fmaR(l[w], zp[w], pz);
            zs = addR(zs, zp[w]);
          }
        }
      }
      if constexpr (MULT) {
        mult_warp((double)part, (double)pz, (double)zs);
        __syncthreads();
        if (warp == 0) mult_publish(0u);
      } else {
        step_sum_warp<R>(sh, par, part);
        __syncthreads();
        if (warp == 0) {
          const typename StepSum<R>::T cta = step_sum_cta<R>(sh, par);
          if (lane == 0) StepSum<R>::publish(grp, 0u, cta);
        }
      }
      grp.epoch = 1u;
      par ^= 1;
    }
    for (int jj = L - 1; jj >= 0; --jj) {
      const long long j = j0 + jj;
      const unsigned ej = (unsigned)(a.J - j);  // epoch of the sums of mu_j
      const bool end_j = j > 0 && j % a.nf == 0;
      const R mj = uni[3 * j];                  // m_j as the forward used it
      R part = (R)0, p3 = (R)0, p1 = (R)0, pb = (R)0, pB = (R)0, pz = (R)0, zs = (R)0;
      for (int i = 0; i < nq; ++i) {
        const int q = qb + tid + i * TPB;
        R l[4], x[4], z[4];
        if constexpr (MULT) {
          Quad<R>::load(bzs + (size_t)jj * a.pitch + 4 * (size_t)q, z);
        } else {
          polar_draws(j, q, z);  // regenerated: half the bytes of a stored row
        }
        lam.get(i, l);
        Quad<R>::load(bxs + (size_t)jj * a.pitch + 4 * (size_t)q, x);
#pragma unroll
        for (int w = 0; w < 4; ++w) l[w] = addR(l[w], s_next);  // lambda_{j+1}
        zero_tail(q, l);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          // step j's parameter partials, then mu_j
          p3 -= l[w] * x[w] * x[w] * x[w];
          p1 += l[w] * x[w];
          const R lz = l[w] * z[w];
          pb += lz;
          pB += lz * x[w];
          const R ax = fmaR((R)3 * nc3, x[w] * x[w], c1);  // -3 c3 x^2 + c1
          if constexpr (MULT) {
            l[w] = mulR(l[w], fmaR(bsq, z[w], fmaR(h, ax, (R)1)));
          } else {
            l[w] = mulR(l[w], fmaR(h, ax, (R)1));
          }
        }
        if (end_j) inject(j, q, x, l);
        zero_tail(q, l);
        lam.put(i, l);
        part = addR(part, addR(addR(l[0], l[1]), addR(l[2], l[3])));
        if constexpr (MULT) {
          if (j > 0) {
            // the draws of step j - 1 (the previous segment's last row is
            // regenerated: that segment is replayed only later)
            R zp[4];
            if (jj > 0) {
              Quad<R>::load(bzs + (size_t)(jj - 1) * a.pitch + 4 * (size_t)q, zp);
            } else {
              draws(j - 1, q, zp);
            }
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              pz = fmaR(l[w], zp[w], pz);
              zs = addR(zs, zp[w]);
            }
          }
        }
      }
      acc3.add(h * p3);
      acc1.add(h * p1);
      accb.add(sqh * pb);
      accB.add(sqh * pB);
      accBE.add(sqh * mj * pb);
      if constexpr (MULT) {
        // warp 0 reads the sums of mu_{j+1} (epoch ej - 1, published a step
        // ago) before the barrier and publishes those of mu_j after it
        mult_warp((double)part, (double)pz, (double)zs);
        if (warp == 0) {
          mult_fetch(ej - 1u);
        } else if (seg > 0) {
          replay_rows(seg - 1, L - 1 - jj);
        }
        __syncthreads();
        if (sh.abort) return;
        const double sn = (double)s_next;
        const double S_d = mtot[par][0] + (double)a.P * sn;
        const double Z_d = mtot[par][1] + sn * mtot[par][2];
        if (g == 0 && tid == 0) {
          acc_k += a.h * (double)mj * S_d;
          acc_c0 += a.h * S_d;
        }
        s_next = (R)((a.kappa * a.h * S_d + a.sqrt_h * a.BE * Z_d) / (double)a.P);  // s_j
        if (warp == 0) mult_publish(ej);
      } else {
        // warp 0 reads sum mu_{j+1} (epoch ej - 1, published a step ago)
        // before the barrier and publishes sum mu_j (epoch ej) after it;
        // meanwhile warps 1.. replay a step of the previous segment
        step_sum_warp<R>(sh, par, part);
        if (warp == 0) {
          typename StepSum<R>::T sum;
          const bool ok = StepSum<R>::fetch(grp, ej - 1u, sum);
          if (lane == 0) {
            StepSum<R>::gsum(sh, par) = sum;
            if (!ok) sh.abort = 1;
          }
        } else if (seg > 0) {
          replay_rows(seg - 1, L - 1 - jj);
        }
        __syncthreads();
        if (sh.abort) return;
        const typename StepSum<R>::T sm = StepSum<R>::gsum(sh, par);
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
          acc_k += a.h * (double)mj * S_d;
          acc_c0 += a.h * S_d;
        }
        s_next = mulR(kh_p, S);  // s_j, pending on lambda_j
        if (warp == 0) {
          const typename StepSum<R>::T cta = step_sum_cta<R>(sh, par);
          if (lane == 0) StepSum<R>::publish(grp, ej, cta);
        }
      }
      grp.epoch = ej + 1u;
      par ^= 1;
    }
    // a segment shorter than c (the last) leaves steps of the previous
    // segment's replay, which are done here; the barrier of the last reverse
    // step (or this one) makes the rows visible to their readers
    if (seg > 0 && L < a.c) {
      for (int r = L; r < a.c; ++r) replay_rows(seg - 1, r);
      __syncthreads();
    }
  }
  // ---- reduce the parameter partials over the group (FP64) -------------
  {
    double v[kNGrad] = {acc3.get(), acc1.get(), acc_k, acc_c0, accb.get(), accB.get(), accBE.get()};
    warp_reduce_to_shared<kNGrad>(sh, v, 0u, 0u);
    __syncthreads();
    if (sh.abort) return;
    const unsigned e = grp.epoch++;
    if (warp == 0 && !group_finish<kNGrad>(sh, grp, e, 0u, 0u) && lane == 0) sh.abort = 1;
    __syncthreads();
    if (sh.abort) return;
    if (g == 0 && tid == 0) {
      bool finite = true;
      for (int k = 0; k < kNGrad; ++k) {
        a.grad[k] = sh.tot[k];
        finite = finite && fabs(sh.tot[k]) < INFINITY;
      }
      if (!finite) atomicOr(a.status, kStatusNumeric);
    }
  }
}

const void* adjoint_kernel(int precision, bool mult) {
  if (precision == MMP_MIXED)
    return mult ? (const void*)k_adjoint<float, true, kAdjTPB> : (const void*)k_adjoint<float, false, kAdjTPB>;
  return mult ? (const void*)k_adjoint<double, true, kAdjTPB> : (const void*)k_adjoint<double, false, kAdjTPB>;
}

size_t adjoint_smem_bytes(int precision, int nq) {
  return (size_t)nq * kAdjTPB * 4 * (precision == MMP_MIXED ? sizeof(float) : sizeof(double));
}

cudaError_t launch_adjoint(int precision, bool mult, const AdjointArgs& args, cudaStream_t stream) {
  AdjointArgs copy = args;
  void* params[] = {&copy};
  return cudaLaunchCooperativeKernel(adjoint_kernel(precision, mult), dim3(args.G), dim3(kAdjTPB), params,
                                     adjoint_smem_bytes(precision, args.nq), stream);
}

}  // namespace mmp
