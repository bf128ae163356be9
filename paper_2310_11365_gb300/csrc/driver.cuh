// driver.cuh -- arguments of the device-side Parareal driver kernel.
#pragma once

#include <cuda_runtime.h>

namespace mmp {

struct DriverArgs {
  double nc3, c1, kappa, c0, B, BE, B0;  // model (nc3 = -c3)
  int family;                            // MMP_FAMILY_POLY / MMP_FAMILY_ROTATOR
  double K, g;                           // plane rotator: coupling, pinning
  int N, I, variant, precision;
  int coarse_model;                      // MMP_COARSE_*
  double dT, hc;                         // slice length, coarse substep
  int nc;                                // coarse substeps per slice
  double thr, thr2, thr3;  // region boundaries t_1 < t_2 < t_3 (the first I - 1)
  long long P;
  double tol;
  int max_sweeps;
  const double* stats;     // [N][kStat] restriction of F_n(u^{k-1}_n), row n
  const double* stats_u0;  // [kStat] restriction of u0
  double* rho;             // [N+1][kMom] macro state (MMP_MOMENT_STRIDE layout)
  double* cache;           // [N][2 kMaxRegions] C_n(rho^{k-1}_n): (mean_i, var_i) per region
  double* aff;             // [N+1][kMaxRegions][kAff] matching records for the inputs u^k_n
  double* ctl;             // control block (see k_driver)
  unsigned* status;
  int sweep;               // 0 = lifting, k >= 1 = after fine sweep k
};

cudaError_t launch_driver(const DriverArgs& args, cudaStream_t stream);
// One warp per problem over a device array of arguments; sweep[b] < 0 skips
// problem b.  summary[5 b ..] receives (change, converged, sweeps, done,
// status word).
cudaError_t launch_driver_batch(const DriverArgs* args, const int* sweep, double* summary, int n,
                                cudaStream_t stream);

}  // namespace mmp
