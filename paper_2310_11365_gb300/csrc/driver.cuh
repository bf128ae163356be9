// driver.cuh -- arguments of the device-side Parareal driver kernel.
#pragma once

#include <cuda_runtime.h>

namespace mmp {

struct DriverArgs {
  double nc3, c1, kappa, c0, B, BE, B0;  // model (nc3 = -c3)
  int N, I, variant, precision;
  int coarse_model;                      // MMP_COARSE_*
  double dT, hc;                         // slice length, coarse substep
  int nc;                                // coarse substeps per slice
  double thr;
  long long P;
  double tol;
  int max_sweeps;
  const double* stats;     // [N][16] restriction of F_n(u^{k-1}_n), row n
  const double* stats_u0;  // [16] restriction of u0
  double* rho;             // [N+1][8] macro state: frac0, mean0, var0, frac1, mean1, var1, M, V
  double* cache;           // [N][4] C_n(rho^{k-1}_n): mean0, var0, mean1, var1
  double* aff;             // [N+1][2][4] matching records for the inputs u^k_n
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
