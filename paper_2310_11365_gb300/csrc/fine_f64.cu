// fine_f64.cu -- double-particle (MMP_FP64) instantiations of the fused
// fine-propagator kernel, NQ = 1..4 quads per thread.
#include "fine_kernel.cuh"

namespace mmp {

#define MMP_F64_CASE(NQ)                                          \
  case NQ:                                                        \
    return mult ? (const void*)k_fine<double, NQ, true>           \
                : (const void*)k_fine<double, NQ, false>;

const void* fine_kernel_f64(int nq, bool mult, int family) {
  if (family == kFamRotator) return nq == 0 ? (const void*)k_fine<double, 0, false, kFamRotator> : nullptr;
  if (nq == 0)
    return mult ? (const void*)k_fine<double, 0, true> : (const void*)k_fine<double, 0, false>;
  switch (nq) {
    MMP_F64_CASE(1)
    MMP_F64_CASE(2)
    MMP_F64_CASE(3)
    MMP_F64_CASE(4)
    default:
      return nullptr;
  }
}

}  // namespace mmp
