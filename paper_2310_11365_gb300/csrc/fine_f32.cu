// fine_f32.cu -- float-particle (MMP_MIXED) instantiations of the fused
// fine-propagator kernel, NQ = 1..8 quads per thread.
#include "fine_kernel.cuh"

namespace mmp {

#define MMP_F32_CASE(NQ)                                          \
  case NQ:                                                        \
    return mult ? (const void*)k_fine<float, NQ, true>            \
                : (const void*)k_fine<float, NQ, false>;

const void* fine_kernel_f32(int nq, bool mult, int family) {
  if (family == kFamRotator) return nq == 0 ? (const void*)k_fine<float, 0, false, kFamRotator> : nullptr;
  if (nq == 0)
    return mult ? (const void*)k_fine<float, 0, true> : (const void*)k_fine<float, 0, false>;
  switch (nq) {
    MMP_F32_CASE(1)
    MMP_F32_CASE(2)
    MMP_F32_CASE(3)
    MMP_F32_CASE(4)
    MMP_F32_CASE(5)
    MMP_F32_CASE(6)
    MMP_F32_CASE(7)
    MMP_F32_CASE(8)
    default:
      return nullptr;
  }
}

}  // namespace mmp
