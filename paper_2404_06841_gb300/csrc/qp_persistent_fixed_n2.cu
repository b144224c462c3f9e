// Instantiations of the persistent PCG solve of a star-1 plan with n = 2 axes, every one carrying the taps
// m = +-e_j, d = 1 and 1 right-hand side: both levels (FP64, and the FP32 level of a refinement solve) take the
// stencil with the geometry compiled in (straight-line axis loop, the same arithmetic as the general star-1
// instantiations; no spills; cfg0's FP64 solve 0.50 -> 0.48 ms). sk = 1 scalar, 2 diagonal coefficient.
#include "qp_persistent.cuh"

namespace qp {

constexpr bool FIX64 = true;

const void* persistent_star_fixed_kernel_n2(bool realc, int sk) {
  if (sk == 2)
    return realc ? reinterpret_cast<const void*>(&k_pcg_persistent<true, 1, 2, 2, 1, FIX64>)
                 : reinterpret_cast<const void*>(&k_pcg_persistent<false, 1, 2, 2, 1, FIX64>);
  return realc ? reinterpret_cast<const void*>(&k_pcg_persistent<true, 1, 1, 2, 1, FIX64>)
               : reinterpret_cast<const void*>(&k_pcg_persistent<false, 1, 1, 2, 1, FIX64>);
}

}  // namespace qp
