// Instantiations of the persistent PCG solve of a star-1 plan with n = 6 axes, every one carrying the taps
// m = +-e_j, d = 3 and 3 right-hand sides: the FP32 level of a refinement solve takes the stencil with the
// geometry compiled in (straight-line axis loop, the same arithmetic as the general star-1 instantiations); the
// FP64 level keeps the general stencil (compiled in there too, the real-coefficient kernels spilled 12 bytes, and
// the kernel reached 255 registers). sk = 1 scalar, 2 diagonal coefficient.
#include "qp_persistent.cuh"

namespace qp {

constexpr bool FIX64 = false;

const void* persistent_star_fixed_kernel_n6(bool realc, int sk) {
  if (sk == 2)
    return realc ? reinterpret_cast<const void*>(&k_pcg_persistent<true, 3, 2, 6, 3, FIX64>)
                 : reinterpret_cast<const void*>(&k_pcg_persistent<false, 3, 2, 6, 3, FIX64>);
  return realc ? reinterpret_cast<const void*>(&k_pcg_persistent<true, 3, 1, 6, 3, FIX64>)
               : reinterpret_cast<const void*>(&k_pcg_persistent<false, 3, 1, 6, 3, FIX64>);
}

}  // namespace qp
