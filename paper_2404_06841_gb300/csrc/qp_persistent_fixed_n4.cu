// Instantiations of the persistent PCG solve of a star-1 plan with n = 4 axes, every one carrying the taps
// m = +-e_j, d = 2 and 2 right-hand sides: the FP32 level of a refinement solve takes the stencil with the
// geometry compiled in (straight-line axis loop, the same arithmetic as the general star-1 instantiations); the
// FP64 level keeps the general stencil (compiled in there too, the real-coefficient kernels spilled 12 bytes, and
// cfg1's FP64 solve ran no faster: its time is grid-barrier and FP64 latency). sk = 1 scalar, 2 diagonal coefficient.
#include "qp_persistent.cuh"

namespace qp {

constexpr bool FIX64 = false;

const void* persistent_star_fixed_kernel_n4(bool realc, int sk) {
  if (sk == 2)
    return realc ? reinterpret_cast<const void*>(&k_pcg_persistent<true, 2, 2, 4, 2, FIX64>)
                 : reinterpret_cast<const void*>(&k_pcg_persistent<false, 2, 2, 4, 2, FIX64>);
  return realc ? reinterpret_cast<const void*>(&k_pcg_persistent<true, 2, 1, 4, 2, FIX64>)
               : reinterpret_cast<const void*>(&k_pcg_persistent<false, 2, 1, 4, 2, FIX64>);
}

}  // namespace qp
