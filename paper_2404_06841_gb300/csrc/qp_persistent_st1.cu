// Instantiations of the persistent PCG solve of a star-1 plan (stencil data as a kernel parameter) for 1
// right-hand side: sk = 1 scalar, 2 diagonal coefficient.
#include "qp_persistent.cuh"

namespace qp {

const void* persistent_star_kernel_nr1(bool realc, int sk) {
  if (sk == 2)
    return realc ? reinterpret_cast<const void*>(&k_pcg_persistent<true, 1, 2>)
                 : reinterpret_cast<const void*>(&k_pcg_persistent<false, 1, 2>);
  return realc ? reinterpret_cast<const void*>(&k_pcg_persistent<true, 1, 1>)
               : reinterpret_cast<const void*>(&k_pcg_persistent<false, 1, 1>);
}

}  // namespace qp
