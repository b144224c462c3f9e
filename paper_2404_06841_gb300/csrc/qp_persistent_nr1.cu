// Instantiations of the persistent PCG solve for 1 right-hand side (one translation unit per count keeps
// the build parallel).
#include "qp_persistent.cuh"

namespace qp {

const void* persistent_kernel_nr1(bool realc) {
  return realc ? reinterpret_cast<const void*>(&k_pcg_persistent<true, 1, 0>)
               : reinterpret_cast<const void*>(&k_pcg_persistent<false, 1, 0>);
}

}  // namespace qp
