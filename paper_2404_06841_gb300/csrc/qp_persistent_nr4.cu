// Instantiations of the persistent PCG solve for 4 right-hand sides (one translation unit per count keeps
// the build parallel).
#include "qp_persistent.cuh"

namespace qp {

const void* persistent_kernel_nr4(bool realc) {
  return realc ? reinterpret_cast<const void*>(&k_pcg_persistent<true, 4, 0>)
               : reinterpret_cast<const void*>(&k_pcg_persistent<false, 4, 0>);
}

}  // namespace qp
