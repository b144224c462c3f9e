// Instantiations of the persistent PCG solve for 3 right-hand sides (one translation unit per count keeps
// the build parallel).
#include "qp_persistent.cuh"

namespace qp {

const void* persistent_kernel_nr3(bool realc) {
  return realc ? reinterpret_cast<const void*>(&k_pcg_persistent<true, 3, 0>)
               : reinterpret_cast<const void*>(&k_pcg_persistent<false, 3, 0>);
}

}  // namespace qp
