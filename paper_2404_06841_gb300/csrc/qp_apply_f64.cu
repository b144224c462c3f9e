// Instantiations of the taps-backend apply kernels (qp_apply.cuh): FP64 batch apply with the (h, Q h) epilogue, and without an epilogue.
#include "qp_apply.cuh"

namespace qp {

template void apply_launch_real<double, EPI_DOT_HW>(bool, int, const BatchDev&, int, int, unsigned long long, int, size_t,
                                              const StarParams*, int, cudaStream_t);
template void apply_launch_real<double, EPI_NONE>(bool, int, const BatchDev&, int, int, unsigned long long, int, size_t,
                                              const StarParams*, int, cudaStream_t);

}  // namespace qp
