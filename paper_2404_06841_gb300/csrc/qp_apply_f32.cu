// Instantiations of the taps-backend apply kernels (qp_apply.cuh): FP32 batch apply (PCG level of the refinement inner solves).
#include "qp_apply.cuh"

namespace qp {

template void apply_launch_real<float, EPI_DOT_HW>(bool, int, const BatchDev&, int, int, unsigned long long, int, size_t,
                                              const StarParams*, int, cudaStream_t);

}  // namespace qp
