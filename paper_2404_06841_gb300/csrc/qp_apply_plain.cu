// Instantiations of the taps-backend apply kernels (qp_apply.cuh): plain apply w = Q h, both precisions.
#include "qp_apply.cuh"

namespace qp {

template void launch_apply_plain<double>(const PlanDev*, bool, int, int, int, const double2*, double2*, int,
                                         const StarParams*, int, cudaStream_t);
template void launch_apply_plain<float>(const PlanDev*, bool, int, int, int, const float2*, float2*, int,
                                        const StarParams*, int, cudaStream_t);

}  // namespace qp
