// Instantiations of the taps-backend apply kernels (qp_apply.cuh): plain apply w = Q h, both precisions, and the
// builder of a star-1 plan's stored FP64 weights.
#include "qp_apply.cuh"

namespace qp {

template void launch_apply_plain<double>(const PlanDev*, bool, int, int, int, const double2*, double2*, int,
                                         const StarParams*, int, cudaStream_t);
template void launch_apply_plain<float>(const PlanDev*, bool, int, int, int, const float2*, float2*, int,
                                        const StarParams*, int, cudaStream_t);

void launch_star_weights(const StarParams& st, bool realc, int kind, int D, void* out, cudaStream_t s) {
  const int nblk = (D / 2 + BLOCK - 1) / BLOCK;
  const bool dg = kind == QP_COEF_DIAG;
  if (realc) {
    if (dg) k_star_weights<true, true><<<nblk, BLOCK, 0, s>>>(st, D, out);
    else k_star_weights<true, false><<<nblk, BLOCK, 0, s>>>(st, D, out);
  } else {
    if (dg) k_star_weights<false, true><<<nblk, BLOCK, 0, s>>>(st, D, out);
    else k_star_weights<false, false><<<nblk, BLOCK, 0, s>>>(st, D, out);
  }
  count_launch();
}

}  // namespace qp
