// Placeholder until the FFT backend lands: every entry raises QP_ERR_UNSUPPORTED.
#include "qp_fft.cuh"

namespace qp {
struct FftPlan {};
static void nb() { raise(QP_ERR_UNSUPPORTED, "FFT backend not built"); }
FftPlan* fft_plan_create(const PlanDev&, int, cudaStream_t) { nb(); return nullptr; }
void fft_plan_destroy(FftPlan* f) { delete f; }
int64_t fft_plan_bytes(const FftPlan*) { return 0; }
void fft_set_grid(FftPlan*, const PlanDev&, const double*, cudaStream_t) { nb(); }
void fft_set_taps(FftPlan*, const PlanDev&, cudaStream_t) { nb(); }
void fft_diag(FftPlan*, const PlanDev&, double*, double*, float*, float*, double*, cudaStream_t) { nb(); }
template <typename T>
void fft_apply(FftPlan*, const PlanDev&, const cplx<T>*, cplx<T>*, int, cudaStream_t) { nb(); }
template void fft_apply<double>(FftPlan*, const PlanDev&, const double2*, double2*, int, cudaStream_t);
template void fft_apply<float>(FftPlan*, const PlanDev&, const float2*, float2*, int, cudaStream_t);
void fft_rhs(FftPlan*, const PlanDev&, int, int, double2*, cudaStream_t) { nb(); }
void fft_astar(FftPlan*, const PlanDev&, const double2*, double*, cudaStream_t) { nb(); }
void fft_standalone(int, const int*, int, void*, int, int, cudaStream_t) { nb(); }
}  // namespace qp
