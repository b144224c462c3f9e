// n-dimensional complex FFT kernels and the FFT-backend stiffness apply (declarations).
#pragma once

#include <string>

#include "qp_internal.cuh"

namespace qp {

struct FftPlan;

// pd: host copy of the plan description; pdp: its device copy (must be uploaded before the set-up calls).
FftPlan* fft_plan_create(const PlanDev& pd, int precisions, int max_rhs, cudaStream_t s);
void fft_plan_destroy(FftPlan* f);
int64_t fft_plan_bytes(const FftPlan* f);
bool fft_supported(int N);
// Coefficient from device grid samples (ncomp x D doubles, C order) or from the plan's tap list.
void fft_set_grid(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, const double* grid, cudaStream_t s);
void fft_set_taps(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, cudaStream_t s);
// Jacobi diagonal (the Frobenius one is not built on this backend: frob = 0) and the set-up checks into
// out[0..2]: min |lambda|^2, min q/|lambda|^2 over k != 0, smallest Cholesky pivot of A over the nodes.
void fft_diag(FftPlan* f, const PlanDev* pd, const PlanDev* pdp, double* jac, double* frob, float* jac32,
              float* frob32, double* out, cudaStream_t s);
// The Frobenius-optimal diagonal (Sec. 4.3) into frob / frob32 by FFT cross-correlations; synchronises s.
void fft_frobenius(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, double* frob, float* frob32, cudaStream_t s);
// w = Q h for nrhs vectors of the plan.
template <typename T>
void fft_apply(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, const cplx<T>* h, cplx<T>* w, int nrhs,
               cudaStream_t s);
// Autotuner of the apply (per precision in the plan's workspace): times every candidate group schedule and the
// per-axis path on this GPU and keeps the fastest; the choice is cached per geometry for the process. Off
// (fft_set_autotune(false)): the balanced-split heuristic.
void fft_autotune(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, cudaStream_t s);
void fft_set_autotune(bool on);
// The process's tuning cache to and from a text file (entries written / loaded; -1: I/O or format error; load: -2
// when the file was written on another kind of GPU), and its clearing.
int fft_tune_cache_save(const char* path);
int fft_tune_cache_load(const char* path);
void fft_tune_cache_clear();
bool fft_autotune_on();
int fft_schedule_count(const FftPlan* f, bool fp64);
// the schedule in use: its candidate index (-1: the heuristic's, untimed), description and timed ms per apply
int fft_schedule_get(const FftPlan* f, bool fp64, std::string& text, float& ms);
void fft_schedule_set(FftPlan* f, bool fp64, int index);
void fft_rhs(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, int j0, int nrhs, double2* F, cudaStream_t s);
void fft_astar(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, const double2* U, double* out, cudaStream_t s);
void fft_standalone(int n, const int* N, int count, void* data, int sign, int precision, cudaStream_t s);

}  // namespace qp
