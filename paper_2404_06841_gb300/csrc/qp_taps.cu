// Taps backend: the compressed mat-vec of Sec. 4.2 as a direct stencil over the coefficient's Fourier modes,
//   (Q h)(k) = sum_t lambda(k)^T C_t lambda(k -N m_t) h(k -N m_t),   lambda(k) = P k,
// (eq. n-discrete_equation; App. D for a matrix coefficient), the diagonal preconditioners (Sec. 4.3), the
// corrector right-hand side (Sec. 5.2) and the a* reduction (eq. homcoefficient) on this representation.
//
// Work is split in chunks of consecutive modes of one unit (a plan and its right-hand sides); each chunk's
// partial sums go to a fixed slot and the block that completes a unit sums them in a fixed order
// (deterministic, no floating-point atomics). Modes are decoded with multiply-shift division; star taps (one
// nonzero axis) are grouped per axis so that each costs one wrap test, one index update and, for a scalar
// coefficient, one fused multiply-add for the weight: lambda(k).lambda(k') = |lambda(k)|^2 + dk (lambda(k).P_j).
#include "qp_stencil.cuh"

namespace qp {

// ------------------------------------------------------------------------------------------------ apply launches

// The apply kernels (qp_apply.cuh) are instantiated per vector precision and epilogue in qp_apply_*.cu.
template <typename T, int EPI>
void apply_launch_real(bool realc, int maxr, const BatchDev& b, int level, int refine, unsigned long long cond,
                       int nblk, size_t smem, const StarParams* st1, int kind, cudaStream_t s);

// realc: every taps plan of the batch has real tap values; mc: the largest ntaps * ncomp of its plans (sizes
// the shared coefficient table); maxr: the largest nrhs of its units; refine: REFINE_* (the refinement
// bookkeeping of the residual epilogue; REFINE_ZERO_U: the solutions are zero, so Q U = 0 is not computed).
// Each unit's stencil runs (UnitDev.run) are its own. st1 (a single star-1 unit with an even last axis, else
// null): its StarParams, passed to the kernel by value; kind: that unit's coefficient kind.
void launch_apply(const BatchDev& b, bool realc, int mc, int maxr, int level, int epi, int refine,
                  unsigned long long cond, int nblk, const StarParams* st1, int kind, cudaStream_t s) {
  if (level == LEVEL_FP32) {
    const size_t smem = (size_t)mc * sizeof(float2);
    apply_launch_real<float, EPI_DOT_HW>(realc, maxr, b, level, refine, cond, nblk, smem, st1, kind, s);
  } else {
    const size_t smem = (size_t)mc * sizeof(double2);
    if (epi == EPI_DOT_HW)
      apply_launch_real<double, EPI_DOT_HW>(realc, maxr, b, level, refine, cond, nblk, smem, st1, kind, s);
    else if (epi == EPI_RESIDUAL)
      apply_launch_real<double, EPI_RESIDUAL>(realc, maxr, b, level, refine, cond, nblk, smem, st1, kind, s);
    else apply_launch_real<double, EPI_NONE>(realc, maxr, b, level, refine, cond, nblk, smem, st1, kind, s);
  }
  count_launch();
}

// ------------------------------------------------------------------------------------------------ set-up kernels

// The stored FP64 entries of a plan with general taps: every tap's weight at every mode ([tap][D], real or complex),
// formed by the general stencil's own arithmetic (apply_run with WM = 2), one run of modes per thread.
template <bool REALC, int RUN>
__global__ void __launch_bounds__(BLOCK) k_gen_weights(const PlanDev* plan, int D, void* out) {
  __shared__ __align__(16) PlanDev sp;
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* scoef = reinterpret_cast<double2*>(smraw);
  load_plan<double>(plan, sp, scoef);
  const int e0 = (blockIdx.x * BLOCK + threadIdx.x) * RUN;
  if (e0 >= D) return;
  double2 acc[RUN][1];
  apply_run<double, REALC, 1, RUN, true, false, 2>(sp, scoef, e0, nullptr, D, 0, acc, out);
}

void launch_gen_weights(const PlanDev* plan_dev, bool realc, int mc, int D, int run, void* out, cudaStream_t s) {
  const size_t smem = (size_t)mc * sizeof(double2);
  const int nblk = (D / run + BLOCK - 1) / BLOCK;
  if (run == 2) {
    if (realc) k_gen_weights<true, 2><<<nblk, BLOCK, smem, s>>>(plan_dev, D, out);
    else k_gen_weights<false, 2><<<nblk, BLOCK, smem, s>>>(plan_dev, D, out);
  } else {
    if (realc) k_gen_weights<true, 1><<<nblk, BLOCK, smem, s>>>(plan_dev, D, out);
    else k_gen_weights<false, 1><<<nblk, BLOCK, smem, s>>>(plan_dev, D, out);
  }
  count_launch();
}

// lambda(k + m) for the tap with mode m (any number of nonzero axes), from the digits of k.
__device__ __forceinline__ void lambda_shift(const PlanDev& p, const int (&ib)[MAXN], const int (&k)[MAXN],
                                             const signed char* m, int sign, const double (&lk)[MAXD],
                                             double (&out)[MAXD]) {
#pragma unroll
  for (int a = 0; a < MAXD; ++a) out[a] = lk[a];
#pragma unroll
  for (int j = 0; j < MAXN; ++j) {
    const int mj = (j < p.n) ? sign * (int)m[j] : 0;
    if (mj != 0) {
      const int Nj = p.N[j];
      int ib2 = ib[j] + mj;
      ib2 += (ib2 < 0) ? Nj : 0;
      ib2 -= (ib2 >= Nj) ? Nj : 0;
      const int k2 = (2 * ib2 < Nj) ? ib2 : ib2 - Nj;
#pragma unroll
      for (int a = 0; a < MAXD; ++a)
        if (a < p.d) out[a] = fma((double)(k2 - k[j]), p.P[a][j], out[a]);
    }
  }
}

// Jacobi diagonal q(k) = lambda(k)^T A~_0 lambda(k) and the Frobenius-optimal diagonal q(k) / ||Q e_k||^2
// (eq. preconditioner) with ||Q e_k||^2 = sum_t |lambda(k +N m_t)^T C_t lambda(k)|^2 (O(gD), Sec. 4.3).
// Stored as M (z = M r), M(0) = 0. out[0] = min over k != 0 of |lambda(k)|^2, out[1] = min over those k of q(k).
// with_frob = 0: the Jacobi diagonal only (the Frobenius one costs a weight per tap and mode: built on first use).
__global__ void __launch_bounds__(BLOCK) k_diag(const PlanDev* plan, int D, double* jac, double* frob, float* jac32,
                                                float* frob32, double* partials, unsigned* counter, double* out,
                                                int with_frob) {
  __shared__ __align__(16) PlanDev sp;
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* scoef = reinterpret_cast<double2*>(smraw);
  load_plan<double>(plan, sp, scoef);
  const int d = sp.d;
  double red[2] = {DBL_MAX, DBL_MAX};
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    int ib[MAXN], k[MAXN];
    mode_digits(sp, e, ib, k);
    double lk[MAXD] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < MAXD; ++a)
#pragma unroll
      for (int j = 0; j < MAXN; ++j)
        if (a < d && j < sp.n) lk[a] = fma(sp.P[a][j], (double)k[j], lk[a]);
    double l2sum = 0.0;
#pragma unroll
    for (int a = 0; a < MAXD; ++a)
      if (a < d) l2sum += lk[a] * lk[a];
    const double q = weight_general<double>(sp.kind, d, scoef, lk, lk).x;
    double cn = 0.0;
    for (int t = 0; with_frob && t < sp.ntaps; ++t) {
      double lv[MAXD];
      lambda_shift(sp, ib, k, sp.m[t], +1, lk, lv);
      const double2 c = weight_general<double>(sp.kind, d, scoef + t * sp.ncomp, lv, lk);
      cn += c.x * c.x + c.y * c.y;
    }
    double mj = 0.0, mf = 0.0;
    bool nyq_row = false;   // a dropped Nyquist mode of a half-spectrum plan: not an unknown
    for (int j = 0; j < sp.n; ++j) nyq_row |= ib[j] == sp.nyq[j];
    if (e != 0 && !nyq_row) {
      mj = q != 0.0 ? 1.0 / q : 0.0;
      mf = cn > 0.0 ? q / cn : 0.0;
      red[0] = fmin(red[0], l2sum);
      red[1] = fmin(red[1], l2sum > 0.0 ? q : -1.0);   // q(k) > 0 at every k != 0 (only its sign is used)
    }
    jac[e] = mj;
    jac32[e] = (float)mj;
    if (with_frob) {
      frob[e] = mf;
      frob32[e] = (float)mf;
    }
  }
  block_reduce<2, true>(red);
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = red[0];
    partials[gridDim.x + blockIdx.x] = red[1];
    __threadfence();
    is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int q = 0; q < 2; ++q) {
    double v[1] = {DBL_MAX};
    for (int i = threadIdx.x; i < (int)gridDim.x; i += BLOCK) v[0] = fmin(v[0], __ldcg(partials + q * gridDim.x + i));
    block_reduce<1, true>(v);
    if (threadIdx.x == 0) out[q] = v[0];
  }
  if (threadIdx.x == 0) *counter = 0;
}

void launch_diag(const PlanDev* plan_dev, int mc, int D, double* jac, double* frob, float* jac32, float* frob32,
                 double* partials, unsigned* counter, double* out, int nblk, bool with_frob, cudaStream_t s) {
  const size_t smem = (size_t)mc * sizeof(double2);
  k_diag<<<nblk, BLOCK, smem, s>>>(plan_dev, D, jac, frob, jac32, frob32, partials, counter, out, with_frob ? 1 : 0);
  count_launch();
}

// Corrector right-hand sides on the taps backend: F_j = 0 except at the tap modes m != 0, where
// F_j(m) = i sum_a lambda_a(m) A~^{aj}_m (Sec. 5.2 eq. corrector; App. D). F is zeroed beforehand. One block.
__device__ __forceinline__ void rhs_taps_block(const PlanDev* plan, int j0, int nrhs, int D, double2* F) {
  __shared__ __align__(16) PlanDev sp;
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* scoef = reinterpret_cast<double2*>(smraw);
  load_plan<double>(plan, sp, scoef);
  const PlanDev& p = sp;
  for (int idx = threadIdx.x; idx < p.ntaps * nrhs; idx += BLOCK) {
    const int t = idx % p.ntaps, jj = idx / p.ntaps, j = j0 + jj;
    if (t == 0) continue;                      // the mean mode: F(0) = 0
    // (a half-spectrum plan stores the modes with m_{n-1} >= 0; the others are the conjugates of their mirrors)
    if (p.hspec && p.m[t][p.n - 1] < 0) continue;
    int e = 0;
    double lm[MAXD] = {0, 0, 0};
    for (int ax = 0; ax < p.n; ++ax) {
      const int mj = p.m[t][ax];
      e += (mj < 0 ? mj + p.N[ax] : mj) * p.stride[ax];
      for (int a = 0; a < p.d; ++a) lm[a] = fma(p.P[a][ax], (double)mj, lm[a]);
    }
    const double2* ct = scoef + (size_t)t * p.ncomp;
    double2 z = mk<double>(0, 0);
    for (int a = 0; a < p.d; ++a) {
      double2 c;
      if (p.kind == QP_COEF_SCALAR) c = (a == j) ? ct[0] : mk<double>(0, 0);
      else if (p.kind == QP_COEF_DIAG) c = (a == j) ? ct[a] : mk<double>(0, 0);
      else c = ct[sym_idx(a, j, p.d)];
      z.x += lm[a] * c.x;
      z.y += lm[a] * c.y;
    }
    F[(size_t)jj * D + e] = mk<double>(-z.y, z.x);   // i * z
  }
}

__global__ void __launch_bounds__(BLOCK) k_rhs_taps(const PlanDev* plan, int j0, int nrhs, int D, double2* F) {
  rhs_taps_block(plan, j0, nrhs, D, F);
}

// The right-hand sides of several plans, one block per plan (jobs: device table).
__global__ void __launch_bounds__(BLOCK) k_rhs_taps_multi(const PlanJob* jobs) {
  const PlanJob& j = jobs[blockIdx.x];
  rhs_taps_block(j.plan, 0, j.nrhs, j.D, j.F);
}

void launch_rhs_taps(const PlanDev* plan_dev, int mc, int j0, int nrhs, int D, double2* F, cudaStream_t s) {
  k_rhs_taps<<<1, BLOCK, (size_t)mc * sizeof(double2), s>>>(plan_dev, j0, nrhs, D, F);
  count_launch();
}

// F = 0 over every job's nrhs x D right-hand sides (blockIdx.y: job).
__global__ void __launch_bounds__(BLOCK) k_zero_rhs_multi(const PlanJob* jobs) {
  const PlanJob& j = jobs[blockIdx.y];
  const size_t n = (size_t)j.nrhs * j.D;
  for (size_t i = (size_t)blockIdx.x * BLOCK + threadIdx.x; i < n; i += (size_t)gridDim.x * BLOCK)
    j.F[i] = make_double2(0.0, 0.0);
}

void launch_rhs_taps_multi(const PlanJob* jobs, int njobs, int mc, cudaStream_t s) {
  k_zero_rhs_multi<<<dim3(16, njobs), BLOCK, 0, s>>>(jobs);
  k_rhs_taps_multi<<<njobs, BLOCK, (size_t)mc * sizeof(double2), s>>>(jobs);
  count_launch(2);
}

// A*_ij = A~^{ij}_0 + i sum_k sum_b A~^{ib}_{-k} lambda_b(k) U_j(k): on the taps backend only k = -m_t
// contribute. One thread per tap computes its d x d terms; a fixed-order block reduction sums them.
// out: (re, im) per entry, row-major. One block.
__device__ __forceinline__ void astar_taps_block(const PlanDev* plan, int D, const double2* __restrict__ U,
                                                 double* out) {
  __shared__ __align__(16) PlanDev sp;
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* scoef = reinterpret_cast<double2*>(smraw);
  load_plan<double>(plan, sp, scoef);
  const PlanDev& p = sp;
  const int d = p.d;
  auto cab = [&](int t, int a, int b) -> double2 {
    const double2* ct = scoef + (size_t)t * p.ncomp;
    if (p.kind == QP_COEF_SCALAR) return (a == b) ? ct[0] : mk<double>(0, 0);
    if (p.kind == QP_COEF_DIAG) return (a == b) ? ct[a] : mk<double>(0, 0);
    return ct[sym_idx(a, b, d)];
  };
  double v[2 * MAXD * MAXD];
#pragma unroll
  for (int q = 0; q < 2 * MAXD * MAXD; ++q) v[q] = 0.0;
  for (int t = 1 + threadIdx.x; t < p.ntaps; t += BLOCK) {
    int e = 0;
    double lneg[MAXD] = {0, 0, 0};   // lambda(-m_t)
    // U(-m_t): stored at -m_t, or (half-spectrum plan, last component of -m_t negative) the conjugate of U(m_t)
    const bool mirror = p.hspec && p.m[t][p.n - 1] > 0;
    for (int ax = 0; ax < p.n; ++ax) {
      const int mj = -(int)p.m[t][ax];
      const int sj = mirror ? -mj : mj;
      e += (sj < 0 ? sj + p.N[ax] : sj) * p.stride[ax];
      for (int a = 0; a < d; ++a) lneg[a] = fma(p.P[a][ax], (double)mj, lneg[a]);
    }
#pragma unroll
    for (int i = 0; i < MAXD; ++i) {
#pragma unroll
      for (int j = 0; j < MAXD; ++j) {
        if (i < d && j < d) {
          double2 sm = mk<double>(0, 0);
          for (int b = 0; b < d; ++b) {
            const double2 c = cab(t, i, b);
            sm.x += c.x * lneg[b];
            sm.y += c.y * lneg[b];
          }
          double2 u = U[(size_t)j * D + e];
          if (mirror) u.y = -u.y;
          const double pr = sm.x * u.x - sm.y * u.y, pim = sm.x * u.y + sm.y * u.x;
          v[2 * (i * MAXD + j)] += -pim;   // i * (s u)
          v[2 * (i * MAXD + j) + 1] += pr;
        }
      }
    }
  }
  block_reduce<2 * MAXD * MAXD>(v);
  if (threadIdx.x == 0) {
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        const double2 c0 = cab(0, i, j);
        out[2 * (i * d + j)] = c0.x + v[2 * (i * MAXD + j)];
        out[2 * (i * d + j) + 1] = c0.y + v[2 * (i * MAXD + j) + 1];
      }
  }
}

__global__ void __launch_bounds__(BLOCK) k_astar_taps(const PlanDev* plan, int D, const double2* __restrict__ U,
                                                      double* out) {
  astar_taps_block(plan, D, U, out);
}

// a* of several plans, one block per plan (jobs: device table).
__global__ void __launch_bounds__(BLOCK) k_astar_taps_multi(const PlanJob* jobs) {
  const PlanJob& j = jobs[blockIdx.x];
  astar_taps_block(j.plan, j.D, j.U, j.out);
}

void launch_astar_taps(const PlanDev* plan_dev, int mc, int D, const double2* U, double* out, cudaStream_t s) {
  k_astar_taps<<<1, BLOCK, (size_t)mc * sizeof(double2), s>>>(plan_dev, D, U, out);
  count_launch();
}

void launch_astar_taps_multi(const PlanJob* jobs, int njobs, int mc, cudaStream_t s) {
  k_astar_taps_multi<<<njobs, BLOCK, (size_t)mc * sizeof(double2), s>>>(jobs);
  count_launch();
}

}  // namespace qp
