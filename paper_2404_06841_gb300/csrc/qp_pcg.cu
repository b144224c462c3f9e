// PCG update and reduction kernels of Algorithm 2 (C-PCG) over a batch of units, and the FP32/FP64
// iterative-refinement steps around it.
//
// Per iteration: the stiffness apply (qp_taps.cu or the FFT passes) writes w = Q h and reduces (h, w); then
//   pcg_update:  alpha = (r, z) / (h, Q h), r -= alpha Q h, reduce (r, z') with z' = M r and ||r||^2;
//                beta = (r', z') / (r, z); convergence ||r|| <= tol ||F||;
//   pcg_hupdate: U += alpha h and h = M r + beta h in one pass over h (h is read once per iteration for both;
//                a right-hand side that converged in this iteration still gets its last U update).
// z = M r is recomputed where needed instead of stored (the preconditioner is diagonal). Dot products are
// accumulated in FP64 above the warp level whatever the vector precision (FP32 vectors: products and the
// 32-lane warp tree in FP32, every sum above it in FP64). The update kernel's last block sets the CUDA-graph
// conditional that keeps the iteration loop running while some right-hand side is not done.
#include "qp_vec.cuh"

namespace qp {

// ndone[which] = 0; which == 1 also resets the outer (refinement) state of every right-hand side.
__global__ void k_level_reset(BatchDev b, int which) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    b.ndone[which] = 0;
    *b.kcount = 0;
  }
  if (which == 1) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.nunits * MAXR; i += gridDim.x * blockDim.x) {
      RhsSt& x = b.st[i];
      x.outer = 0;
      x.inner_total = 0;
      x.iters = 0;
      x.odone = (i % MAXR) < unit_at(b, i / MAXR).nrhs ? 0 : 1;
      x.ostatus = QP_ERR_NO_CONVERGENCE;
      x.prev_rel = INFINITY;
      x.scale = 0.0;
      x.inv_scale = 0.0;
    }
  }
}

void launch_level_reset(const BatchDev& b, int which, cudaStream_t s) {
  k_level_reset<<<1, BLOCK, 0, s>>>(b, which);
  count_launch();
}

template <typename T> __device__ __forceinline__ const cplx<T>* vF(const UnitDev& u, int level);
template <> __device__ __forceinline__ const double2* vF<double>(const UnitDev& u, int) { return u.F; }
template <> __device__ __forceinline__ const float2* vF<float>(const UnitDev& u, int) { return u.F32; }
template <typename T> __device__ __forceinline__ cplx<T>* vU(const UnitDev& u);
template <> __device__ __forceinline__ double2* vU<double>(const UnitDev& u) { return u.U; }
template <> __device__ __forceinline__ float2* vU<float>(const UnitDev& u) { return u.U32; }
template <typename T> __device__ __forceinline__ cplx<T>* vR(const UnitDev& u);
template <> __device__ __forceinline__ double2* vR<double>(const UnitDev& u) { return u.r; }
template <> __device__ __forceinline__ float2* vR<float>(const UnitDev& u) { return u.r32; }
template <typename T> __device__ __forceinline__ cplx<T>* vH(const UnitDev& u);
template <> __device__ __forceinline__ double2* vH<double>(const UnitDev& u) { return u.h; }
template <> __device__ __forceinline__ float2* vH<float>(const UnitDev& u) { return u.h32; }
template <typename T> __device__ __forceinline__ cplx<T>* vW(const UnitDev& u);
template <> __device__ __forceinline__ double2* vW<double>(const UnitDev& u) { return u.w; }
template <> __device__ __forceinline__ float2* vW<float>(const UnitDev& u) { return u.w32; }
template <typename T> __device__ __forceinline__ const T* vM(const UnitDev& u);
template <> __device__ __forceinline__ const double* vM<double>(const UnitDev& u) { return u.minv64; }
template <> __device__ __forceinline__ const float* vM<float>(const UnitDev& u) { return u.minv32; }

// r = F - w (warm start: w = Q U) or r = F, r(0) = 0, h = M r; FP32 level: U32 = 0, and right-hand sides that
// already meet the outer tolerance start from F = 0. Reduces ||F||^2, (r, M r), ||r||^2.
// HW: compiled for batches with half-spectrum units (their sums weighted per mode); the other batches take the
// form without weights, which keeps its registers and occupancy.
template <typename T, int NR, bool HW>
__global__ void __launch_bounds__(BLOCK) k_pcg_init(BatchDev b, int level, int warm, unsigned long long cond) {
  for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x) {
    const int u = unit_of_chunk(b, c);
    const UnitDev& un = unit_at(b, u);
    RhsSt* st = b.st + (size_t)u * MAXR;
    const int nrhs = un.nrhs, D = un.D;
    const cplx<T>* F = vF<T>(un, level);
    cplx<T>* U = vU<T>(un);
    cplx<T>* r = vR<T>(un);
    cplx<T>* h = vH<T>(un);
    const cplx<T>* w = reinterpret_cast<const cplx<T>*>(vW<T>(un));
    const T* M = vM<T>(un);
    int zero_rhs[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) zero_rhs[k] = (k < nrhs && level == LEVEL_FP32) ? ld_int(&st[k].odone) : 0;
    T vt[3 * NR];
    double v[3 * NR];
#pragma unroll
    for (int q = 0; q < 3 * NR; ++q) vt[q] = T(0);
    const int base = (c - un.chunk0) * un.chunk, end = min(base + un.chunk, D);
    const bool zu = level == LEVEL_FP32;
    if (HW && un.hspec) vec_init<T, NR, true>(un, base, end, D, nrhs, warm != 0, zu, zero_rhs, F, U, r, h, w, M, vt);
    else vec_init<T, NR>(un, base, end, D, nrhs, warm != 0, zu, zero_rhs, F, U, r, h, w, M, vt);
    block_reduce_mixed<T, 3 * NR>(vt, v);
    if (!chunk_arrive<3 * NR>(b, c, u, v)) continue;
    unit_sums<3 * NR>(b, un, v);
    if (threadIdx.x == 0) {
      int nd = 0;
      for (int k = 0; k < nrhs && k < NR; ++k) {
        const double f2 = v[3 * k], rz = v[3 * k + 1], rr = v[3 * k + 2];
        RhsSt& x = st[k];
        x.f2 = f2;
        x.rz = rz;
        x.rr = rr;
        x.iters = 0;
        x.status = QP_OK;
        x.upend = 0;
        x.done = (f2 == 0.0 || rr <= b.tol2 * f2) ? 1 : 0;
        if (!isfinite(rr)) {
          x.done = 1;
          x.status = QP_ERR_BREAKDOWN;
        }
        nd += x.done;
      }
      atomicAdd(&b.ndone[0], nd);
      b.ucount[u] = 0;
      // every unit is initialised here: the last one to finish sets the loop condition once
      __threadfence();
      if (atomicAdd(b.kcount, 1u) == (unsigned)b.nunits - 1u) {
        *b.kcount = 0;
        if (cond != 0ull) cudaGraphSetConditional(cond, ld_int(&b.ndone[0]) < b.nslots ? 1u : 0u);
      }
    }
  }
}

// alpha step on the residual, and the reductions for beta and the convergence test (U is updated by
// k_pcg_hupdate, which reads h anyway). The chunks go against the apply's direction (downwards after the single
// star-1 apply, upwards after the general batch apply): the pass starts where the apply ended, whose Q h is then
// still in L2 (a chunk's partial sums do not depend on the order).
template <typename T, int NR, bool HW>
__global__ void __launch_bounds__(BLOCK) k_pcg_update(BatchDev b, int level, unsigned long long cond) {
  for (int ci = blockIdx.x; ci < b.nchunks; ci += gridDim.x) {
    const int c = b.apply_down ? ci : b.nchunks - 1 - ci;
    const int u = unit_of_chunk(b, c);
    const UnitDev& un = unit_at(b, u);
    RhsSt* st = b.st + (size_t)u * MAXR;
    const int nrhs = un.nrhs, D = un.D;
    int done[NR];
    T alpha[NR];
    bool active = false;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      done[k] = k < nrhs ? ld_int(&st[k].done) : 1;
      alpha[k] = done[k] ? T(0) : (T)__ldcg(&st[k].alpha);
      active |= !done[k];
    }
    if (!active) continue;
    cplx<T>* r = vR<T>(un);
    const cplx<T>* w = vW<T>(un);
    const T* M = vM<T>(un);
    T vt[2 * NR];
    double v[2 * NR];
#pragma unroll
    for (int q = 0; q < 2 * NR; ++q) vt[q] = T(0);
    const int base = (c - un.chunk0) * un.chunk, end = min(base + un.chunk, D);
    if (HW && un.hspec) vec_update<T, NR, true>(un, base, end, D, nrhs, done, alpha, r, w, M, vt);
    else vec_update<T, NR>(un, base, end, D, nrhs, done, alpha, r, w, M, vt);
    block_reduce_mixed<T, 2 * NR>(vt, v);
    if (!chunk_arrive<2 * NR>(b, c, u, v)) continue;
    unit_sums<2 * NR>(b, un, v);
    if (threadIdx.x == 0) {
      int nd = 0;
      for (int k = 0; k < nrhs && k < NR; ++k) {
        if (done[k]) continue;
        const double rz = v[2 * k], rr = v[2 * k + 1];
        RhsSt& x = st[k];
        x.iters += 1;
        x.rr = rr;
        int dn = 0;
        if (!isfinite(rr)) {
          dn = 1;
          x.status = QP_ERR_BREAKDOWN;
        } else if (rr <= b.tol2 * x.f2) {
          dn = 1;
        } else if (x.iters >= b.maxit) {   // iteration cap: also bounds the graph's WHILE loop
          dn = 1;
          x.status = QP_ERR_NO_CONVERGENCE;
        }
        x.beta = rz / x.rz;
        x.rz = rz;
        if (dn) {
          x.done = 1;
          x.upend = 1;   // its last U += alpha h comes in this iteration's k_pcg_hupdate
        }
        nd += dn;
      }
      b.ucount[u] = 0;
      count_done(b, 0, nd, cond);   // the right-hand side that completes the count ends the loop
    }
  }
}

// U += alpha h for the right-hand sides active in this iteration (those that converged in it included), then
// h = M r + beta h for those still running. The last block of a unit clears the pending U updates of its
// converged right-hand sides. The chunks go in the apply's direction, against the update pass before it, so that
// this pass starts where the update ended (its r still in L2).
template <typename T, int NR>
__global__ void __launch_bounds__(BLOCK) k_pcg_hupdate(BatchDev b, int level) {
  for (int ci = blockIdx.x; ci < b.nchunks; ci += gridDim.x) {
    const int c = b.apply_down ? b.nchunks - 1 - ci : ci;
    const int u = unit_of_chunk(b, c);
    const UnitDev& un = unit_at(b, u);
    RhsSt* st = b.st + (size_t)u * MAXR;
    const int nrhs = un.nrhs, D = un.D;
    int upd[NR], hup[NR];
    T alpha[NR], beta[NR];
    bool active = false;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int dn = k < nrhs ? ld_int(&st[k].done) : 1;
      upd[k] = k < nrhs && (!dn || ld_int(&st[k].upend));
      hup[k] = !dn;
      alpha[k] = upd[k] ? (T)__ldcg(&st[k].alpha) : T(0);
      beta[k] = hup[k] ? (T)__ldcg(&st[k].beta) : T(0);
      active |= upd[k] != 0;
    }
    if (!active) continue;
    const cplx<T>* r = vR<T>(un);
    cplx<T>* h = vH<T>(un);
    cplx<T>* U = vU<T>(un);
    const T* M = vM<T>(un);
    const int base = (c - un.chunk0) * un.chunk, end = min(base + un.chunk, D);
    vec_hupdate<T, NR>(base, end, D, nrhs, upd, alpha, hup, beta, r, h, U, M);
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&b.ucount[u], 1u) == (unsigned)un.nchunk - 1u);
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
      for (int k = 0; k < nrhs && k < NR; ++k)
        if (ld_int(&st[k].done)) st[k].upend = 0;
      b.ucount[u] = 0;
    }
  }
}

// Elements a thread of the refinement passes has in flight: their loads are issued before any of their stores.
constexpr int REFINE_ILP = 4;

// Refinement: F32 = 2^-e (F - Q64 U64) for the right-hand sides still refining (2^e <= ||F - Q U|| < 2^(e+1), the
// inverse of the right-hand side's scale): narrow_pow2, no FP64 arithmetic.
__global__ void __launch_bounds__(BLOCK) k_refine_prep(BatchDev b) {
  for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x) {
    const int u = unit_of_chunk(b, c);
    const UnitDev& un = unit_at(b, u);
    const RhsSt* st = b.st + (size_t)u * MAXR;
    const int nrhs = un.nrhs, D = un.D;
    const int base = (c - un.chunk0) * un.chunk, end = min(base + un.chunk, D);
    for (int k = 0; k < nrhs; ++k) {
      if (ld_int(&st[k].odone)) continue;
      const int ex = pow2_exponent(__ldcg(&st[k].inv_scale));
      const double2* w = un.w + (size_t)k * D;
      float2* f = un.F32 + (size_t)k * D;
      for (int e0 = base + threadIdx.x; e0 < end; e0 += REFINE_ILP * BLOCK) {
        double2 v[REFINE_ILP];
#pragma unroll
        for (int i = 0; i < REFINE_ILP; ++i)
          if (e0 + i * BLOCK < end) v[i] = w[e0 + i * BLOCK];
#pragma unroll
        for (int i = 0; i < REFINE_ILP; ++i)
          if (e0 + i * BLOCK < end) f[e0 + i * BLOCK] = make_float2(narrow_pow2(v[i].x, ex), narrow_pow2(v[i].y, ex));
      }
    }
  }
}

// Refinement: U64 += 2^e c32 for the right-hand sides still refining (widen_pow2: exact, one FP64 add per value).
__global__ void __launch_bounds__(BLOCK) k_refine_accum(BatchDev b) {
  for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x) {
    const int u = unit_of_chunk(b, c);
    const UnitDev& un = unit_at(b, u);
    const RhsSt* st = b.st + (size_t)u * MAXR;
    const int nrhs = un.nrhs, D = un.D;
    const int base = (c - un.chunk0) * un.chunk, end = min(base + un.chunk, D);
    for (int k = 0; k < nrhs; ++k) {
      if (ld_int(&st[k].odone)) continue;
      const int ex = pow2_exponent(__ldcg(&st[k].inv_scale));
      const float2* c32 = un.U32 + (size_t)k * D;
      double2* U = un.U + (size_t)k * D;
      for (int e0 = base + threadIdx.x; e0 < end; e0 += REFINE_ILP * BLOCK) {
        float2 cv[REFINE_ILP];
        double2 uv[REFINE_ILP];
#pragma unroll
        for (int i = 0; i < REFINE_ILP; ++i) {
          if (e0 + i * BLOCK < end) {
            cv[i] = c32[e0 + i * BLOCK];
            uv[i] = U[e0 + i * BLOCK];
          }
        }
#pragma unroll
        for (int i = 0; i < REFINE_ILP; ++i) {
          if (e0 + i * BLOCK < end) {
            uv[i].x += widen_pow2(cv[i].x, ex);
            uv[i].y += widen_pow2(cv[i].y, ex);
            U[e0 + i * BLOCK] = uv[i];
          }
        }
      }
    }
  }
}

#define QP_NR_SWITCH(maxr, CALL) \
  switch (maxr) {                  \
    case 1: CALL(1); break;        \
    case 2: CALL(2); break;        \
    case 3: CALL(3); break;        \
    default: CALL(4); break;       \
  }

void launch_pcg_init(const BatchDev& b, int maxr, int level, bool warm, unsigned long long cond, int nblk,
                     cudaStream_t s) {
#define QP_CALL2(NR, HW)                                                                                  \
  if (level == LEVEL_FP32) k_pcg_init<float, NR, HW><<<nblk, BLOCK, 0, s>>>(b, level, warm ? 1 : 0, cond); \
  else k_pcg_init<double, NR, HW><<<nblk, BLOCK, 0, s>>>(b, level, warm ? 1 : 0, cond)
#define QP_CALL(NR)            \
  if (b.hspec_any) {           \
    QP_CALL2(NR, true);        \
  } else {                     \
    QP_CALL2(NR, false);       \
  }
  QP_NR_SWITCH(maxr, QP_CALL)
#undef QP_CALL
#undef QP_CALL2
  count_launch();
}
void launch_pcg_update(const BatchDev& b, int maxr, int level, unsigned long long cond, int nblk, cudaStream_t s) {
#define QP_CALL2(NR, HW)                                                                      \
  if (level == LEVEL_FP32) k_pcg_update<float, NR, HW><<<nblk, BLOCK, 0, s>>>(b, level, cond); \
  else k_pcg_update<double, NR, HW><<<nblk, BLOCK, 0, s>>>(b, level, cond)
#define QP_CALL(NR)            \
  if (b.hspec_any) {           \
    QP_CALL2(NR, true);        \
  } else {                     \
    QP_CALL2(NR, false);       \
  }
  QP_NR_SWITCH(maxr, QP_CALL)
#undef QP_CALL
#undef QP_CALL2
  count_launch();
}
void launch_pcg_hupdate(const BatchDev& b, int maxr, int level, int nblk, cudaStream_t s) {
#define QP_CALL(NR)                                                                 \
  if (level == LEVEL_FP32) k_pcg_hupdate<float, NR><<<nblk, BLOCK, 0, s>>>(b, level); \
  else k_pcg_hupdate<double, NR><<<nblk, BLOCK, 0, s>>>(b, level)
  QP_NR_SWITCH(maxr, QP_CALL)
#undef QP_CALL
  count_launch();
}
void launch_refine_prep(const BatchDev& b, int nblk, cudaStream_t s) {
  k_refine_prep<<<nblk, BLOCK, 0, s>>>(b);
  count_launch();
}
void launch_refine_accum(const BatchDev& b, int nblk, cudaStream_t s) {
  k_refine_accum<<<nblk, BLOCK, 0, s>>>(b);
  count_launch();
}

}  // namespace qp
