// Persistent form of the PCG solve (Algorithm 2) for one taps-backend plan: the whole solve, including the
// FP64 iterative-refinement loop around FP32 inner solves, runs in one cooperative launch whose blocks meet at
// grid barriers instead of kernel boundaries. For small and medium problems, where one PCG iteration is a few
// microseconds of memory traffic, this removes the per-kernel launch, fence and atomic latency of the graph
// form (three kernels per iteration).
//
// The arithmetic is the graph form's: the same stencil (apply_run), the same per-element updates, the same
// per-chunk partial sums (block tree; FP32 warp level for FP32 vectors), and the same fixed-order sum over the
// chunks, which every block now computes for itself after a barrier instead of one finalizing block. Iterates,
// iteration counts and a* are therefore bitwise those of the graph form. Consecutive reductions write
// disjoint partial slots, so a block may start the next phase while another still sums the previous one.
//
// Every barrier wait is bounded (%globaltimer): a block that waits longer than the limit sets the error flag;
// every block returns as soon as it sees the flag, and the host reports QP_ERR_TIMEOUT.
#pragma once
#include "qp_stencil.cuh"
#include "qp_vec.cuh"

namespace qp {

namespace {

constexpr int S_INIT = 0, S_HW = 12, S_UPD = 16, S_RES = 24;   // partial slots of the four reductions
// stencil runs of two modes as in the graph form (the plan's last axis has even length)
template <typename T> __host__ __device__ constexpr int prun() { return 2; }
static_assert(S_HW >= 3 * MAXR && S_UPD >= S_HW + MAXR && S_RES >= S_UPD + 2 * MAXR &&
                  NSLOT_PERSIST >= S_RES + 2 * MAXR,
              "persistent partial slots overlap");

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned atom_add_release(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier with a bounded wait; false (in every thread of the block) on timeout or error.
// bar[0] counts arrivals over the whole launch: the k-th barrier is passed once it reaches (k + 1) * gridDim.x.
// Each block's thread 0 arrives with one release-ordered atomic add (after the block barrier, so it publishes
// the block's writes) and polls with acquire loads; no separate fences and no reset step. A single-block grid
// needs only the block barrier.
__device__ __noinline__ bool grid_barrier(unsigned* bar, int* err, unsigned long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (gridDim.x == 1) return true;
  if (threadIdx.x == 0) {
    const unsigned ticket = atom_add_release(bar, 1u);
    const unsigned target = (ticket / gridDim.x + 1u) * gridDim.x;
    int ok = 1;
    if ((int)(ld_acquire(bar) - target) < 0) {
      const unsigned long long t0 = global_ns();
      for (;;) {
        if ((int)(ld_acquire(bar) - target) >= 0) break;
        if (*((volatile int*)err)) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > timeout_ns) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok && !*((volatile int*)err);
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ bool grid_sync(const PersistArgs& a) { return grid_barrier(a.bar, a.err, a.timeout_ns); }

// The fixed-order sum over the unit's chunks of slots slot0 .. slot0 + NV - 1, in every thread.
template <int NV>
__device__ __forceinline__ void all_sums(const BatchDev& b, const UnitDev& un, int slot0, double (&v)[NV]) {
  __shared__ double s_v[NV];
  unit_sums<NV>(b, un, v, slot0);
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) s_v[q] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = s_v[q];
  __syncthreads();
}

template <int NV>
__device__ __forceinline__ void store_partials(const BatchDev& b, int c, int slot0, const double (&v)[NV]) {
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) b.partials[(size_t)(slot0 + q) * b.nchunks + c] = v[q];
}

__device__ __forceinline__ void chunk_range(const UnitDev& un, int c, int& base, int& end) {
  base = (c - un.chunk0) * un.chunk;
  end = min(base + un.chunk, un.D);
}

// ---- phases over one chunk of modes (thread t handles modes base + t, base + t + BLOCK, ...: the mapping of
//      the graph-form kernels, so that the per-chunk partial sums are the same). The persistent form runs
//      full-spectrum plans only (half-spectrum solves run as graphs), so its sums carry no mode weights.

// r = F - w (warm) or F, r(0) = 0, h = M r; U = 0 where asked; reduces ||F||^2, (r, M r), ||r||^2.
template <typename T, int NR>
__device__ __forceinline__ void ph_init(const BatchDev& b, const UnitDev& un, int c, bool warm, bool zero_u,
                                        const int* zero_rhs, const cplx<T>* F, cplx<T>* U, cplx<T>* r, cplx<T>* h,
                                        const cplx<T>* w, const T* M) {
  const int D = un.D, nrhs = un.nrhs;
  T vt[3 * NR];
  double v[3 * NR];
#pragma unroll
  for (int q = 0; q < 3 * NR; ++q) vt[q] = T(0);
  int base, end;
  chunk_range(un, c, base, end);
  vec_init<T, NR>(un, base, end, D, nrhs, warm, zero_u, zero_rhs, F, U, r, h, w, M, vt);
  block_reduce_mixed<T, 3 * NR>(vt, v);
  store_partials<3 * NR>(b, c, S_INIT, v);
}

// dst = Q src with the epilogue: EPI_DOT_HW reduces (src, dst); EPI_RESIDUAL writes F - Q src (0 at k = 0) and
// reduces its norm and ||F||^2 over k != 0; EPI_NONE writes Q src.
// SK: 0 the plan's stencil from shared memory; 1 / 2 the star-1 stencil of a scalar / diagonal coefficient
// from st (the kernel parameter; FP64 from the plan's stored weights).
template <typename T, bool REALC, int NR, int EPI, int SK, int NAX = 0, int DC = 0>
__device__ __forceinline__ void ph_apply(const BatchDev& b, const UnitDev& un, int c, const PlanDev& sp,
                                         const cplx<T>* scoef, const StarParams& st, const cplx<T>* src,
                                         cplx<T>* dst, const cplx<T>* F, bool zero_src = false) {
  const int D = un.D, nrhs = un.nrhs;
  constexpr int NV = (EPI == EPI_RESIDUAL) ? 2 * NR : NR;
  T vt[NV];
  double v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) vt[q] = T(0);
  constexpr int PRUN = prun<T>();
  int start, stride, limit;
  chunk_runs<T>(un, c - un.chunk0, PRUN, start, stride, limit);   // the graph form's runs of this chunk
  for (int e0 = start; e0 < limit; e0 += stride) {
    cplx<T> acc[PRUN][NR];
    if (zero_src) {   // src = 0: Q src = 0
#pragma unroll
      for (int s = 0; s < PRUN; ++s)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[s][r] = mk<T>(0, 0);
    } else if constexpr (SK != 0) {
      // FP64 level: the plan's stored weights; FP32 level: formed
      apply_run_star<T, REALC, NR, false, SK == 2, sizeof(T) == 8 ? 1 : 0, NAX, DC>(st, e0, src, D, nrhs, acc);
    } else {
      apply_run<T, REALC, NR, PRUN, false>(sp, scoef, e0, src, D, nrhs, acc);
    }
    if constexpr (sizeof(T) == 4 && EPI == EPI_DOT_HW) {
      // FP32: one 16-byte store and load per right-hand side, the sums in the graph form's order (plain loads:
      // this kernel writes h in another phase)
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (r < nrhs) {
          const size_t o = (size_t)r * D + e0;
          *reinterpret_cast<float4*>(dst + o) = make_float4((float)acc[0][r].x, (float)acc[0][r].y,
                                                            (float)acc[1][r].x, (float)acc[1][r].y);
          const float4 hv = *reinterpret_cast<const float4*>(src + o);
          vt[r] = fma((T)hv.x, acc[0][r].x, fma((T)hv.y, acc[0][r].y, vt[r]));
          vt[r] = fma((T)hv.z, acc[1][r].x, fma((T)hv.w, acc[1][r].y, vt[r]));
        }
      }
      continue;
    }
#pragma unroll
    for (int s = 0; s < PRUN; ++s) {
      const int e = e0 + s;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (r < nrhs) {
          const size_t o = (size_t)r * D + e;
          if (EPI == EPI_DOT_HW) {
            dst[o] = acc[s][r];
            const cplx<T> hv = src[o];
            vt[r] = fma(hv.x, acc[s][r].x, fma(hv.y, acc[s][r].y, vt[r]));
          } else if (EPI == EPI_RESIDUAL) {
            const cplx<T> f = F[o];
            const cplx<T> res = (e == 0) ? mk<T>(0, 0) : mk<T>(f.x - acc[s][r].x, f.y - acc[s][r].y);
            dst[o] = res;
            vt[2 * r] = fma(res.x, res.x, fma(res.y, res.y, vt[2 * r]));
            if (e != 0) vt[2 * r + 1] = fma(f.x, f.x, fma(f.y, f.y, vt[2 * r + 1]));
          } else {
            dst[o] = acc[s][r];
          }
        }
      }
    }
  }
  if (EPI == EPI_NONE) return;
  block_reduce_mixed<T, NV>(vt, v);
  store_partials<NV>(b, c, EPI == EPI_RESIDUAL ? S_RES : S_HW, v);
}

// r -= alpha w; reduces (r, M r) and ||r||^2 (U is updated in the h-update phase, as in the graph form).
template <typename T, int NR>
__device__ __forceinline__ void ph_update(const BatchDev& b, const UnitDev& un, int c, const int* done,
                                          const T* alpha, cplx<T>* r, const cplx<T>* w, const T* M) {
  const int D = un.D, nrhs = un.nrhs;
  T vt[2 * NR];
  double v[2 * NR];
#pragma unroll
  for (int q = 0; q < 2 * NR; ++q) vt[q] = T(0);
  int base, end;
  chunk_range(un, c, base, end);
  vec_update<T, NR>(un, base, end, D, nrhs, done, alpha, r, w, M, vt);
  block_reduce_mixed<T, 2 * NR>(vt, v);
  store_partials<2 * NR>(b, c, S_UPD, v);
}

// U += alpha h for the right-hand sides active in this iteration (act), h = M r + beta h for those still running.
template <typename T, int NR>
__device__ __forceinline__ void ph_hupdate(const UnitDev& un, int c, const int* act, const T* alpha, const int* done,
                                           const T* beta, const cplx<T>* r, cplx<T>* h, cplx<T>* U, const T* M) {
  int hup[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) hup[k] = !done[k];
  int base, end;
  chunk_range(un, c, base, end);
  vec_hupdate<T, NR>(base, end, un.D, un.nrhs, act, alpha, hup, beta, r, h, U, M);
}

template <typename T> struct LevelVecs {
  const cplx<T>* F;
  cplx<T>* U;
  cplx<T>* r;
  cplx<T>* h;
  cplx<T>* w;
  const T* M;
};
__device__ __forceinline__ LevelVecs<double> level_vecs(const UnitDev& un, double) {
  return {un.F, un.U, un.r, un.h, un.w, un.minv64};
}
__device__ __forceinline__ LevelVecs<float> level_vecs(const UnitDev& un, float) {
  return {un.F32, un.U32, un.r32, un.h32, un.w32, un.minv32};
}

// One PCG solve (Algorithm 2) at vector precision T on the unit's vectors of that level, to the relative
// tolerance sqrt(tol2), at most maxit iterations. The solver state lives in ls (shared, written by thread 0).
// zero_rhs marks right-hand sides started from F = 0 (refinement: already converged). zero_u: U = 0 first (T =
// float always; FP64 without a warm start). Returns false on a barrier timeout.
template <typename T, bool REALC, int NR, int SK, int NAX = 0, int DC = 0>
__device__ __forceinline__ bool pcg_solve_block(const PersistArgs& a, const UnitDev& un, const PlanDev& sp, const cplx<T>* scoef,
                                bool warm, bool zero_u, RhsSt* ls, const int* zero_rhs, double tol2, int maxit) {
  const BatchDev& b = a.b;
  const int nrhs = un.nrhs;
  const LevelVecs<T> L = level_vecs(un, T(0));
  __shared__ int s_done[MAXR], s_act[MAXR];
  __shared__ T s_coef[MAXR], s_alpha[MAXR];
  if (warm) {
    for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x)
      ph_apply<T, REALC, NR, EPI_NONE, SK, NAX, DC>(b, un, c, sp, scoef, a.star, L.U, L.w, L.F);
    if (!grid_sync(a)) return false;
  }
  for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x)
    ph_init<T, NR>(b, un, c, warm, zero_u, zero_rhs, L.F, L.U, L.r, L.h, L.w, L.M);
  if (!grid_sync(a)) return false;
  {
    double v[3 * NR];
    all_sums<3 * NR>(b, un, S_INIT, v);
    if (threadIdx.x == 0) {
      for (int k = 0; k < nrhs && k < NR; ++k) {
        RhsSt& x = ls[k];
        x.f2 = v[3 * k];
        x.rz = v[3 * k + 1];
        x.rr = v[3 * k + 2];
        x.iters = 0;
        x.status = QP_OK;
        x.done = (x.f2 == 0.0 || x.rr <= tol2 * x.f2) ? 1 : 0;
        if (!isfinite(x.rr)) {
          x.done = 1;
          x.status = QP_ERR_BREAKDOWN;
        }
      }
    }
    __syncthreads();
  }
  for (int it = 0; it <= maxit; ++it) {
    bool all = true;
    for (int k = 0; k < nrhs && k < NR; ++k) all = all && ls[k].done;
    if (all) break;
    // w = Q h and (h, w); alpha = (r, z) / (h, Q h)
    for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x)
      ph_apply<T, REALC, NR, EPI_DOT_HW, SK, NAX, DC>(b, un, c, sp, scoef, a.star, L.h, L.w, L.F);
    if (!grid_sync(a)) return false;
    {
      double v[NR];
      all_sums<NR>(b, un, S_HW, v);
      if (threadIdx.x == 0) {
        for (int k = 0; k < nrhs && k < NR; ++k) {
          RhsSt& x = ls[k];
          if (x.done) continue;
          x.hw = v[k];
          if (!(v[k] > 0.0) || !isfinite(v[k])) {   // (h, Q h) <= 0 or NaN: breakdown
            x.done = 1;
            x.status = QP_ERR_BREAKDOWN;
          } else {
            x.alpha = x.rz / v[k];
          }
        }
      }
      __syncthreads();
      if (threadIdx.x < MAXR) {
        const int k = threadIdx.x;
        s_done[k] = k < nrhs ? ls[k].done : 1;
        s_act[k] = !s_done[k];
        s_alpha[k] = s_done[k] ? T(0) : (T)ls[k].alpha;
      }
      __syncthreads();
    }
    for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x)
      ph_update<T, NR>(b, un, c, s_done, s_alpha, L.r, L.w, L.M);
    if (!grid_sync(a)) return false;
    {
      double v[2 * NR];
      all_sums<2 * NR>(b, un, S_UPD, v);
      if (threadIdx.x == 0) {
        for (int k = 0; k < nrhs && k < NR; ++k) {
          if (s_done[k]) continue;
          RhsSt& x = ls[k];
          const double rz = v[2 * k], rr = v[2 * k + 1];
          x.iters += 1;
          x.rr = rr;
          int dn = 0;
          if (!isfinite(rr)) {
            dn = 1;
            x.status = QP_ERR_BREAKDOWN;
          } else if (rr <= tol2 * x.f2) {
            dn = 1;
          } else if (x.iters >= maxit) {
            dn = 1;
            x.status = QP_ERR_NO_CONVERGENCE;
          }
          x.beta = rz / x.rz;
          x.rz = rz;
          if (dn) x.done = 1;
        }
      }
      __syncthreads();
      if (threadIdx.x < MAXR) {
        const int k = threadIdx.x;
        s_done[k] = k < nrhs ? ls[k].done : 1;
        s_coef[k] = s_done[k] ? T(0) : (T)ls[k].beta;
      }
      __syncthreads();
    }
    // U += alpha h for this iteration's right-hand sides, h = M r + beta h for those still running
    for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x)
      ph_hupdate<T, NR>(un, c, s_act, s_alpha, s_done, s_coef, L.r, L.h, L.U, L.M);
    if (!grid_sync(a)) return false;
    bool all2 = true;
    for (int k = 0; k < nrhs && k < NR; ++k) all2 = all2 && s_done[k];
    if (all2) break;
  }
  return true;
}

// FP64 true residual w = F - Q U and its reduction; every thread gets (|r|^2, |F|^2) per right-hand side.
// zero_u: U = 0, so w = F without an apply.
template <bool REALC, int NR, int SK, int NAX = 0, int DC = 0>
__device__ __forceinline__ bool true_residual(const PersistArgs& a, const UnitDev& un, const PlanDev& sp, const double2* sc64,
                              double (&v)[2 * NR], bool zero_u = false) {
  const BatchDev& b = a.b;
  for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x)
    ph_apply<double, REALC, NR, EPI_RESIDUAL, SK, NAX, DC>(b, un, c, sp, sc64, a.star, un.U, un.w, un.F, zero_u);
  if (!grid_sync(a)) return false;
  all_sums<2 * NR>(b, un, S_RES, v);
  return true;
}

// NAX, DC (0: from the plan at run time): the number of axes (every one with taps) and d compiled into the FP32
// level's star-1 stencil, and with FIX64 into the FP64 level's too.
template <bool REALC, int NR, int SK, int NAX = 0, int DC = 0, bool FIX64 = false>
__global__ void __launch_bounds__(BLOCK, NR >= 3 ? 1 : 2) k_pcg_persistent(const __grid_constant__ PersistArgs a) {
  __shared__ __align__(16) PlanDev sp;
  __shared__ RhsSt ls[MAXR];
  __shared__ int s_zero[MAXR];
  extern __shared__ __align__(16) unsigned char smraw[];
  const BatchDev& b = a.b;
  const UnitDev& un = b.pu;
  const int nrhs = un.nrhs, D = un.D;
  const bool refine = a.mode == QP_MODE_FP32_REFINE;
  // coefficient tables in shared memory: FP64, then (refinement) FP32
  double2* sc64 = reinterpret_cast<double2*>(smraw);
  load_plan<double>(un.plan, sp, sc64);
  const int nc = sp.ntaps * sp.ncomp;
  float2* sc32 = reinterpret_cast<float2*>(smraw + (size_t)nc * sizeof(double2));
  if (refine)
    for (int i = threadIdx.x; i < nc; i += BLOCK) sc32[i] = sp.coef32[i];
  if (threadIdx.x < MAXR) {
    RhsSt& x = ls[threadIdx.x];
    x = RhsSt{};
    x.prev_rel = INFINITY;
    x.odone = threadIdx.x < nrhs ? 0 : 1;
    x.ostatus = QP_ERR_NO_CONVERGENCE;
    x.done = 1;
    s_zero[threadIdx.x] = 0;
  }
  __syncthreads();
  bool ok = true;
  if (!refine) {
    ok = pcg_solve_block<double, REALC, NR, SK, FIX64 ? NAX : 0, FIX64 ? DC : 0>(a, un, sp, sc64, a.warm != 0, a.warm == 0, ls, s_zero, b.tol2,
                                                b.maxit);
    if (ok) {
      double v[2 * NR];
      ok = true_residual<REALC, NR, SK, FIX64 ? NAX : 0, FIX64 ? DC : 0>(a, un, sp, sc64, v);
      if (ok && threadIdx.x == 0)
        for (int k = 0; k < nrhs && k < NR; ++k) {
          ls[k].orr = v[2 * k];
          ls[k].of2 = v[2 * k + 1];
        }
    }
  } else {
    if (!a.warm) {
      for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x) {
        int base, end;
        chunk_range(un, c, base, end);
        for (int k = 0; k < nrhs; ++k)
          for (int e = base + threadIdx.x; e < end; e += BLOCK) un.U[(size_t)k * D + e] = make_double2(0.0, 0.0);
      }
      ok = grid_sync(a);
    }
    for (int outer = 0; ok && outer <= b.max_outer + 1; ++outer) {
      // FP64 true residual: the outer convergence test and the scale of the next inner right-hand side
      double v[2 * NR];
      if (!(ok = true_residual<REALC, NR, SK, FIX64 ? NAX : 0, FIX64 ? DC : 0>(a, un, sp, sc64, v,
                                                                              outer == 0 && !a.warm)))
        break;
      if (threadIdx.x == 0) {
        for (int k = 0; k < nrhs && k < NR; ++k) {
          RhsSt& x = ls[k];
          if (x.odone) continue;
          const double s0 = v[2 * k], s1 = v[2 * k + 1];
          x.orr = s0;
          x.of2 = s1;
          x.outer += 1;
          x.inner_total += x.iters;
          const double rel = s1 > 0.0 ? sqrt(s0 / s1) : 0.0;
          int od = 0, os = QP_ERR_NO_CONVERGENCE;
          if (s1 == 0.0 || s0 <= b.otol2 * s1) {
            od = 1;
            os = QP_OK;
          } else if (!isfinite(rel)) {
            od = 1;
            os = QP_ERR_BREAKDOWN;
          } else if (rel > 0.9 * x.prev_rel || x.outer > b.max_outer || x.inner_total >= b.maxit) {
            od = 1;   // stagnation or cap
          }
          x.prev_rel = rel;
          refine_scale(s0, x.scale, x.inv_scale);
          x.ostatus = os;
          if (od) x.odone = 1;
        }
      }
      __syncthreads();
      if (threadIdx.x < MAXR) s_zero[threadIdx.x] = threadIdx.x < nrhs ? ls[threadIdx.x].odone : 1;
      __syncthreads();
      bool all = true;
      for (int k = 0; k < nrhs && k < NR; ++k) all = all && s_zero[k];
      if (all) break;
      // F32 = r64 2^-e (2^e <= |r64| < 2^(e+1)) for the right-hand sides still refining
      for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x) {
        int base, end;
        chunk_range(un, c, base, end);
        for (int k = 0; k < nrhs; ++k) {
          if (s_zero[k]) continue;
          const int ex = pow2_exponent(ls[k].inv_scale);
          for (int e = base + threadIdx.x; e < end; e += BLOCK) {
            const size_t o = (size_t)k * D + e;
            const double2 wv = un.w[o];
            un.F32[o] = make_float2(narrow_pow2(wv.x, ex), narrow_pow2(wv.y, ex));
          }
        }
      }
      // the inner init reads F32 in this block's chunks only, with its own mapping of modes to threads: a block
      // barrier before it suffices
      __syncthreads();
      if (!(ok = pcg_solve_block<float, REALC, NR, SK, NAX, DC>(a, un, sp, sc32, false, true, ls, s_zero, b.tol2, b.maxit)))
        break;
      // U64 += 2^e c32 for the right-hand sides still refining
      for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x) {
        int base, end;
        chunk_range(un, c, base, end);
        for (int k = 0; k < nrhs; ++k) {
          if (s_zero[k]) continue;
          const int ex = pow2_exponent(ls[k].inv_scale);
          for (int e = base + threadIdx.x; e < end; e += BLOCK) {
            const size_t o = (size_t)k * D + e;
            const float2 cv = un.U32[o];
            double2 uv = un.U[o];
            uv.x += widen_pow2(cv.x, ex);
            uv.y += widen_pow2(cv.y, ex);
            un.U[o] = uv;
          }
        }
      }
      if (!(ok = grid_sync(a))) break;
    }
  }
  if (!ok) return;
  // the excluded mean mode U(0) = 0 and the final solver state (block 0; nothing reads U any more)
  if (blockIdx.x == 0) {
    if (threadIdx.x < nrhs) un.U[(size_t)threadIdx.x * D] = make_double2(0.0, 0.0);
    if (threadIdx.x < MAXR) b.st[threadIdx.x] = ls[threadIdx.x];
  }
}

}  // namespace

}  // namespace qp
