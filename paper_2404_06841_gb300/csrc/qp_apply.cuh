// The stiffness-apply kernels of the taps backend (batch apply with the PCG epilogues, plain apply), shared by
// the translation units that instantiate them per vector precision and epilogue (qp_apply_*.cu), so that the
// instantiations compile in parallel.
#pragma once
#include "qp_stencil.cuh"

namespace qp {

// ------------------------------------------------------------------------------------------------ batch apply

// One chunk (cl) of a unit: dst = Q src with the epilogue, per-thread partials into vt. Thread t takes the runs
// of RUN consecutive modes chunk_runs gives it.
// SK: the stencil's data source: 0 the plan in shared memory (apply_run), 1 / 2 the star-1 stencil of a scalar /
// diagonal coefficient from st (a kernel parameter).
template <typename T, int EPI, bool REALC, int NR, int RUN, int NV, int SK = 0, int NAX = 0, int DC = 0,
          bool HSP = false, int NG = 0>
__device__ __forceinline__ void apply_chunk(const PlanDev& sp, const cplx<T>* scoef, const StarParams& st,
                                            const UnitDev& un, int cl, int D, int nrhs, int refine, bool fft_unit,
                                            const cplx<T>* src, cplx<T>* dst, const cplx<T>* F, T (&vt)[NV]) {
  int start, stride, limit;
  chunk_runs<T>(un, cl, RUN, start, stride, limit);
  // half-spectrum units weigh each mode 1 or 2 in the sums (mode_weight); the star-1 kernels are compiled per
  // storage, so the full-spectrum ones carry no weights (an FP64 multiply per term is not free)
  const bool hw = (SK == 0 || HSP) && un.hspec;
  for (int e0 = start; e0 < limit; e0 += stride) {
    cplx<T> acc[RUN][NR];
    if (EPI == EPI_RESIDUAL && refine == REFINE_ZERO_U) {
#pragma unroll
      for (int s = 0; s < RUN; ++s)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[s][r] = mk<T>(0, 0);
    } else if (fft_unit) {
#pragma unroll
      for (int s = 0; s < RUN; ++s)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[s][r] = (r < nrhs) ? dst[(size_t)r * D + e0 + s] : mk<T>(0, 0);
    } else if constexpr (SK != 0 && RUN == 2) {
      // FP64: the plan's stored weights; FP32: formed
      apply_run_star<T, REALC, NR, true, SK == 2, sizeof(T) == 8 ? 1 : 0, NAX, DC, HSP>(st, e0, src, D, nrhs, acc);
    } else {
      apply_run<T, REALC, NR, RUN, true, true, 0, NG>(sp, scoef, e0, src, D, nrhs, acc);
    }
    if constexpr (RUN == 2 && sizeof(T) == 4 && EPI != EPI_RESIDUAL) {
      // FP32 runs of two: one 16-byte store (and load of h) per right-hand side; the sums in the order below
      if (!fft_unit) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r < nrhs) {
            const size_t o = (size_t)r * D + e0;
            *reinterpret_cast<float4*>(dst + o) = make_float4((float)acc[0][r].x, (float)acc[0][r].y,
                                                              (float)acc[1][r].x, (float)acc[1][r].y);
            if (EPI == EPI_DOT_HW) {
              const T w0 = hw ? (T)mode_weight(un, e0) : T(1), w1 = hw ? (T)mode_weight(un, e0 + 1) : T(1);
              const float4 hv = __ldg(reinterpret_cast<const float4*>(src + o));
              vt[r] = fma(w0 * (T)hv.x, acc[0][r].x, fma(w0 * (T)hv.y, acc[0][r].y, vt[r]));
              vt[r] = fma(w1 * (T)hv.z, acc[1][r].x, fma(w1 * (T)hv.w, acc[1][r].y, vt[r]));
            }
          }
        }
        continue;
      }
    }
#pragma unroll
    for (int s = 0; s < RUN; ++s) {
      const int e = e0 + s;
      const T we = (EPI == EPI_NONE || !hw) ? T(1) : (T)mode_weight(un, e);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (r < nrhs) {
          const size_t o = (size_t)r * D + e;
          if (EPI == EPI_DOT_HW) {
            if (!fft_unit) dst[o] = acc[s][r];
            const cplx<T> hv = src[o];
            vt[r] = fma(we * hv.x, acc[s][r].x, fma(we * hv.y, acc[s][r].y, vt[r]));
          } else if (EPI == EPI_RESIDUAL) {
            const cplx<T> f = F[o];
            const cplx<T> res = (e == 0) ? mk<T>(0, 0) : mk<T>(f.x - acc[s][r].x, f.y - acc[s][r].y);
            dst[o] = res;
            vt[2 * r] = fma(we * res.x, res.x, fma(we * res.y, res.y, vt[2 * r]));
            if (e != 0) vt[2 * r + 1] = fma(we * f.x, f.x, fma(we * f.y, f.y, vt[2 * r + 1]));
          } else {
            if (!fft_unit) dst[o] = acc[s][r];
          }
        }
      }
    }
  }
}

// The block that completes a unit's chunks sums them and updates its right-hand sides' solver state (a call of its
// own: it runs once per unit and launch, and its registers stay out of the chunk loop).
template <int EPI, int NR, int NV>
__device__ __noinline__ void unit_finalize(const BatchDev& b, const UnitDev& un, RhsSt* st, int nrhs, int refine,
                                           unsigned long long cond, double (&v)[NV]) {
  unit_sums<NV>(b, un, v);
  for (int r = 0; r < nrhs && r < NR; ++r) {
    const double s0 = (EPI == EPI_RESIDUAL) ? v[2 * r] : v[r];
    const double s1 = (EPI == EPI_RESIDUAL) ? v[(2 * r + 1) % NV] : 0.0;
    if (threadIdx.x == 0) {
      RhsSt& x = st[r];
      if (EPI == EPI_DOT_HW) {
        if (!x.done) {
          x.hw = s0;
          if (!(s0 > 0.0) || !isfinite(s0)) {   // (h, Q h) <= 0 or NaN: breakdown
            x.done = 1;
            x.status = QP_ERR_BREAKDOWN;
            count_done(b, 0, 1, cond);           // completing the count here ends the PCG loop
          } else {
            x.alpha = x.rz / s0;
          }
        }
      } else if (!refine) {
        x.orr = s0;
        x.of2 = s1;
      } else if (!x.odone) {
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
        if (od) {
          x.odone = 1;
          count_done(b, 1, 1, cond);             // the right-hand side that completes the count ends the loop
        }
      }
    }
  }
}

static __device__ PlanDev g_no_plan;   // the plan argument of apply_chunk, which the star-1 stencil does not read

// A batch of one star-1 unit (the star kernels; the unit and its stencil come from the kernel parameters). A block
// walks its chunks c, c + grid, ... without a block barrier per chunk: each warp keeps its warp sums of the chunk in
// shared memory, and every NS chunks (and after its last one) the block combines them per chunk as
// block_reduce_mixed does and stores the chunk partials, the same values in the same order; the block counts its
// chunks' arrival once, after its last chunk (per chunk, the fence and the atomic cost 12 of the 314 us of the
// 16^6 FP32 apply, the block barrier 2).
// NS = 3 pending chunks: the 16^6 apply walks four chunks per block, so both flushes (full and last) run there.
template <typename T, int EPI, bool REALC, int NR, int SK, int NAX, int DC, bool HSP>
__device__ __forceinline__ void apply_single_star(const BatchDev& b, int level, int refine, unsigned long long cond,
                                                  const StarParams& stp) {
  constexpr int NV = (EPI == EPI_RESIDUAL) ? 2 * NR : NR;
  constexpr int NS = 3, NW = BLOCK / 32;
  const UnitDev& un = b.pu;
  RhsSt* st = b.st;
  const int nrhs = un.nrhs;
  bool active = false;   // the same for every chunk: only this launch's finalizer changes it, after every chunk
  for (int r = 0; r < nrhs; ++r) {
    if (EPI == EPI_DOT_HW) active |= !ld_int(&st[r].done);
    else if (EPI == EPI_RESIDUAL && refine) active |= !ld_int(&st[r].odone);
    else active = true;
  }
  if (!active) return;
  const int D = un.D;
  const cplx<T>* src;
  cplx<T>* dst;
  if (level == LEVEL_FP32) {
    src = reinterpret_cast<const cplx<T>*>(un.h32);
    dst = reinterpret_cast<cplx<T>*>(un.w32);
  } else {
    src = reinterpret_cast<const cplx<T>*>(EPI == EPI_DOT_HW ? (const double2*)un.h : (const double2*)un.U);
    dst = reinterpret_cast<cplx<T>*>(un.w);
  }
  const cplx<T>* F = reinterpret_cast<const cplx<T>*>(un.F);
  __shared__ double wsum[NS][NV][NW];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int pend = 0, cfirst = blockIdx.x;
  unsigned mine = 0;
  for (int c = blockIdx.x; c < b.nchunks; c += gridDim.x) {
    T vt[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) vt[q] = T(0);
    apply_chunk<T, EPI, REALC, NR, 2, NV, SK, NAX, DC, HSP>(g_no_plan, nullptr, stp, un, c - un.chunk0, D,
                                                           NAX != 0 ? NR : nrhs, refine, false, src, dst, F, vt);
    if (EPI == EPI_NONE) continue;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      if (sizeof(T) == 4) vt[q] = (T)warp_sum_f((float)vt[q]);
      else vt[q] = (T)warp_sum((double)vt[q]);
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < NV; ++q) wsum[pend][q][wid] = (double)vt[q];
    }
    ++pend;
    ++mine;
    if (pend == NS || c + (int)gridDim.x >= b.nchunks) {
      __syncthreads();
      if (wid == 0) {
        for (int i = 0; i < pend; ++i) {
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            const double x = warp_sum(lane < NW ? wsum[i][q][lane] : 0.0);
            if (lane == 0) b.partials[(size_t)q * b.nchunks + cfirst + i * (int)gridDim.x] = x;
          }
        }
      }
      __syncthreads();
      cfirst += pend * (int)gridDim.x;
      pend = 0;
    }
  }
  if (EPI == EPI_NONE || mine == 0) return;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(&b.ucount[0], mine) + mine == (unsigned)un.nchunk) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double v[NV];
  unit_finalize<EPI, NR, NV>(b, un, st, nrhs, refine, cond, v);
  if (threadIdx.x == 0) b.ucount[0] = 0;
}

template <typename T, int EPI, bool REALC, int NR, int SK, int NAX = 0, int DC = 0, bool HSP = false>
__device__ __forceinline__ void apply_units(const BatchDev& b, int level, int refine, unsigned long long cond,
                                            const StarParams& stp) {
  if constexpr (SK != 0) {
    apply_single_star<T, EPI, REALC, NR, SK, NAX, DC, HSP>(b, level, refine, cond, stp);
    return;
  }
  __shared__ __align__(16) PlanDev sp;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* scoef = reinterpret_cast<cplx<T>*>(smraw);
  const PlanDev* cur = nullptr;
  // chunks in descending order: the batch's last units first (a batch lists its plans in order, and the large units
  // that come last then do not form the tail of the launch); a chunk's sums do not depend on the order
  for (int ci = blockIdx.x; ci < b.nchunks; ci += gridDim.x) {
    const int c = b.nchunks - 1 - ci;
    // a star-1 kernel runs a batch of one unit: its description straight from the kernel parameter
    const int u = SK != 0 ? 0 : unit_of_chunk(b, c);
    const UnitDev& un = SK != 0 ? b.pu : unit_at(b, u);
    RhsSt* st = b.st + (size_t)u * MAXR;
    const int nrhs = un.nrhs;
    // skip units with nothing left to do at this level (same decision for every chunk of the unit)
    bool active = false;
    for (int r = 0; r < nrhs; ++r) {
      if (EPI == EPI_DOT_HW) active |= !ld_int(&st[r].done);
      else if (EPI == EPI_RESIDUAL && refine) active |= !ld_int(&st[r].odone);
      else active = true;
    }
    if (!active) continue;
    // star-1 kernels take the stencil from their kernel parameter instead; FFT units need no stencil
    const bool fft_unit = SK == 0 && un.fft != 0;
    if constexpr (SK == 0) {
      if (!fft_unit && un.plan != cur) {
        cur = un.plan;
        load_plan<T>(cur, sp, scoef);
      }
    }
    const int D = un.D;
    const cplx<T>* src;
    cplx<T>* dst;
    if (level == LEVEL_FP32) {
      src = reinterpret_cast<const cplx<T>*>(un.h32);
      dst = reinterpret_cast<cplx<T>*>(un.w32);
    } else {
      src = reinterpret_cast<const cplx<T>*>(EPI == EPI_DOT_HW ? (const double2*)un.h : (const double2*)un.U);
      dst = reinterpret_cast<cplx<T>*>(un.w);
    }
    const cplx<T>* F = reinterpret_cast<const cplx<T>*>(un.F);
    constexpr int NV = (EPI == EPI_RESIDUAL) ? 2 * NR : NR;   // reduced quantities: (h,w) or (|F-w|^2, |F|^2)
    T vt[NV];                                                   // per-thread partials in the vector precision
    double v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) vt[q] = T(0);
    const int cl = c - un.chunk0;
    // the unit's own run length (so that its reduction order does not depend on the batch)
    if constexpr (SK != 0) {
      apply_chunk<T, EPI, REALC, NR, 2, NV, SK, NAX, DC, HSP>(sp, scoef, stp, un, cl, D, nrhs, refine, fft_unit, src,
                                                             dst, F, vt);
    } else {
      // the common axis counts compiled in (the same arithmetic; fewer per-axis tests)
      if (un.run == 2) {
        if (sp.n == 2)
          apply_chunk<T, EPI, REALC, NR, 2, NV, 0, 0, 0, false, 2>(sp, scoef, stp, un, cl, D, nrhs, refine, fft_unit,
                                                                  src, dst, F, vt);
        else if (sp.n == 4)
          apply_chunk<T, EPI, REALC, NR, 2, NV, 0, 0, 0, false, 4>(sp, scoef, stp, un, cl, D, nrhs, refine, fft_unit,
                                                                  src, dst, F, vt);
        else
          apply_chunk<T, EPI, REALC, NR, 2, NV>(sp, scoef, stp, un, cl, D, nrhs, refine, fft_unit, src, dst, F, vt);
      } else {
        apply_chunk<T, EPI, REALC, NR, 1, NV>(sp, scoef, stp, un, cl, D, nrhs, refine, fft_unit, src, dst, F, vt);
      }
    }
    if (EPI == EPI_NONE) continue;
    block_reduce_mixed<T, NV>(vt, v);
    if (!chunk_arrive<NV>(b, c, u, v)) continue;
    // this block completes unit u: finalize its right-hand sides
    unit_finalize<EPI, NR, NV>(b, un, st, nrhs, refine, cond, v);
    if (threadIdx.x == 0) b.ucount[u] = 0;
  }
}

// Stands in for the kernel-parameter StarParams in kernels that read each plan's own (never dereferenced).
static __device__ StarParams g_no_star;

// Batch apply over every chunk of the batch (plans from the unit table, in shared memory).
template <typename T, int EPI, bool REALC, int NR>
__global__ void __launch_bounds__(BLOCK, sizeof(T) == 8 ? 2 : 3)
    k_apply(const __grid_constant__ BatchDev b, int level, int refine, unsigned long long cond) {
  apply_units<T, EPI, REALC, NR, 0>(b, level, refine, cond, g_no_star);
}

// Batch apply of a single star-1 unit (even last axis): the stencil data as a kernel parameter. The FP32 star
// stencil waits on the L2 latency of its neighbour reads: the run-time-geometry kernels run four blocks per SM (64
// registers); the fixed-geometry ones, whose packed stencil with the chunk loop and epilogue spilled at 64 registers,
// two (up to 128 registers).
template <typename T, int EPI, bool REALC, int NR, int SK, int NAX = 0, int DC = 0, bool HSP = false>
__global__ void __launch_bounds__(BLOCK, sizeof(T) == 8 ? 2 : (NAX != 0 ? 2 : 4))
    k_apply_star(const __grid_constant__ BatchDev b, int level, int refine, unsigned long long cond,
                 const __grid_constant__ StarParams st) {
  apply_units<T, EPI, REALC, NR, SK, NAX, DC, HSP>(b, level, refine, cond, st);
}

// Batch FP32 (h, Q h) apply of a single star-1 unit of a fixed geometry (qp_apply_fixed_batch.cu); false: not one
// of them, nothing launched.
bool launch_batch_star_fixed(const BatchDev& b, int level, int refine, unsigned long long cond, int nblk, size_t smem,
                             const StarParams& st, bool realc, int nr, int kind, cudaStream_t s);

// Plain FP32 star-1 apply of the common fixed geometries (qp_apply_fixed.cu); false: not one of them, nothing
// launched.
bool launch_plain_star_fixed(const StarParams& st, bool realc, int nrhs, int kind, int D, const float2* h, float2* w,
                             cudaStream_t s);

template <typename T, int EPI, int NR, bool REALC>
static void apply_launch_rc(const BatchDev& b, int level, int refine, unsigned long long cond, int nblk, size_t smem,
                            const StarParams* st1, int kind, cudaStream_t s) {
  if constexpr (sizeof(T) == 4 && EPI == EPI_DOT_HW) {
    if (st1 && launch_batch_star_fixed(b, level, refine, cond, nblk, smem, *st1, REALC, NR, kind, s)) return;
  }
  if (!st1) k_apply<T, EPI, REALC, NR><<<nblk, BLOCK, smem, s>>>(b, level, refine, cond);
  else if (st1->hspec) {
    if (kind == QP_COEF_DIAG)
      k_apply_star<T, EPI, REALC, NR, 2, 0, 0, true><<<nblk, BLOCK, smem, s>>>(b, level, refine, cond, *st1);
    else k_apply_star<T, EPI, REALC, NR, 1, 0, 0, true><<<nblk, BLOCK, smem, s>>>(b, level, refine, cond, *st1);
  } else if (kind == QP_COEF_DIAG) {
    k_apply_star<T, EPI, REALC, NR, 2><<<nblk, BLOCK, smem, s>>>(b, level, refine, cond, *st1);
  } else {
    k_apply_star<T, EPI, REALC, NR, 1><<<nblk, BLOCK, smem, s>>>(b, level, refine, cond, *st1);
  }
}

// st1: the StarParams of the batch's single unit when it is a star-1 plan with an even last axis (kind its
// coefficient kind), else null.
template <typename T, int EPI>
void apply_launch_real(bool realc, int maxr, const BatchDev& b, int level, int refine, unsigned long long cond,
                       int nblk, size_t smem, const StarParams* st1, int kind, cudaStream_t s) {
  switch (maxr * 2 + (realc ? 1 : 0)) {
    case 2: apply_launch_rc<T, EPI, 1, false>(b, level, refine, cond, nblk, smem, st1, kind, s); break;
    case 3: apply_launch_rc<T, EPI, 1, true>(b, level, refine, cond, nblk, smem, st1, kind, s); break;
    case 4: apply_launch_rc<T, EPI, 2, false>(b, level, refine, cond, nblk, smem, st1, kind, s); break;
    case 5: apply_launch_rc<T, EPI, 2, true>(b, level, refine, cond, nblk, smem, st1, kind, s); break;
    case 6: apply_launch_rc<T, EPI, 3, false>(b, level, refine, cond, nblk, smem, st1, kind, s); break;
    case 7: apply_launch_rc<T, EPI, 3, true>(b, level, refine, cond, nblk, smem, st1, kind, s); break;
    case 8: apply_launch_rc<T, EPI, 4, false>(b, level, refine, cond, nblk, smem, st1, kind, s); break;
    default: apply_launch_rc<T, EPI, 4, true>(b, level, refine, cond, nblk, smem, st1, kind, s); break;
  }
}


template <typename T, bool REALC, int NR, int RUN>
__global__ void __launch_bounds__(BLOCK, sizeof(T) == 8 ? 2 : 3) k_apply_plain(const PlanDev* plan, int D, int nrhs,
                                                                             const cplx<T>* h, cplx<T>* w) {
  __shared__ __align__(16) PlanDev sp;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* scoef = reinterpret_cast<cplx<T>*>(smraw);
  load_plan<T>(plan, sp, scoef);
  const int e0 = (blockIdx.x * BLOCK + threadIdx.x) * RUN;   // one run per thread: blocks sweep memory in order
  if (e0 >= D) return;
  cplx<T> acc[RUN][NR];
  apply_run<T, REALC, NR, RUN>(sp, scoef, e0, h, D, nrhs, acc);
#pragma unroll
  for (int s = 0; s < RUN; ++s)
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nrhs) w[(size_t)r * D + e0 + s] = acc[s][r];
}

// Plain apply of a star-1 plan with an even last axis: the stencil data as a kernel parameter; one run of two
// modes per thread.
// Blocks per SM of the star-1 plain kernels (their launch bounds) and the grid that keeps exactly those resident.
template <typename T, int NAX> __host__ __device__ constexpr int plain_star_bps() {
  return sizeof(T) == 8 ? 2 : (NAX != 0 ? 2 : 4);
}
template <typename T, int NAX> inline int plain_star_grid(int D) {
  return (int)std::min<long long>(((long long)D / 2 + BLOCK - 1) / BLOCK, 152LL * plain_star_bps<T, NAX>());
}

// The resident blocks sweep the modes together: block b takes the 512-mode segments b, b + grid, b + 2 grid, ...
// (thread t the run of two modes at 2t), so that at any time they work in one window of the vectors and the
// stencil's reads along the outer axes hit L2; no block is started per segment.
template <typename T, bool REALC, int NR, int SK, int NAX = 0, int DC = 0, bool HSP = false>
__global__ void __launch_bounds__(BLOCK, plain_star_bps<T, NAX>())
    k_apply_plain_star(const __grid_constant__ StarParams st, int D, int nrhs, const cplx<T>* h, cplx<T>* w) {
  const int step = (int)gridDim.x * BLOCK * 2;
  for (int e0 = (blockIdx.x * BLOCK + threadIdx.x) * 2; e0 < D; e0 += step) {
    cplx<T> acc[2][NR];
    apply_run_star<T, REALC, NR, true, SK == 2, sizeof(T) == 8 ? 1 : 0, NAX, DC, HSP>(st, e0, h, D, nrhs, acc);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < nrhs) {
        cplx<T>* o = w + (size_t)r * D + e0;
        if (sizeof(T) == 4) {
          *reinterpret_cast<float4*>(o) = make_float4((float)acc[0][r].x, (float)acc[0][r].y, (float)acc[1][r].x,
                                                      (float)acc[1][r].y);
        } else {
          o[0] = acc[0][r];
          o[1] = acc[1][r];
        }
      }
    }
  }
}

template <typename T, bool REALC, int SK>
static void plain_star_nr(int nrhs, const StarParams& st, int D, const cplx<T>* h, cplx<T>* w, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (launch_plain_star_fixed(st, REALC, nrhs, SK == 2 ? QP_COEF_DIAG : QP_COEF_SCALAR, D, h, w, s)) return;
  }
  const int nblk = plain_star_grid<T, 0>(D);
  if (st.hspec) {
    switch (nrhs) {
      case 1: k_apply_plain_star<T, REALC, 1, SK, 0, 0, true><<<nblk, BLOCK, 0, s>>>(st, D, nrhs, h, w); break;
      case 2: k_apply_plain_star<T, REALC, 2, SK, 0, 0, true><<<nblk, BLOCK, 0, s>>>(st, D, nrhs, h, w); break;
      case 3: k_apply_plain_star<T, REALC, 3, SK, 0, 0, true><<<nblk, BLOCK, 0, s>>>(st, D, nrhs, h, w); break;
      default: k_apply_plain_star<T, REALC, 4, SK, 0, 0, true><<<nblk, BLOCK, 0, s>>>(st, D, nrhs, h, w); break;
    }
    return;
  }
  switch (nrhs) {
    case 1: k_apply_plain_star<T, REALC, 1, SK><<<nblk, BLOCK, 0, s>>>(st, D, nrhs, h, w); break;
    case 2: k_apply_plain_star<T, REALC, 2, SK><<<nblk, BLOCK, 0, s>>>(st, D, nrhs, h, w); break;
    case 3: k_apply_plain_star<T, REALC, 3, SK><<<nblk, BLOCK, 0, s>>>(st, D, nrhs, h, w); break;
    default: k_apply_plain_star<T, REALC, 4, SK><<<nblk, BLOCK, 0, s>>>(st, D, nrhs, h, w); break;
  }
}

template <typename T, bool REALC, int RUN>
static void plain_nr(int nrhs, const PlanDev* plan_dev, int D, const cplx<T>* h, cplx<T>* w, size_t smem,
                     cudaStream_t s) {
  const int nblk = (D / RUN + BLOCK - 1) / BLOCK;
  switch (nrhs) {
    case 1: k_apply_plain<T, REALC, 1, RUN><<<nblk, BLOCK, smem, s>>>(plan_dev, D, nrhs, h, w); break;
    case 2: k_apply_plain<T, REALC, 2, RUN><<<nblk, BLOCK, smem, s>>>(plan_dev, D, nrhs, h, w); break;
    case 3: k_apply_plain<T, REALC, 3, RUN><<<nblk, BLOCK, smem, s>>>(plan_dev, D, nrhs, h, w); break;
    default: k_apply_plain<T, REALC, 4, RUN><<<nblk, BLOCK, smem, s>>>(plan_dev, D, nrhs, h, w); break;
  }
}

// The stored FP64 weights of a star-1 plan: one run of two modes per thread, the stencil's own arithmetic. (The
// weights do not depend on the storage's edge handling: one instantiation serves both storages.)
template <bool REALC, bool DIAGK>
__global__ void __launch_bounds__(BLOCK) k_star_weights(const __grid_constant__ StarParams st, int D, void* out) {
  const int e0 = (blockIdx.x * BLOCK + threadIdx.x) * 2;
  if (e0 >= D) return;
  double2 acc[2][1];
  apply_run_star<double, REALC, 1, true, DIAGK, 2>(st, e0, nullptr, D, 0, acc, out);
}

// run: modes per thread (2 when the last axis has even length, else 1). st1: the plan's StarParams when it is
// star-1 and run is 2 (kind its coefficient kind), else null.
template <typename T>
void launch_apply_plain(const PlanDev* plan_dev, bool realc, int mc, int D, int nrhs, const cplx<T>* h, cplx<T>* w,
                        int run, const StarParams* st1, int kind, cudaStream_t s) {
  const size_t smem = (size_t)mc * sizeof(cplx<T>);
  if (st1 && run == 2) {
    const bool dg = kind == QP_COEF_DIAG;
    if (realc) {
      if (dg) plain_star_nr<T, true, 2>(nrhs, *st1, D, h, w, s);
      else plain_star_nr<T, true, 1>(nrhs, *st1, D, h, w, s);
    } else {
      if (dg) plain_star_nr<T, false, 2>(nrhs, *st1, D, h, w, s);
      else plain_star_nr<T, false, 1>(nrhs, *st1, D, h, w, s);
    }
  } else if (run == 2) {
    if (realc) plain_nr<T, true, 2>(nrhs, plan_dev, D, h, w, smem, s);
    else plain_nr<T, false, 2>(nrhs, plan_dev, D, h, w, smem, s);
  } else {
    if (realc) plain_nr<T, true, 1>(nrhs, plan_dev, D, h, w, smem, s);
    else plain_nr<T, false, 1>(nrhs, plan_dev, D, h, w, smem, s);
  }
  count_launch();
}

}  // namespace qp
