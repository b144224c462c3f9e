// Device helpers shared by the stencil and PCG kernels: reductions, chunk arrivals, fast division,
// mode digits and the tap weight lambda(k)^T C_t lambda(k -N m_t).
#pragma once

#include <cfloat>

#include "qp_convert.cuh"
#include "qp_internal.cuh"

namespace qp {

template <typename T> __device__ __forceinline__ cplx<T> mk(T x, T y) {
  cplx<T> r;
  r.x = x;
  r.y = y;
  return r;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Sum (or min) NV values over the block in a fixed tree; thread 0 holds the results afterwards.
template <int NV, bool MIN = false>
__device__ __forceinline__ void block_reduce(double (&v)[NV]) {
  __shared__ double sm[NV][BLOCK / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = MIN ? warp_min(v[q]) : warp_sum(v[q]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sm[q][wid] = v[q];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double x = lane < BLOCK / 32 ? sm[q][lane] : (MIN ? DBL_MAX : 0.0);
      v[q] = MIN ? warp_min(x) : warp_sum(x);
    }
  }
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of per-thread partials held in the vector precision T: the 32 lanes of a warp are summed in T
// (a fixed 5-level tree), the warp sums are converted to FP64 and summed in FP64 (fixed order); thread 0
// gets the results in out. For T = float this keeps FP64 work to one conversion per warp and value while the
// accumulation above the warp level stays FP64.
template <typename T, int NV>
__device__ __forceinline__ void block_reduce_mixed(T (&v)[NV], double (&out)[NV]) {
  __shared__ double sm[NV][BLOCK / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    if (sizeof(T) == 4) v[q] = (T)warp_sum_f((float)v[q]);
    else v[q] = (T)warp_sum((double)v[q]);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sm[q][wid] = (double)v[q];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) out[q] = warp_sum(lane < BLOCK / 32 ? sm[q][lane] : 0.0);
  }
}

__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv& f) {
  return (uint32_t)(((uint64_t)x * f.m) >> f.p);
}

// Storage digits ibar_j of linear index e (last axis fastest) and the signed modes k_j. (A half-spectrum plan's
// last-axis digit is k_{n-1} itself: 0 <= ibar < ceil(N/2), so the signed rule returns it unchanged.)
// NG: the number of axes when the caller compiles it in (0: the plan's, at run time).
template <int NG = 0>
__device__ __forceinline__ void mode_digits(const PlanDev& p, int e, int (&ib)[MAXN], int (&k)[MAXN]) {
  uint32_t x = (uint32_t)e;
#pragma unroll
  for (int j = MAXN - 1; j >= 0; --j) {
    if (j < (NG ? NG : p.n)) {
      const uint32_t q = fdiv(x, p.div[j]);
      ib[j] = (int)(x - q * (uint32_t)p.Nst[j]);
      k[j] = (2 * ib[j] < p.N[j]) ? ib[j] : ib[j] - p.N[j];
      x = q;
    } else {
      ib[j] = 0;
      k[j] = 0;
    }
  }
}

template <typename T> __device__ __forceinline__ T pcoef(const PlanDev& p, int a, int j);
template <> __device__ __forceinline__ double pcoef<double>(const PlanDev& p, int a, int j) { return p.P[a][j]; }
template <> __device__ __forceinline__ float pcoef<float>(const PlanDev& p, int a, int j) { return p.P32[a][j]; }

__device__ __forceinline__ int sym_idx(int a, int b, int d) {
  if (a > b) {
    int t = a;
    a = b;
    b = t;
  }
  return a * d - (a * (a - 1)) / 2 + (b - a);
}

// lambda(k)^T C lambda' for a coefficient with stored components c (kind, d at run time).
template <typename T>
__device__ __forceinline__ cplx<T> weight_general(int kind, int d, const cplx<T>* c, const T (&lk)[MAXD],
                                                  const T (&l2)[MAXD]) {
  cplx<T> r = mk<T>(0, 0);
  if (kind == QP_COEF_SCALAR) {
    T s = 0;
#pragma unroll
    for (int a = 0; a < MAXD; ++a)
      if (a < d) s = fma(lk[a], l2[a], s);
    r.x = c[0].x * s;
    r.y = c[0].y * s;
  } else if (kind == QP_COEF_DIAG) {
#pragma unroll
    for (int a = 0; a < MAXD; ++a) {
      if (a < d) {
        const T s = lk[a] * l2[a];
        r.x = fma(c[a].x, s, r.x);
        r.y = fma(c[a].y, s, r.y);
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < MAXD; ++a) {
#pragma unroll
      for (int b = 0; b < MAXD; ++b) {
        if (a < d && b < d) {
          const cplx<T> cab = c[sym_idx(a, b, d)];
          const T s = lk[a] * l2[b];
          r.x = fma(cab.x, s, r.x);
          r.y = fma(cab.y, s, r.y);
        }
      }
    }
  }
  return r;
}

// Width of one sweep below, in chunks: the FP32 applies of large units (the compiled-in-geometry star-1 kernel runs two
// blocks per SM) sweep 152 x 2 chunks at a time: with 608 the batched FP32 apply at 14^6 read 359 MB from DRAM for
// 181 MB of vectors, with 304 it reads 208 MB. The FP64 applies, bound by FP64 arithmetic, keep 608 (the cfg4 FP64
// residual took 11.7 ms in three applies with 304 against 10.3 ms with 608).
template <typename T> __host__ __device__ constexpr int sweep_chunks() { return sizeof(T) == 4 ? 152 * 2 : 152 * 4; }

// The stencil runs (RUN modes, one per thread and step) of chunk cl of a unit, as e0 = start, start + stride, ...
// below limit. A chunk of fewer than four segments (segment: RUN x BLOCK modes) is its contiguous range of modes.
// Larger chunks go in waves of SWEEP_CHUNKS consecutive chunks (about the blocks resident together); wave w takes a
// contiguous share of the unit's segments, in proportion to its chunks, and its chunk p the segments
// s0 + p, s0 + p + rw, s0 + p + 2 rw, ... of that share (rw: the wave's chunks). The resident blocks then sweep
// one contiguous window together and the stencil's reads along the outer axes hit L2 (contiguous chunks of 13,824
// modes at 16^6 spread the resident blocks over the whole vector: 2.2x the DRAM reads; one interleave over the
// whole unit left each of the two waves at 14^6 sweeping every other segment of it: 277 MB read per batched FP32
// apply, against 215 MB in waves and 208 MB for the plain apply). A unit of at most SWEEP_CHUNKS chunks is one
// wave: segments cl, cl + nchunk, cl + 2 nchunk, ...
template <typename T>
__device__ __forceinline__ void chunk_runs(const UnitDev& un, int cl, int run, int& start, int& stride, int& limit) {
  constexpr int SWEEP_CHUNKS = sweep_chunks<T>();
  const int seg = run * BLOCK;
  if (un.chunk >= 4 * seg) {
    const int nseg = (un.D + seg - 1) / seg;
    const int w = cl / SWEEP_CHUNKS, p = cl - w * SWEEP_CHUNKS;
    const int c1 = min((w + 1) * SWEEP_CHUNKS, un.nchunk);
    const int s0 = (int)((int64_t)nseg * (w * SWEEP_CHUNKS) / un.nchunk);
    const int s1 = (int)((int64_t)nseg * c1 / un.nchunk);
    start = (s0 + p) * seg + run * (int)threadIdx.x;
    stride = (c1 - w * SWEEP_CHUNKS) * seg;
    limit = min(s1 * seg, un.D);
  } else {
    start = cl * un.chunk + run * (int)threadIdx.x;
    stride = seg;
    limit = min(cl * un.chunk + un.chunk, un.D);
  }
}

// The unit a chunk belongs to, and its description (kernel parameter for a single unit, else the table).
__device__ __forceinline__ int unit_of_chunk(const BatchDev& b, int c) { return b.single ? 0 : b.chunk_unit[c]; }
__device__ __forceinline__ const UnitDev& unit_at(const BatchDev& b, int u) { return b.single ? b.pu : b.units[u]; }

// Record this block's chunk partials (thread 0 holds them in v), count the chunk's arrival for its unit and
// return true in the block that completes the unit (all its chunks are in).
template <int NV>
__device__ __forceinline__ bool chunk_arrive(const BatchDev& b, int c, int u, const double (&v)[NV]) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) b.partials[(size_t)q * b.nchunks + c] = v[q];
    __threadfence();
    s_last = (atomicAdd(&b.ucount[u], 1u) == (unsigned)unit_at(b, u).nchunk - 1u);
  }
  __syncthreads();
  const bool last = s_last != 0;
  if (last) __threadfence();
  return last;
}

// In the completing block: sums every slot (slot0 .. slot0 + NV - 1) over the unit's chunks in a fixed order;
// thread 0 gets the sums.
template <int NV>
__device__ __forceinline__ void unit_sums(const BatchDev& b, const UnitDev& un, double (&v)[NV], int slot0 = 0) {
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = 0.0;
  for (int i = threadIdx.x; i < un.nchunk; i += BLOCK) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __ldcg(b.partials + (size_t)(slot0 + q) * b.nchunks + un.chunk0 + i);
  }
  block_reduce<NV>(v);
}

// Counts "n" newly finished right-hand sides into ndone[which]; when the count reaches every right-hand
// side, ends the WHILE loop driven by "cond" (the one call that completes the count sets it).
__device__ __forceinline__ void count_done(const BatchDev& b, int which, int n, unsigned long long cond) {
  if (n == 0) return;
  const int before = atomicAdd(&b.ndone[which], n);
  if (cond != 0ull && before + n >= b.nslots) cudaGraphSetConditional(cond, 0u);
}

__device__ __forceinline__ int ld_int(const int* p) { return *((volatile const int*)p); }

// Weight of storage index e in the inner products of a half-spectrum unit (1 on the self-conjugate plane
// k_{n-1} = 0, 2 elsewhere: the entry stands for the mode and its mirror); 1 for full-spectrum units.
__device__ __forceinline__ int mode_weight(const UnitDev& un, int e) {
  if (!un.hspec) return 1;
  return (e - (int)fdiv((uint32_t)e, un.hdiv) * un.Hl) == 0 ? 1 : 2;
}

}  // namespace qp
