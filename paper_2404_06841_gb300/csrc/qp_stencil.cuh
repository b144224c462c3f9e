// The stencil of the taps backend, shared by the batch apply kernels (qp_taps.cu) and the persistent solve
// (qp_persistent.cu): the compressed mat-vec of Sec. 4.2,
//   (Q h)(k) = sum_t lambda(k)^T C_t lambda(k -N m_t) h(k -N m_t),   lambda(k) = P k,
// (eq. n-discrete_equation; App. D for a matrix coefficient), evaluated on runs of consecutive modes along the
// last axis. Star taps (one nonzero axis) are grouped per axis; for a scalar coefficient a star tap's weight
// costs one fused multiply-add per mode: lambda(k).lambda(k') = |lambda(k)|^2 + dk (lambda(k).P_j).
#pragma once
#include "qp_device.cuh"

namespace qp {
// Operand load: RO (the operand is not written while the kernel runs) takes the read-only data path; a kernel
// that writes the operand itself between grid barriers reads it with plain coherent loads.
template <bool RO, typename V> __device__ __forceinline__ V ldh(const V* p) {
  if (RO) return __ldg(p);
  return *p;
}

// RUN consecutive complex values from p (p aligned to RUN elements): one 16-byte load for two FP32 values.
template <bool RO, typename T, int RUN>
__device__ __forceinline__ void ld_run(const cplx<T>* p, cplx<T> (&v)[RUN]) {
  if (sizeof(T) == 4 && RUN == 2) {
    const float4 q = RO ? __ldg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
    v[0] = mk<T>((T)q.x, (T)q.y);
    v[RUN - 1] = mk<T>((T)q.z, (T)q.w);
  } else {
#pragma unroll
    for (int s = 0; s < RUN; ++s) v[s] = ldh<RO>(p + s);
  }
}


template <typename T>
__device__ __forceinline__ void load_plan(const PlanDev* src, PlanDev& dst, cplx<T>* coef) {
  __syncthreads();
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(PlanDev) / sizeof(int4)); i += BLOCK) d[i] = s[i];
  __syncthreads();
  const int nc = dst.ntaps * dst.ncomp;
  if (sizeof(T) == 8) {
    const double2* c = dst.coef64;
    for (int i = threadIdx.x; i < nc; i += BLOCK) reinterpret_cast<double2*>(coef)[i] = c[i];
  } else {
    const float2* c = dst.coef32;
    for (int i = threadIdx.x; i < nc; i += BLOCK) reinterpret_cast<float2*>(coef)[i] = c[i];
  }
  __syncthreads();
}

template <typename T, bool REALC>
__device__ __forceinline__ void mac(cplx<T>& acc, const cplx<T>& c, const cplx<T>& hv) {
  if (REALC) {
    acc.x = fma(c.x, hv.x, acc.x);
    acc.y = fma(c.x, hv.y, acc.y);
  } else {
    acc.x = fma(c.x, hv.x, fma(-c.y, hv.y, acc.x));
    acc.y = fma(c.x, hv.y, fma(c.y, hv.x, acc.y));
  }
}

// acc[s][r] = (Q h_r)(e0 + s), s < RUN: the whole tap sum at RUN consecutive modes of one row of the last
// axis (e0 a multiple of RUN, RUN dividing N_{n-1}). Everything that depends only on the row is done once per
// run: the digits of e0, lambda over the other axes, and for every tap along another axis its wrapped offset and
// its mode step dk; that tap then reads RUN consecutive entries of h. The weights are formed per mode:
//   scalar:  c_t (|lambda|^2 + dk lambda.P_j),   otherwise  lambda^T C_t (lambda + dk P_j)   (star tap on axis j).
template <typename T, bool REALC, int NR, int RUN, bool RO = true>
__device__ __forceinline__ void apply_run(const PlanDev& p, const cplx<T>* __restrict__ sc, int e0,
                                          const cplx<T>* h, int D, int nrhs, cplx<T> (&acc)[RUN][NR]) {
  int ib[MAXN], k[MAXN];
  mode_digits(p, e0, ib, k);
  const int d = p.d, kind = p.kind, nc = p.ncomp, n = p.n;
  const int jl = n - 1, Nl = p.N[jl];
  const int ibl = e0 - (int)fdiv((uint32_t)e0, p.div[jl]) * Nl;   // digit of the last axis (kept in registers)
  const bool scalar = (kind == QP_COEF_SCALAR);
  const cplx<T>* hr[NR];   // each right-hand side's vector
#pragma unroll
  for (int r = 0; r < NR; ++r) hr[r] = h + (size_t)r * D;
  // lambda per mode of the run
  T lk[RUN][MAXD];
  int kl[RUN];
  {
    T lr[MAXD];
#pragma unroll
    for (int a = 0; a < MAXD; ++a) {
      lr[a] = T(0);
#pragma unroll
      for (int j = 0; j < MAXN - 1; ++j)
        if (a < d && j < jl) lr[a] = fma(pcoef<T>(p, a, j), (T)k[j], lr[a]);
    }
#pragma unroll
    for (int s = 0; s < RUN; ++s) {
      const int ibs = ibl + s;
      kl[s] = (2 * ibs < Nl) ? ibs : ibs - Nl;
#pragma unroll
      for (int a = 0; a < MAXD; ++a) lk[s][a] = (a < d) ? fma(pcoef<T>(p, a, jl), (T)kl[s], lr[a]) : T(0);
    }
  }
  // scalar coefficient: |lambda|^2 per mode (lambda.P_j is formed per axis below)
  T lam2[RUN];
#pragma unroll
  for (int s = 0; s < RUN; ++s) {
    lam2[s] = T(0);
#pragma unroll
    for (int a = 0; a < MAXD; ++a)
      if (a < d) lam2[s] = fma(lk[s][a], lk[s][a], lam2[s]);
  }
#pragma unroll
  for (int s = 0; s < RUN; ++s)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[s][r] = mk<T>(0, 0);

  // mean tap (sorted index 0): k' = k
  {
    cplx<T> c[RUN];
#pragma unroll
    for (int s = 0; s < RUN; ++s) {
      if (scalar) {
        c[s].x = sc[0].x * lam2[s];
        c[s].y = REALC ? T(0) : sc[0].y * lam2[s];
      } else {
        c[s] = weight_general<T>(kind, d, sc, lk[s], lk[s]);
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < nrhs) {
        cplx<T> hv[RUN];
        ld_run<RO, T, RUN>(hr[r] + e0, hv);
#pragma unroll
        for (int s = 0; s < RUN; ++s) mac<T, REALC>(acc[s][r], c[s], hv[s]);
      }
    }
  }
  // star taps of the axes before the last: one offset per run, RUN consecutive reads per tap
#pragma unroll
  for (int j = 0; j < MAXN - 1; ++j) {
    if (j < jl) {
      const int Nj = p.N[j], sj = p.stride[j];
      T pj[MAXD], lp[RUN];
#pragma unroll
      for (int a = 0; a < MAXD; ++a) pj[a] = pcoef<T>(p, a, j);
#pragma unroll
      for (int s = 0; s < RUN; ++s) {
        lp[s] = T(0);
#pragma unroll
        for (int a = 0; a < MAXD; ++a)
          if (scalar && a < d) lp[s] = fma(lk[s][a], pj[a], lp[s]);
      }
      const int t1 = p.star_begin[j + 1];
      for (int t = p.star_begin[j]; t < t1; ++t) {
        int ib2 = ib[j] - (int)p.m[t][j];
        ib2 += (ib2 < 0) ? Nj : 0;
        ib2 -= (ib2 >= Nj) ? Nj : 0;
        const int e2 = e0 + (ib2 - ib[j]) * sj;
        const int k2 = (2 * ib2 < Nj) ? ib2 : ib2 - Nj;
        const T dk = (T)(k2 - k[j]);
        const cplx<T>* ct = sc + t * nc;
        cplx<T> c[RUN];
#pragma unroll
        for (int s = 0; s < RUN; ++s) {
          if (scalar) {
            const T w = fma(dk, lp[s], lam2[s]);
            c[s].x = ct[0].x * w;
            c[s].y = REALC ? T(0) : ct[0].y * w;
          } else {
            T l2[MAXD];
#pragma unroll
            for (int a = 0; a < MAXD; ++a) l2[a] = (a < d) ? fma(dk, pj[a], lk[s][a]) : T(0);
            c[s] = weight_general<T>(kind, d, ct, lk[s], l2);
          }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r < nrhs) {
            cplx<T> hv[RUN];
            ld_run<RO, T, RUN>(hr[r] + e2, hv);
#pragma unroll
            for (int s = 0; s < RUN; ++s) mac<T, REALC>(acc[s][r], c[s], hv[s]);
          }
        }
      }
    }
  }
  // star taps of the last axis: per mode (the neighbour may wrap around the row)
  {
    const int row0 = e0 - ibl;
    T pl[MAXD], lp[RUN];
#pragma unroll
    for (int a = 0; a < MAXD; ++a) pl[a] = pcoef<T>(p, a, jl);
#pragma unroll
    for (int s = 0; s < RUN; ++s) {
      lp[s] = T(0);
#pragma unroll
      for (int a = 0; a < MAXD; ++a)
        if (scalar && a < d) lp[s] = fma(lk[s][a], pl[a], lp[s]);
    }
    const int t1 = p.star_begin[jl + 1];
    for (int t = p.star_begin[jl]; t < t1; ++t) {
      const int mt = (int)p.m[t][jl];
      const cplx<T>* ct = sc + t * nc;
#pragma unroll
      for (int s = 0; s < RUN; ++s) {
        int ib2 = ibl + s - mt;
        ib2 += (ib2 < 0) ? Nl : 0;
        ib2 -= (ib2 >= Nl) ? Nl : 0;
        const int k2 = (2 * ib2 < Nl) ? ib2 : ib2 - Nl;
        const T dk = (T)(k2 - kl[s]);
        cplx<T> c;
        if (scalar) {
          const T w = fma(dk, lp[s], lam2[s]);
          c.x = ct[0].x * w;
          c.y = REALC ? T(0) : ct[0].y * w;
        } else {
          T l2[MAXD];
#pragma unroll
          for (int a = 0; a < MAXD; ++a) l2[a] = (a < d) ? fma(dk, pl[a], lk[s][a]) : T(0);
          c = weight_general<T>(kind, d, ct, lk[s], l2);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (r < nrhs) mac<T, REALC>(acc[s][r], c, ldh<RO>(hr[r] + row0 + ib2));
      }
    }
  }
  // taps with several nonzero axes: the other axes once per run, the last axis per mode
  for (int t = p.star_begin[n]; t < p.ntaps; ++t) {
    int eo = e0 - ibl;
    T lo[MAXD];
#pragma unroll
    for (int a = 0; a < MAXD; ++a) lo[a] = T(0);
#pragma unroll
    for (int j = 0; j < MAXN - 1; ++j) {
      const int mj = (j < jl) ? (int)p.m[t][j] : 0;
      if (mj != 0) {
        const int Nj = p.N[j];
        int ib2 = ib[j] - mj;
        ib2 += (ib2 < 0) ? Nj : 0;
        ib2 -= (ib2 >= Nj) ? Nj : 0;
        eo += (ib2 - ib[j]) * p.stride[j];
        const int k2 = (2 * ib2 < Nj) ? ib2 : ib2 - Nj;
        const T dk = (T)(k2 - k[j]);
#pragma unroll
        for (int a = 0; a < MAXD; ++a)
          if (a < d) lo[a] = fma(dk, pcoef<T>(p, a, j), lo[a]);
      }
    }
    const int mt = (int)p.m[t][jl];
    const cplx<T>* ct = sc + t * nc;
#pragma unroll
    for (int s = 0; s < RUN; ++s) {
      int ib2 = ibl + s - mt;
      ib2 += (ib2 < 0) ? Nl : 0;
      ib2 -= (ib2 >= Nl) ? Nl : 0;
      const int k2 = (2 * ib2 < Nl) ? ib2 : ib2 - Nl;
      const T dk = (T)(k2 - kl[s]);
      T l2[MAXD];
#pragma unroll
      for (int a = 0; a < MAXD; ++a) l2[a] = (a < d) ? fma(dk, pcoef<T>(p, a, jl), lk[s][a] + lo[a]) : T(0);
      const cplx<T> c = weight_general<T>(kind, d, ct, lk[s], l2);
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r < nrhs) mac<T, REALC>(acc[s][r], c, ldh<RO>(hr[r] + eo + ib2));
    }
  }
}

}  // namespace qp
