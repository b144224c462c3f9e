// The per-mode stencil of the taps backend, shared by the batch apply kernels (qp_taps.cu) and the persistent
// solve (qp_persistent.cu): the compressed mat-vec of Sec. 4.2,
//   (Q h)(k) = sum_t lambda(k)^T C_t lambda(k -N m_t) h(k -N m_t),   lambda(k) = P k,
// (eq. n-discrete_equation; App. D for a matrix coefficient). Star taps (one nonzero axis) are grouped per
// axis so that each costs one wrap test, one index update and, for a scalar coefficient, one fused
// multiply-add for the weight: lambda(k).lambda(k') = |lambda(k)|^2 + dk (lambda(k).P_j).
#pragma once
#include "qp_device.cuh"

namespace qp {
// Operand load: RO (the operand is not written while the kernel runs) takes the read-only data path; a kernel
// that writes the operand itself between grid barriers reads it with plain coherent loads.
template <bool RO, typename V> __device__ __forceinline__ V ldh(const V* p) {
  if (RO) return __ldg(p);
  return *p;
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

// acc[r] = (Q h_r)(e) for r < nrhs: the whole tap sum at one mode.
template <typename T, bool REALC, int NR, bool RO = true>
__device__ __forceinline__ void apply_point(const PlanDev& p, const cplx<T>* __restrict__ sc, int e,
                                            const cplx<T>* h, int D, int nrhs, cplx<T> (&acc)[NR]) {
  int ib[MAXN], k[MAXN];
  mode_digits(p, e, ib, k);
  const int d = p.d, kind = p.kind, nc = p.ncomp;
  T lk[MAXD];
#pragma unroll
  for (int a = 0; a < MAXD; ++a) {
    lk[a] = T(0);
#pragma unroll
    for (int j = 0; j < MAXN; ++j)
      if (a < d && j < p.n) lk[a] = fma(pcoef<T>(p, a, j), (T)k[j], lk[a]);
  }
  const bool scalar = (kind == QP_COEF_SCALAR);
  T lam2 = T(0), lp[MAXN];
#pragma unroll
  for (int a = 0; a < MAXD; ++a)
    if (a < d) lam2 = fma(lk[a], lk[a], lam2);
#pragma unroll
  for (int j = 0; j < MAXN; ++j) {
    lp[j] = T(0);
    if (scalar && j < p.n) {
#pragma unroll
      for (int a = 0; a < MAXD; ++a)
        if (a < d) lp[j] = fma(lk[a], pcoef<T>(p, a, j), lp[j]);
    }
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r] = mk<T>(0, 0);

  // mean tap (sorted index 0): k' = k
  {
    cplx<T> c;
    if (scalar) {
      c.x = sc[0].x * lam2;
      c.y = REALC ? T(0) : sc[0].y * lam2;
    } else {
      c = weight_general<T>(kind, d, sc, lk, lk);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nrhs) mac<T, REALC>(acc[r], c, ldh<RO>(h + (size_t)r * D + e));
  }
  // star taps, grouped by axis
#pragma unroll
  for (int j = 0; j < MAXN; ++j) {
    if (j < p.n) {
      const int Nj = p.N[j], sj = p.stride[j];
      const int t1 = p.star_begin[j + 1];
      for (int t = p.star_begin[j]; t < t1; ++t) {
        int ib2 = ib[j] - (int)p.m[t][j];
        ib2 += (ib2 < 0) ? Nj : 0;
        ib2 -= (ib2 >= Nj) ? Nj : 0;
        const int e2 = e + (ib2 - ib[j]) * sj;
        const int k2 = (2 * ib2 < Nj) ? ib2 : ib2 - Nj;
        const T dk = (T)(k2 - k[j]);
        cplx<T> c;
        if (scalar) {
          const T s = fma(dk, lp[j], lam2);
          c.x = sc[t].x * s;
          c.y = REALC ? T(0) : sc[t].y * s;
        } else {
          T l2[MAXD];
#pragma unroll
          for (int a = 0; a < MAXD; ++a) l2[a] = (a < d) ? fma(dk, pcoef<T>(p, a, j), lk[a]) : T(0);
          c = weight_general<T>(kind, d, sc + t * nc, lk, l2);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (r < nrhs) mac<T, REALC>(acc[r], c, ldh<RO>(h + (size_t)r * D + e2));
      }
    }
  }
  // taps with several nonzero axes
  for (int t = p.star_begin[p.n]; t < p.ntaps; ++t) {
    int e2 = e;
    T l2[MAXD];
#pragma unroll
    for (int a = 0; a < MAXD; ++a) l2[a] = lk[a];
#pragma unroll
    for (int j = 0; j < MAXN; ++j) {
      const int mj = (j < p.n) ? (int)p.m[t][j] : 0;
      if (mj != 0) {
        const int Nj = p.N[j];
        int ib2 = ib[j] - mj;
        ib2 += (ib2 < 0) ? Nj : 0;
        ib2 -= (ib2 >= Nj) ? Nj : 0;
        e2 += (ib2 - ib[j]) * p.stride[j];
        const int k2 = (2 * ib2 < Nj) ? ib2 : ib2 - Nj;
        const T dk = (T)(k2 - k[j]);
#pragma unroll
        for (int a = 0; a < MAXD; ++a)
          if (a < d) l2[a] = fma(dk, pcoef<T>(p, a, j), l2[a]);
      }
    }
    const cplx<T> c = weight_general<T>(kind, d, sc + t * nc, lk, l2);
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nrhs) mac<T, REALC>(acc[r], c, ldh<RO>(h + (size_t)r * D + e2));
  }
}

}  // namespace qp
