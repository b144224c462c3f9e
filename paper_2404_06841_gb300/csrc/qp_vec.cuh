// Per-chunk element loops of the PCG vector steps of Algorithm 2, shared by the kernel-per-step form (qp_pcg.cu)
// and the persistent form (qp_persistent.cuh), so that both take the same arithmetic in the same order.
//
// Thread t of a block walks a chunk [base, end) of a unit's modes: FP32 vectors in pairs of modes (e, e + 1) with
// e = base + 2t, base + 2t + 2 BLOCK, ... (one 16-byte access per vector and right-hand side), FP64 vectors one mode
// at a time (e = base + t, base + t + BLOCK, ...). Chunk bases are even; an odd chunk end leaves its last mode
// alone in the pair that starts there. A pair is one 16-byte access only when D is even (vector k starts at
// element k D, which is then 16-byte aligned); for odd D its two modes are accessed one by one. Every operand
// of a step is loaded before the step stores anything, so that the loads of all right-hand sides are in
// flight together.
#pragma once
#include "qp_device.cuh"

namespace qp {

template <typename T> __host__ __device__ constexpr int vec_width() { return sizeof(T) == 4 ? 2 : 1; }

// n (1 or W) consecutive complex values at p; the rest of v is zero. v16: p is 16-byte aligned.
template <typename T, int W>
__device__ __forceinline__ void vld(const cplx<T>* p, int n, bool v16, cplx<T> (&v)[W]) {
  if constexpr (W == 2) {
    if (n == 2 && v16) {
      const float4 q = *reinterpret_cast<const float4*>(p);
      v[0] = mk<T>((T)q.x, (T)q.y);
      v[1] = mk<T>((T)q.z, (T)q.w);
    } else {
      v[0] = p[0];
      v[1] = n == 2 ? p[1] : mk<T>(0, 0);
    }
  } else {
    v[0] = p[0];
  }
}

template <typename T, int W>
__device__ __forceinline__ void vst(cplx<T>* p, int n, bool v16, const cplx<T> (&v)[W]) {
  if constexpr (W == 2) {
    if (n == 2 && v16) {
      *reinterpret_cast<float4*>(p) = make_float4((float)v[0].x, (float)v[0].y, (float)v[1].x, (float)v[1].y);
    } else {
      p[0] = v[0];
      if (n == 2) p[1] = v[1];
    }
  } else {
    p[0] = v[0];
  }
}

template <typename T, int W>
__device__ __forceinline__ void vld_real(const T* p, int n, T (&v)[W]) {
  if constexpr (W == 2) {
    if (n == 2) {
      const float2 q = *reinterpret_cast<const float2*>(p);
      v[0] = (T)q.x;
      v[1] = (T)q.y;
    } else {
      v[0] = p[0];
      v[1] = T(0);
    }
  } else {
    v[0] = p[0];
  }
}

// r = F - w (warm: w = Q U) or r = F, with r(0) = 0 and F = 0 for the right-hand sides in zero_rhs; h = M r;
// U = 0 where zero_u. Per-thread partials vt: ||F||^2, (r, M r), ||r||^2 per right-hand side. HW (half-spectrum
// units): each mode weighted by mode_weight, an entry off the plane k_{n-1} = 0 counting for its mirror too; the
// full-spectrum form has no weights (in FP64 a multiply per term is not free).
template <typename T, int NR, bool HW = false>
__device__ __forceinline__ void vec_init(const UnitDev& un, int base, int end, int D, int nrhs, bool warm, bool zero_u,
                                         const int* zero_rhs, const cplx<T>* __restrict__ F, cplx<T>* __restrict__ U,
                                         cplx<T>* __restrict__ r, cplx<T>* __restrict__ h,
                                         const cplx<T>* __restrict__ w, const T* __restrict__ M, T (&vt)[3 * NR]) {
  constexpr int W = vec_width<T>();
  const bool v16 = (D & 1) == 0;
  for (int e = base + W * (int)threadIdx.x; e < end; e += W * BLOCK) {
    const int n = min(W, end - e);
    T m[W];
    vld_real<T, W>(M + e, n, m);
    T wts[W];   // inner-product weights (half-spectrum units: 1 or 2; else 1)
#pragma unroll
    for (int s = 0; s < W; ++s) wts[s] = HW ? (T)mode_weight(un, e + s) : T(1);
    cplx<T> fv[NR][W], wv[NR][W];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      if (k < nrhs) {
        vld<T, W>(F + (size_t)k * D + e, n, v16, fv[k]);
        if (warm) vld<T, W>(w + (size_t)k * D + e, n, v16, wv[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      if (k < nrhs) {
        const size_t o = (size_t)k * D + e;
        cplx<T> rv[W], hv[W];
#pragma unroll
        for (int s = 0; s < W; ++s) {
          cplx<T> f = fv[k][s];
          if (e + s == 0 || zero_rhs[k]) f = mk<T>(0, 0);
          cplx<T> x = f;
          if (warm && e + s != 0) x = mk<T>(f.x - wv[k][s].x, f.y - wv[k][s].y);
          rv[s] = x;
          hv[s] = mk<T>(m[s] * x.x, m[s] * x.y);
          const T we = wts[s];
          const T rr = we * fma(x.x, x.x, x.y * x.y);
          vt[3 * k] = fma(we * f.x, f.x, fma(we * f.y, f.y, vt[3 * k]));
          vt[3 * k + 1] = fma(m[s], rr, vt[3 * k + 1]);
          vt[3 * k + 2] += rr;
        }
        vst<T, W>(r + o, n, v16, rv);
        vst<T, W>(h + o, n, v16, hv);
        if (zero_u) {
          cplx<T> z[W];
#pragma unroll
          for (int s = 0; s < W; ++s) z[s] = mk<T>(0, 0);
          vst<T, W>(U + o, n, v16, z);
        }
      }
    }
  }
}

// r -= alpha w for the right-hand sides not done; partials vt: (r, M r), ||r||^2 per right-hand side (HW: as in
// vec_init).
template <typename T, int NR, bool HW = false>
__device__ __forceinline__ void vec_update(const UnitDev& un, int base, int end, int D, int nrhs, const int* done,
                                           const T* alpha,
                                           cplx<T>* __restrict__ r, const cplx<T>* __restrict__ w,
                                           const T* __restrict__ M, T (&vt)[2 * NR]) {
  constexpr int W = vec_width<T>();
  const bool v16 = (D & 1) == 0;
  for (int e = base + W * (int)threadIdx.x; e < end; e += W * BLOCK) {
    const int n = min(W, end - e);
    T m[W];
    vld_real<T, W>(M + e, n, m);
    T wts[W];
#pragma unroll
    for (int s = 0; s < W; ++s) wts[s] = HW ? (T)mode_weight(un, e + s) : T(1);
    cplx<T> rv[NR][W], wv[NR][W];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      if (k < nrhs && !done[k]) {
        vld<T, W>(r + (size_t)k * D + e, n, v16, rv[k]);
        vld<T, W>(w + (size_t)k * D + e, n, v16, wv[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      if (k < nrhs && !done[k]) {
        const T al = alpha[k];
#pragma unroll
        for (int s = 0; s < W; ++s) {
          cplx<T>& x = rv[k][s];
          x.x = fma(-al, wv[k][s].x, x.x);
          x.y = fma(-al, wv[k][s].y, x.y);
          const T rr = wts[s] * fma(x.x, x.x, x.y * x.y);
          vt[2 * k] = fma(m[s], rr, vt[2 * k]);
          vt[2 * k + 1] += rr;
        }
        vst<T, W>(r + (size_t)k * D + e, n, v16, rv[k]);
      }
    }
  }
}

// U += alpha h for the right-hand sides in upd (active in this iteration), then h = M r + beta h for those in hup
// (still running), both from the same read of h.
template <typename T, int NR>
__device__ __forceinline__ void vec_hupdate(int base, int end, int D, int nrhs, const int* upd, const T* alpha,
                                            const int* hup, const T* beta, const cplx<T>* __restrict__ r,
                                            cplx<T>* __restrict__ h, cplx<T>* __restrict__ U,
                                            const T* __restrict__ M) {
  constexpr int W = vec_width<T>();
  const bool v16 = (D & 1) == 0;
  for (int e = base + W * (int)threadIdx.x; e < end; e += W * BLOCK) {
    const int n = min(W, end - e);
    T m[W];
    vld_real<T, W>(M + e, n, m);
    cplx<T> hv[NR][W], uv[NR][W], rv[NR][W];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      if (k < nrhs && upd[k]) {
        const size_t o = (size_t)k * D + e;
        vld<T, W>(h + o, n, v16, hv[k]);
        vld<T, W>(U + o, n, v16, uv[k]);
        if (hup[k]) vld<T, W>(r + o, n, v16, rv[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      if (k < nrhs && upd[k]) {
        const size_t o = (size_t)k * D + e;
#pragma unroll
        for (int s = 0; s < W; ++s) {
          uv[k][s].x = fma(alpha[k], hv[k][s].x, uv[k][s].x);
          uv[k][s].y = fma(alpha[k], hv[k][s].y, uv[k][s].y);
        }
        vst<T, W>(U + o, n, v16, uv[k]);
        if (hup[k]) {
#pragma unroll
          for (int s = 0; s < W; ++s) {
            hv[k][s].x = fma(beta[k], hv[k][s].x, m[s] * rv[k][s].x);
            hv[k][s].y = fma(beta[k], hv[k][s].y, m[s] * rv[k][s].y);
          }
          vst<T, W>(h + o, n, v16, hv[k]);
        }
      }
    }
  }
}

}  // namespace qp
