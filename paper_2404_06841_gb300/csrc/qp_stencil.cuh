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


// Copies the plan description and its coefficient table (precision T) to shared memory.
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

// ---- star-1 stencils (PlanDev.star1: scalar or diagonal coefficient, taps at m = 0 and m = +-e_j only)
//
// The neighbour of the tap m = +-e_j is k -+ e_j, with lambda(k -+ e_j) = lambda(k) + dk P_j; the weight
// lambda(k)^T C_t lambda(k -+ e_j) is then
//   scalar:    c_t (q + dk r_j),                 q = |lambda|^2,   r_j = lambda . P_j
//   diagonal:  sum_a c_t,a (q_a + dk r_a,j),     q_a = lambda_a^2, r_a,j = lambda_a P_a,j
// with q formed once per mode and r once per axis. dk is -+1 except across the frequency wrap between
// k_j = ceil(N_j/2) - 1 and ceil(N_j/2) - N_j, and the neighbour's storage index steps by -+stride_j except
// across the storage wrap at index 0 / N_j - 1: each exception is one compare and one select. Runs of two
// modes along the last axis (even length): its own taps read the run's two values and one neighbour each side.
// Everything but the vectors comes from a StarParams (kernel parameter or shared memory) at fixed offsets.

template <typename T> __device__ __forceinline__ T sp_P(const StarParams& s, int a, int j);
template <> __device__ __forceinline__ double sp_P<double>(const StarParams& s, int a, int j) { return s.P64[a][j]; }
template <> __device__ __forceinline__ float sp_P<float>(const StarParams& s, int a, int j) { return s.P32[a][j]; }
// component a of the tap m = +e_j (sg = 0) or m = -e_j (sg = 1); sp_c0: of the mean tap
template <typename T> __device__ __forceinline__ cplx<T> sp_c(const StarParams& s, int j, int sg, int a);
template <> __device__ __forceinline__ double2 sp_c<double>(const StarParams& s, int j, int sg, int a) {
  return s.c64[j][sg][a];
}
template <> __device__ __forceinline__ float2 sp_c<float>(const StarParams& s, int j, int sg, int a) {
  return s.c32[j][sg][a];
}
template <typename T> __device__ __forceinline__ cplx<T> sp_c0(const StarParams& s, int a);
template <> __device__ __forceinline__ double2 sp_c0<double>(const StarParams& s, int a) { return s.c064[a]; }
template <> __device__ __forceinline__ float2 sp_c0<float>(const StarParams& s, int a) { return s.c032[a]; }

// Weight slots of a star-1 plan's stored weights (StarParams.w64): 0 the mean tap, 1 + 2j / 2 + 2j the taps
// m = +e_j / -e_j; [slot][D] complex (real for real tap values).
__host__ __device__ constexpr int star_slots() { return 1 + 2 * MAXN; }

// (a kernel for complex taps may serve a plan with real ones, whose table then has the real layout)
template <bool REALC>
__device__ __forceinline__ void wload(const StarParams& sp, int slot, int e0, int D, double2 (&c)[2]) {
  if (REALC || sp.wreal) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(static_cast<const double*>(sp.w64) + (size_t)slot * D + e0));
    c[0] = make_double2(v.x, 0.0);
    c[1] = make_double2(v.y, 0.0);
  } else {
    const double2* w = static_cast<const double2*>(sp.w64) + (size_t)slot * D + e0;
    c[0] = __ldg(w);
    c[1] = __ldg(w + 1);
  }
}
template <bool REALC>
__device__ __forceinline__ void wstore(void* out, int slot, int e0, int D, const double2 (&c)[2]) {
  if (REALC) {
    *reinterpret_cast<double2*>(static_cast<double*>(out) + (size_t)slot * D + e0) = make_double2(c[0].x, c[1].x);
  } else {
    double2* w = static_cast<double2*>(out) + (size_t)slot * D + e0;
    w[0] = c[0];
    w[1] = c[1];
  }
}

// ---- FP32 star-1 run in packed form: the taps as Hermitian pairs, two FP32 lanes per instruction
//
// For a real coefficient the tap -e_j holds the conjugate of the tap +e_j (c_j,a), so the two weights of axis j at
// mode k come from the same two complex sums
//   A = sum_a c_j,a q_a(k),   B = sum_a (c_j,a P_aj) lambda_a(k)         (q_a = lambda_a^2; scalar: c_j,a = c_j)
// as  w(+e_j) = A + dp B  and  w(-e_j) = conj(A + dm B)  (dp, dm: the mode steps of the two neighbours, -1 and +1
// away from the frequency wrap). Each complex sum is formed as a (re, im) pair with packed FP32 multiply-adds
// (__ffma2_rn: two independent round-to-nearest fused multiply-adds), the lambda and q factors broadcast to both
// lanes. The products with the vectors accumulate per mode in two pairs, P = sum w.re (h.re, h.im) and
// S = sum w.im (h.re, h.im), so that each loaded value enters as it is stored; Q h = (P.re - S.im, P.im + S.re).
// Real tap values skip S. The mean tap is real.
__device__ __forceinline__ float2 pk(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 pk_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pk_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }

// ---- half-spectrum storage (StarParams.hspec): the last axis holds k_l = 0 .. Hl - 1 only. Of a run's last-axis
// neighbours, k - e_l of its first mode at k_l = 0 is the conjugate of the stored mirror entry (-k, k_l = 1), and
// k + e_l of its second mode at k_l = Hl - 1 is the dropped Nyquist mode (even N_l: 0) or, across the frequency
// wrap, the conjugate of the mirror entry (-k, k_l = Hl - 1) (odd N_l). A mode with a dropped Nyquist digit on
// another axis is not an unknown: its output is 0 (and its stored input is 0, so it adds nothing elsewhere).
struct HalfEdges {
  int il, ir;          // storage indices of the run's left and right last-axis neighbours
  bool cl, cr, zr;     // conjugate the left / right value; the right value is 0
  bool nyq_row;        // the run's modes have a dropped Nyquist digit
};

template <bool HSP>
__device__ __forceinline__ HalfEdges half_edges(const StarParams& sp, const int (&ib)[MAXN], int n, int e0, int ibl) {
  HalfEdges he;
  const int jl = n - 1, Nsl = sp.Nst[jl];
  he.il = e0 + ((ibl == 0) ? Nsl - 1 : -1);
  he.ir = e0 + ((ibl + 2 == Nsl) ? 2 - Nsl : 2);
  he.cl = he.cr = he.zr = he.nyq_row = false;
  if (HSP) {
    if (ibl == 0 || ibl + 2 == Nsl) {
      int mr = 0;   // storage index of (-k_0, .., -k_{n-2}, 0)
#pragma unroll
      for (int j = 0; j < MAXN - 1; ++j)
        if (j < jl) mr += (ib[j] == 0 ? 0 : sp.N[j] - ib[j]) * sp.stride[j];
      if (ibl == 0) {
        he.il = mr + 1;
        he.cl = true;
      }
      if (ibl + 2 == Nsl) {
        if (sp.N[jl] % 2 == 0) {
          he.zr = true;
          he.ir = e0;
        } else {
          he.ir = mr + Nsl - 1;
          he.cr = true;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < MAXN - 1; ++j)
      if (j < jl) he.nyq_row |= ib[j] == sp.nyq[j];
  }
  return he;
}

template <bool RO, bool HSP, typename V>
__device__ __forceinline__ V ld_edge(const V* p, bool conj, bool zero) {
  V v = ldh<RO>(p);
  if (HSP) {
    if (conj) v.y = -v.y;
    if (zero) {
      v.x = 0;
      v.y = 0;
    }
  }
  return v;
}

template <bool REALC, int NR, bool RO, int NAX = 0, int DC = 0, bool HSP = false>
__device__ __forceinline__ void apply_run_star_f32(const StarParams& sp, int e0, const float2* h, int D, int nrhs,
                                                   float2 (&acc)[2][NR]) {
  const int d = DC ? DC : sp.d, n = NAX ? NAX : sp.n, jl = n - 1, Nl = sp.N[jl];
  if (NAX != 0) nrhs = NR;   // the compiled-in geometries run with d = NR right-hand sides
  int ib[MAXN], k[MAXN];
  {
    uint32_t x = (uint32_t)e0;
#pragma unroll
    for (int j = MAXN - 1; j >= 0; --j) {
      if (j < n) {
        const uint32_t qd = fdiv(x, sp.div[j]);
        ib[j] = (int)(x - qd * (uint32_t)sp.Nst[j]);
        k[j] = (2 * ib[j] < sp.N[j]) ? ib[j] : ib[j] - sp.N[j];
        x = qd;
      } else {
        ib[j] = 0;
        k[j] = 0;
      }
    }
  }
  int ibl = 0, kl0 = 0;
#pragma unroll
  for (int j = 0; j < MAXN; ++j)
    if (j == jl) {
      ibl = ib[j];
      kl0 = k[j];
    }
  const int kl1 = (2 * (ibl + 1) < Nl) ? ibl + 1 : ibl + 1 - Nl;
  const HalfEdges he = half_edges<HSP>(sp, ib, n, e0, ibl);   // k - e_l of the run's first mode, k + e_l of its second
  // broadcast pairs per mode s of the run: (q_a, q_a) and (lambda_a, lambda_a)
  float2 QQ[2][MAXD], LL[2][MAXD];
  {
    float lr[MAXD];
#pragma unroll
    for (int a = 0; a < MAXD; ++a) {
      lr[a] = 0.f;
#pragma unroll
      for (int j = 0; j < MAXN - 1; ++j)
        if (a < d && j < jl) lr[a] = fmaf(sp.P32[a][j], (float)k[j], lr[a]);
    }
#pragma unroll
    for (int a = 0; a < MAXD; ++a) {
      const float pl = sp.P32[a][jl];
      const float l0 = (a < d) ? fmaf(pl, (float)kl0, lr[a]) : 0.f;
      const float l1 = (a < d) ? fmaf(pl, (float)kl1, lr[a]) : 0.f;
      LL[0][a] = pk(l0, l0);
      LL[1][a] = pk(l1, l1);
      QQ[0][a] = pk(l0 * l0, l0 * l0);
      QQ[1][a] = pk(l1 * l1, l1 * l1);
    }
  }
  const float2* hr[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) hr[r] = h + (size_t)r * D;
  float2 Pa[2][NR], Sa[2][NR];
  // mean tap (real): P = w0 h
  {
    float2 w0[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      w0[s] = pk_mul(pk(sp.c0r32[0], sp.c0r32[0]), QQ[s][0]);
#pragma unroll
      for (int a = 1; a < MAXD; ++a)
        if (a < d) w0[s] = pk_fma(pk(sp.c0r32[a], sp.c0r32[a]), QQ[s][a], w0[s]);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < nrhs) {
        float2 v[2];
        ld_run<RO, float, 2>(hr[r] + e0, v);
        Pa[0][r] = pk_mul(w0[0], v[0]);
        Pa[1][r] = pk_mul(w0[1], v[1]);
      } else {
        Pa[0][r] = Pa[1][r] = pk(0.f, 0.f);
      }
      Sa[0][r] = Sa[1][r] = pk(0.f, 0.f);
    }
  }
  // weights of axis j at mode s: wp (tap +e_j) and wmc, the conjugate of the tap -e_j's weight
  auto weights = [&](int j, int s, float dp, float dm, float2& wp, float2& wmc) {
    float2 A = pk_mul(sp.hc32[j][0], QQ[s][0]);
    float2 B = pk_mul(sp.hcp32[j][0], LL[s][0]);
#pragma unroll
    for (int a = 1; a < MAXD; ++a) {
      if (a < d) {
        A = pk_fma(sp.hc32[j][a], QQ[s][a], A);
        B = pk_fma(sp.hcp32[j][a], LL[s][a], B);
      }
    }
    wp = pk_fma(pk(dp, dp), B, A);
    wmc = pk_fma(pk(dm, dm), B, A);
  };
  // the product of weight w (conj: the conjugate of w) with the stored value v
  auto mac = [&](float2& P, float2& S, float2 w, bool conj, float2 v) {
    P = pk_fma(pk(w.x, w.x), v, P);
    if (!REALC) {
      const float wy = conj ? -w.y : w.y;
      S = pk_fma(pk(wy, wy), v, S);
    }
  };
  // the last axis: one neighbour each side of the run, the run's own values for the inner taps
  if (NAX != 0 || sp.has[jl]) {
    const int hl = sp.half[jl];
    const float dp0 = (ibl == hl) ? (float)(Nl - 1) : -1.f, dp1 = (ibl + 1 == hl) ? (float)(Nl - 1) : -1.f;
    const float dm0 = (ibl == hl - 1) ? (float)(1 - Nl) : 1.f, dm1 = (ibl + 1 == hl - 1) ? (float)(1 - Nl) : 1.f;
    float2 wp0, wm0, wp1, wm1;
    weights(jl, 0, dp0, dm0, wp0, wm0);
    weights(jl, 1, dp1, dm1, wp1, wm1);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < nrhs) {
        float2 v[2];
        ld_run<RO, float, 2>(hr[r] + e0, v);
        mac(Pa[0][r], Sa[0][r], wm0, true, v[1]);
        mac(Pa[1][r], Sa[1][r], wp1, false, v[0]);
        mac(Pa[0][r], Sa[0][r], wp0, false, ld_edge<RO, HSP>(hr[r] + he.il, he.cl, false));
        mac(Pa[1][r], Sa[1][r], wm1, true, ld_edge<RO, HSP>(hr[r] + he.ir, he.cr, he.zr));
      }
    }
  }
  // the other axes: one neighbour offset and one mode step per tap for the whole run
#pragma unroll
  for (int j = 0; j < MAXN - 1; ++j) {
    if (j < jl && (NAX != 0 || sp.has[j])) {
      const int Nj = sp.N[j], ibj = ib[j], hj = sp.half[j];
      const int ep = e0 + ((ibj == 0) ? sp.woff[j] : -sp.stride[j]);        // k - e_j (tap +e_j)
      const int em = e0 + ((ibj == Nj - 1) ? -sp.woff[j] : sp.stride[j]);   // k + e_j (tap -e_j)
      const float dp = (ibj == hj) ? (float)(Nj - 1) : -1.f;
      const float dm = (ibj == hj - 1) ? (float)(1 - Nj) : 1.f;
      float2 wp0, wm0, wp1, wm1;
      weights(j, 0, dp, dm, wp0, wm0);
      weights(j, 1, dp, dm, wp1, wm1);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (r < nrhs) {
          float2 u[2], v[2];
          ld_run<RO, float, 2>(hr[r] + ep, u);
          ld_run<RO, float, 2>(hr[r] + em, v);
          mac(Pa[0][r], Sa[0][r], wp0, false, u[0]);
          mac(Pa[1][r], Sa[1][r], wp1, false, u[1]);
          mac(Pa[0][r], Sa[0][r], wm0, true, v[0]);
          mac(Pa[1][r], Sa[1][r], wm1, true, v[1]);
        }
      }
    }
  }
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int r = 0; r < NR; ++r)
      acc[s][r] = (HSP && he.nyq_row) ? pk(0.f, 0.f)
                                      : (REALC ? Pa[s][r] : pk(Pa[s][r].x - Sa[s][r].y, Pa[s][r].y + Sa[s][r].x));
}

// WM: 0 the weights are formed here; 1 (T = double) they are read from sp.w64; 2 (T = double) they are formed and
// written to wout (the same arithmetic as WM = 0, so stored and formed weights agree bit for bit) and nothing
// else is done.
// NAX, DC (0: from sp at run time): the number of axes, every one of them with taps, and d known at compile time,
// so that the axis loop is straight-line code whose neighbour reads the compiler can issue early.
// FP32 with formed weights (WM = 0) takes apply_run_star_f32 above. HSP: compiled for half-spectrum plans (kernels
// are instantiated for both and launched by the plan's storage, so the full-spectrum code carries none of the
// half-spectrum edge handling).
template <typename T, bool REALC, int NR, bool RO, bool DIAGK, int WM = 0, int NAX = 0, int DC = 0, bool HSP = false>
__device__ __forceinline__ void apply_run_star(const StarParams& sp, int e0, const cplx<T>* h, int D, int nrhs,
                                               cplx<T> (&acc)[2][NR], void* wout = nullptr) {
  if constexpr (sizeof(T) == 4 && WM == 0) {
    apply_run_star_f32<REALC, NR, RO, NAX, DC, HSP>(sp, e0, reinterpret_cast<const float2*>(h), D, nrhs,
                                                    reinterpret_cast<float2(&)[2][NR]>(acc));
    return;
  } else {
  constexpr int NQ = DIAGK ? MAXD : 1;   // weight terms per mode: q_a (diagonal) or q (scalar)
  constexpr bool FORM = WM != 1;         // the weights are formed from lambda
  const int d = DC ? DC : sp.d, n = NAX ? NAX : sp.n, jl = n - 1, Nl = sp.N[jl];
  // storage digits and signed modes of the run's first mode
  int ib[MAXN], k[MAXN];
  {
    uint32_t x = (uint32_t)e0;
#pragma unroll
    for (int j = MAXN - 1; j >= 0; --j) {
      if (j < n) {
        const uint32_t qd = fdiv(x, sp.div[j]);
        ib[j] = (int)(x - qd * (uint32_t)sp.Nst[j]);
        k[j] = (2 * ib[j] < sp.N[j]) ? ib[j] : ib[j] - sp.N[j];
        x = qd;
      } else {
        ib[j] = 0;
        k[j] = 0;
      }
    }
  }
  int ibl = 0, kl0 = 0;
#pragma unroll
  for (int j = 0; j < MAXN; ++j)
    if (j == jl) {
      ibl = ib[j];
      kl0 = k[j];
    }
  const HalfEdges he = half_edges<HSP>(sp, ib, n, e0, ibl);   // k - e_l of the run's first mode, k + e_l of its second
  const cplx<T>* hr[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) hr[r] = h + (size_t)r * D;
  T lk[2][MAXD];
  T q[2][NQ];
  if constexpr (FORM) {
    T lr[MAXD];
#pragma unroll
    for (int a = 0; a < MAXD; ++a) {
      lr[a] = T(0);
#pragma unroll
      for (int j = 0; j < MAXN - 1; ++j)
        if (a < d && j < jl) lr[a] = fma(sp_P<T>(sp, a, j), (T)k[j], lr[a]);
    }
    const int kl1 = (2 * (ibl + 1) < Nl) ? ibl + 1 : ibl + 1 - Nl;
#pragma unroll
    for (int a = 0; a < MAXD; ++a) {
      const T pl = sp_P<T>(sp, a, jl);
      lk[0][a] = (a < d) ? fma(pl, (T)kl0, lr[a]) : T(0);
      lk[1][a] = (a < d) ? fma(pl, (T)kl1, lr[a]) : T(0);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (DIAGK) {
#pragma unroll
        for (int a = 0; a < NQ; ++a) q[s][a] = lk[s][a] * lk[s][a];
      } else {
        q[s][0] = T(0);
#pragma unroll
        for (int a = 0; a < MAXD; ++a)
          if (a < d) q[s][0] = fma(lk[s][a], lk[s][a], q[s][0]);
      }
    }
  }
  auto rterms = [&](int j, T (&rt)[2][NQ]) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (DIAGK) {
#pragma unroll
        for (int a = 0; a < NQ; ++a) rt[s][a] = lk[s][a] * sp_P<T>(sp, a, j);
      } else {
        rt[s][0] = T(0);
#pragma unroll
        for (int a = 0; a < MAXD; ++a)
          if (a < d) rt[s][0] = fma(lk[s][a], sp_P<T>(sp, a, j), rt[s][0]);
      }
    }
  };
  // weight of the tap m = +e_j (sg = 0) or -e_j (sg = 1) at one mode
  auto wgt = [&](int j, int sg, T dk, const T (&qs)[NQ], const T (&rs)[NQ]) {
    cplx<T> c;
    if (DIAGK) {
      c = mk<T>(0, 0);
#pragma unroll
      for (int a = 0; a < MAXD; ++a) {
        if (a < d) {
          const cplx<T> ca = sp_c<T>(sp, j, sg, a);
          const T x = fma(dk, rs[a], qs[a]);
          c.x = fma(ca.x, x, c.x);
          if (!REALC) c.y = fma(ca.y, x, c.y);
        }
      }
    } else {
      const cplx<T> c0 = sp_c<T>(sp, j, sg, 0);
      const T w = fma(dk, rs[0], qs[0]);
      c.x = c0.x * w;
      c.y = REALC ? T(0) : c0.y * w;
    }
    return c;
  };
  // the weights of the taps m = +-e_j at the run's two modes: formed (dp, dm per mode) or read
  auto pair_weights = [&](int j, const T (&dp)[2], const T (&dm)[2], cplx<T> (&wp)[2], cplx<T> (&wm)[2]) {
    if constexpr (FORM) {
      T rt[2][NQ];
      rterms(j, rt);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        wp[s] = wgt(j, 0, dp[s], q[s], rt[s]);
        wm[s] = wgt(j, 1, dm[s], q[s], rt[s]);
      }
      if constexpr (WM == 2) {
        wstore<REALC>(wout, 1 + 2 * j, e0, D, reinterpret_cast<const double2(&)[2]>(wp));
        wstore<REALC>(wout, 2 + 2 * j, e0, D, reinterpret_cast<const double2(&)[2]>(wm));
      }
    } else {
      wload<REALC>(sp, 1 + 2 * j, e0, D, reinterpret_cast<double2(&)[2]>(wp));
      wload<REALC>(sp, 2 + 2 * j, e0, D, reinterpret_cast<double2(&)[2]>(wm));
    }
  };
  // mean tap and the last axis' taps, from the run's own values and one neighbour on each side
  {
    cplx<T> c0[2];
    if constexpr (FORM) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (DIAGK) {
          c0[s] = mk<T>(0, 0);
#pragma unroll
          for (int a = 0; a < MAXD; ++a) {
            if (a < d) {
              const cplx<T> ca = sp_c0<T>(sp, a);
              c0[s].x = fma(ca.x, q[s][a], c0[s].x);
              if (!REALC) c0[s].y = fma(ca.y, q[s][a], c0[s].y);
            }
          }
        } else {
          const cplx<T> ca = sp_c0<T>(sp, 0);
          c0[s].x = ca.x * q[s][0];
          c0[s].y = REALC ? T(0) : ca.y * q[s][0];
        }
      }
      if constexpr (WM == 2) wstore<REALC>(wout, 0, e0, D, reinterpret_cast<const double2(&)[2]>(c0));
    } else {
      wload<REALC>(sp, 0, e0, D, reinterpret_cast<double2(&)[2]>(c0));
    }
    const bool has = NAX != 0 || sp.has[jl] != 0;
    cplx<T> wp[2], wm[2];
    if (has) {
      const int hl = sp.half[jl];
      const T dp[2] = {(ibl == hl) ? T(Nl - 1) : T(-1), (ibl + 1 == hl) ? T(Nl - 1) : T(-1)};
      const T dm[2] = {(ibl == hl - 1) ? T(1 - Nl) : T(1), (ibl + 1 == hl - 1) ? T(1 - Nl) : T(1)};
      pair_weights(jl, dp, dm, wp, wm);
    }
    if constexpr (WM != 2) {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (r < nrhs) {
          cplx<T> hv[2];
          ld_run<RO, T, 2>(hr[r] + e0, hv);
          cplx<T> a0 = mk<T>(0, 0), a1 = mk<T>(0, 0);
          mac<T, REALC>(a0, c0[0], hv[0]);
          mac<T, REALC>(a1, c0[1], hv[1]);
          if (has) {
            mac<T, REALC>(a0, wm[0], hv[1]);
            mac<T, REALC>(a1, wp[1], hv[0]);
            mac<T, REALC>(a0, wp[0], ld_edge<RO, HSP>(hr[r] + he.il, he.cl, false));
            mac<T, REALC>(a1, wm[1], ld_edge<RO, HSP>(hr[r] + he.ir, he.cr, he.zr));
          }
          acc[0][r] = a0;
          acc[1][r] = a1;
        } else {
          acc[0][r] = mk<T>(0, 0);
          acc[1][r] = mk<T>(0, 0);
        }
      }
    }
  }
  // the other axes: one neighbour offset and one dk per tap for the whole run
#pragma unroll
  for (int j = 0; j < MAXN - 1; ++j) {
    if (j < jl && (NAX != 0 || sp.has[j])) {
      const int Nj = sp.N[j], ibj = ib[j], hj = sp.half[j];
      const int ep = e0 + ((ibj == 0) ? sp.woff[j] : -sp.stride[j]);        // k - e_j (tap m = +e_j)
      const int em = e0 + ((ibj == Nj - 1) ? -sp.woff[j] : sp.stride[j]);   // k + e_j (tap m = -e_j)
      const T dpj = (ibj == hj) ? T(Nj - 1) : T(-1);
      const T dmj = (ibj == hj - 1) ? T(1 - Nj) : T(1);
      const T dp[2] = {dpj, dpj}, dm[2] = {dmj, dmj};
      cplx<T> wp[2], wm[2];
      pair_weights(j, dp, dm, wp, wm);
      if constexpr (WM != 2) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r < nrhs) {
            cplx<T> hv[2];
            ld_run<RO, T, 2>(hr[r] + ep, hv);
            mac<T, REALC>(acc[0][r], wp[0], hv[0]);
            mac<T, REALC>(acc[1][r], wp[1], hv[1]);
            ld_run<RO, T, 2>(hr[r] + em, hv);
            mac<T, REALC>(acc[0][r], wm[0], hv[0]);
            mac<T, REALC>(acc[1][r], wm[1], hv[1]);
          }
        }
      }
    }
  }
  if constexpr (WM != 2 && HSP) {
    if (he.nyq_row) {
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[q][r] = mk<T>(0, 0);
    }
  }
  }
}

// The star-1 run as a call of its own in kernels that also run the general stencil (batches of several plans):
// its registers are then allocated apart from the general stencil's, which keeps that one's register budget.
// FP64 runs read the plan's stored entries Q_ij where it has them (bitwise the weights formed here).
template <typename T, bool REALC, int NR, bool RO>
__device__ __noinline__ void star_run_call(const StarParams* st, bool diag, int e0, const cplx<T>* h, int D, int nrhs,
                                           cplx<T>* out) {
  cplx<T> acc[2][NR];
  const bool hs = st->hspec != 0;
  if constexpr (sizeof(T) == 8) {
    if (st->w64 != nullptr) {
      if (hs) {
        if (diag) apply_run_star<T, REALC, NR, RO, true, 1, 0, 0, true>(*st, e0, h, D, nrhs, acc);
        else apply_run_star<T, REALC, NR, RO, false, 1, 0, 0, true>(*st, e0, h, D, nrhs, acc);
      } else {
        if (diag) apply_run_star<T, REALC, NR, RO, true, 1>(*st, e0, h, D, nrhs, acc);
        else apply_run_star<T, REALC, NR, RO, false, 1>(*st, e0, h, D, nrhs, acc);
      }
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int r = 0; r < NR; ++r) out[s * NR + r] = acc[s][r];
      return;
    }
  }
  if (hs) {
    if (diag) apply_run_star<T, REALC, NR, RO, true, 0, 0, 0, true>(*st, e0, h, D, nrhs, acc);
    else apply_run_star<T, REALC, NR, RO, false, 0, 0, 0, true>(*st, e0, h, D, nrhs, acc);
  } else {
    if (diag) apply_run_star<T, REALC, NR, RO, true>(*st, e0, h, D, nrhs, acc);
    else apply_run_star<T, REALC, NR, RO, false>(*st, e0, h, D, nrhs, acc);
  }
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int r = 0; r < NR; ++r) out[s * NR + r] = acc[s][r];
}

// acc[s][r] = (Q h_r)(e0 + s), s < RUN: the whole tap sum at RUN consecutive modes (STAR: a star-1 plan takes the
// star-1 stencil with its StarParams from global memory; kernels that never see one leave it out) of one row of the last
// axis (e0 a multiple of RUN, RUN dividing N_{n-1}). Everything that depends only on the row is done once per
// run: the digits of e0, lambda over the other axes, and for every tap along another axis its wrapped offset and
// its mode step dk; that tap then reads RUN consecutive entries of h. The weights are formed per mode:
//   scalar:  c_t (|lambda|^2 + dk lambda.P_j),   otherwise  lambda^T C_t (lambda + dk P_j)   (star tap on axis j).
// (Q h)(e0 + s), s < RUN, of a half-spectrum plan with any taps, one mode and one tap at a time (kernels call it
// as a function of its own, so that its registers do not add to the full-spectrum stencil's). For tap t the
// neighbour k' = k - m_t is wrapped into [-N_j/2, N_j/2) per axis; a dropped Nyquist component makes it 0; a
// negative last component makes it the conjugate of the stored mirror entry -k'. The weight is
// lambda(k)^T C_t lambda(k') with the unmirrored k'. out[s * NR + r].
template <typename T, bool REALC, int NR, int RUN, bool RO>
__device__ __noinline__ void apply_run_half(const PlanDev& p, const cplx<T>* sc, int e0, const cplx<T>* h, int D,
                                            int nrhs, cplx<T>* out) {
  const int d = p.d, n = p.n, nc = p.ncomp, jl = n - 1;
  for (int s = 0; s < RUN; ++s) {
    int ib[MAXN], k[MAXN];
    mode_digits(p, e0 + s, ib, k);
    bool nyq_row = false;
    for (int j = 0; j < jl; ++j) nyq_row |= ib[j] == p.nyq[j];
    cplx<T> acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = mk<T>(0, 0);
    if (!nyq_row) {
      T lk[MAXD];
#pragma unroll
      for (int a = 0; a < MAXD; ++a) {
        lk[a] = T(0);
        for (int j = 0; j < n; ++j)
          if (a < d) lk[a] = fma(pcoef<T>(p, a, j), (T)k[j], lk[a]);
      }
      for (int t = 0; t < p.ntaps; ++t) {
        int kk[MAXN];
        bool zero = false, neg = false;
        for (int j = 0; j < n; ++j) {
          const int Nj = p.N[j];
          int x = k[j] - (int)p.m[t][j];
          x = ((x % Nj) + Nj) % Nj;                 // storage index of k_j - m_j
          x = (2 * x < Nj) ? x : x - Nj;            // signed, in [-N_j/2, N_j/2)
          zero |= (Nj % 2 == 0) && (2 * x == -Nj);  // the dropped Nyquist mode
          kk[j] = x;
        }
        if (zero) continue;
        neg = kk[jl] < 0;
        T l2[MAXD];
#pragma unroll
        for (int a = 0; a < MAXD; ++a) {
          l2[a] = T(0);
          for (int j = 0; j < n; ++j)
            if (a < d) l2[a] = fma(pcoef<T>(p, a, j), (T)kk[j], l2[a]);
        }
        int idx = 0;
        for (int j = 0; j < n; ++j) {
          const int x = neg ? -kk[j] : kk[j];
          idx += (j == jl ? x : (x < 0 ? x + p.N[j] : x)) * p.stride[j];
        }
        const cplx<T> c = weight_general<T>(p.kind, d, sc + t * nc, lk, l2);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r < nrhs) {
            cplx<T> v = ldh<RO>(h + (size_t)r * D + idx);
            if (neg) v.y = -v.y;
            mac<T, REALC>(acc[r], c, v);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) out[s * NR + r] = acc[r];
  }
}

// Stored FP64 entries of a general-taps plan (PlanDev.wgen): the weight of sorted tap t at mode e.
template <bool REALC>
__device__ __forceinline__ double2 wgen_load(const PlanDev& p, int t, int e, int D) {
  if (REALC || p.wgen_real) return make_double2(__ldg(static_cast<const double*>(p.wgen) + (size_t)t * D + e), 0.0);
  return __ldg(static_cast<const double2*>(p.wgen) + (size_t)t * D + e);
}
template <bool REALC>
__device__ __forceinline__ void wgen_store(void* out, int t, int e, int D, double2 c) {
  if (REALC) static_cast<double*>(out)[(size_t)t * D + e] = c.x;
  else static_cast<double2*>(out)[(size_t)t * D + e] = c;
}

// WM (general taps; T = double): 0 the weights are formed; 1 they are read from p.wgen (chosen at run time when the
// plan stores them); 2 they are formed and written to wout, nothing else is done (the stencil's own arithmetic, so
// stored and formed weights agree bit for bit).
// NG: the plan's number of axes compiled in (the batch kernels dispatch the common ones; 0: read at run time). The
// per-axis loops then stop at the plan's axes instead of testing every axis up to MAXN; the arithmetic is the same.
template <typename T, bool REALC, int NR, int RUN, bool RO = true, bool STAR = true, int WM = 0, int NG = 0>
__device__ __forceinline__ void apply_run(const PlanDev& p, const cplx<T>* __restrict__ sc, int e0,
                                          const cplx<T>* h, int D, int nrhs, cplx<T> (&acc)[RUN][NR],
                                          void* wout = nullptr) {
  if constexpr (RUN == 2 && STAR && WM != 2) {
    if (p.star1) {   // the plan's StarParams read from global memory (L1-resident across the block)
      star_run_call<T, REALC, NR, RO>(p.star, p.kind == QP_COEF_DIAG, e0, h, D, nrhs, &acc[0][0]);
      return;
    }
  }
  if (p.hspec) {
    apply_run_half<T, REALC, NR, RUN, RO>(p, sc, e0, h, D, nrhs, &acc[0][0]);
    return;
  }
  if constexpr (sizeof(T) == 8 && WM == 0) {
    if (p.wgen) {
      apply_run<T, REALC, NR, RUN, RO, STAR, 1, NG>(p, sc, e0, h, D, nrhs, acc);
      return;
    }
  }
  // the weight of sorted tap t at mode e0 + s: read (WM 1), or the formed value, also stored (WM 2)
  auto wsel = [&](int t, int s, const cplx<T>& formed) -> cplx<T> {
    if constexpr (WM == 1) {
      const double2 c = wgen_load<REALC>(p, t, e0 + s, D);
      return mk<T>((T)c.x, (T)c.y);
    } else {
      if constexpr (WM == 2) wgen_store<REALC>(wout, t, e0 + s, D, make_double2((double)formed.x, (double)formed.y));
      return formed;
    }
  };
  int ib[MAXN], k[MAXN];
  mode_digits<NG>(p, e0, ib, k);
  const int d = p.d, kind = p.kind, nc = p.ncomp, n = NG ? NG : p.n;
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
      cplx<T> f = mk<T>(0, 0);
      if constexpr (WM != 1) {
        if (scalar) {
          f.x = sc[0].x * lam2[s];
          f.y = REALC ? T(0) : sc[0].y * lam2[s];
        } else {
          f = weight_general<T>(kind, d, sc, lk[s], lk[s]);
        }
      }
      c[s] = wsel(0, s, f);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (WM != 2 && r < nrhs) {
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
          cplx<T> f = mk<T>(0, 0);
          if constexpr (WM != 1) {
            if (scalar) {
              const T w = fma(dk, lp[s], lam2[s]);
              f.x = ct[0].x * w;
              f.y = REALC ? T(0) : ct[0].y * w;
            } else {
              T l2[MAXD];
#pragma unroll
              for (int a = 0; a < MAXD; ++a) l2[a] = (a < d) ? fma(dk, pj[a], lk[s][a]) : T(0);
              f = weight_general<T>(kind, d, ct, lk[s], l2);
            }
          }
          c[s] = wsel(t, s, f);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (WM != 2 && r < nrhs) {
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
        cplx<T> f = mk<T>(0, 0);
        if constexpr (WM != 1) {
          if (scalar) {
            const T w = fma(dk, lp[s], lam2[s]);
            f.x = ct[0].x * w;
            f.y = REALC ? T(0) : ct[0].y * w;
          } else {
            T l2[MAXD];
#pragma unroll
            for (int a = 0; a < MAXD; ++a) l2[a] = (a < d) ? fma(dk, pl[a], lk[s][a]) : T(0);
            f = weight_general<T>(kind, d, ct, lk[s], l2);
          }
        }
        const cplx<T> c = wsel(t, s, f);
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (WM != 2 && r < nrhs) mac<T, REALC>(acc[s][r], c, ldh<RO>(hr[r] + row0 + ib2));
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
      cplx<T> f = mk<T>(0, 0);
      if constexpr (WM != 1) {
        T l2[MAXD];
#pragma unroll
        for (int a = 0; a < MAXD; ++a) l2[a] = (a < d) ? fma(dk, pcoef<T>(p, a, jl), lk[s][a] + lo[a]) : T(0);
        f = weight_general<T>(kind, d, ct, lk[s], l2);
      }
      const cplx<T> c = wsel(t, s, f);
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (WM != 2 && r < nrhs) mac<T, REALC>(acc[s][r], c, ldh<RO>(hr[r] + eo + ib2));
    }
  }
}

}  // namespace qp
