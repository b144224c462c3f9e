// Conversions between the FP64 vectors of the refinement loop and its FP32 inner vectors, scaled by a power of two
// 2^-e (the refinement's scale, near 1 / ||r||): with a power of two the scaling is exact, so the narrowing
// (float)(x 2^-e) is one rounding and the widening (double)c 2^e is exact. Both are done on the bit patterns with
// integer instructions, because a GB300 SM issues only about two FP64 operations per clock: an FP64 multiply and an
// FP64 conversion per value made the two refinement passes FP64-bound instead of bandwidth-bound. The cases the bit
// manipulation does not cover (FP64 subnormals, infinities and NaNs, exponents outside the normal range) take the
// FP64 expression, which gives the same value.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define QP_HD __host__ __device__ __forceinline__
#define QP_HD_COLD static __host__ __device__ __noinline__
#else
#define QP_HD inline
#define QP_HD_COLD static __attribute__((noinline))
#endif

namespace qp {

QP_HD uint64_t f64_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  __builtin_memcpy(&u, &x, sizeof u);
  return u;
#endif
}
QP_HD double f64_from(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  __builtin_memcpy(&x, &u, sizeof x);
  return x;
#endif
}
QP_HD uint32_t f32_bits(float x) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(x);
#else
  uint32_t u;
  __builtin_memcpy(&u, &x, sizeof u);
  return u;
#endif
}
QP_HD float f32_from(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  __builtin_memcpy(&x, &u, sizeof x);
  return x;
#endif
}

// 2^k for the exponents of the normal FP64 range (|k| <= 1022).
QP_HD double pow2(int k) { return f64_from((uint64_t)(k + 1023) << 52); }

// The exponent e of a power of two 2^e in the normal FP64 range.
QP_HD int pow2_exponent(double p) { return (int)((f64_bits(p) >> 52) & 0x7ff) - 1023; }

// The refinement's scale for a residual of squared norm s0: inv = 2^e with 2^e <= ||r|| < 2^(e + 1) (e = floor(E / 2)
// for s0 = 2^E m, 1 <= m < 2), scale = 2^-e; both 0 unless s0 is positive and finite.
QP_HD void refine_scale(double s0, double& scale, double& inv) {
  const int E = (int)((f64_bits(s0) >> 52) & 0x7ff) - 1023;
  if (!(s0 > 0.0) || E > 1023) {
    scale = inv = 0.0;
    return;
  }
  const int Ec = E >= -1022 ? E : -1022;   // an FP64 subnormal s0 takes 2^-511
  int e = (Ec - (Ec < 0 ? 1 : 0)) / 2;      // floor(Ec / 2)
  e = e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
  inv = pow2(e);
  scale = pow2(-e);
}

// The FP64 expressions themselves, for the cases below that the bit manipulation leaves out: calls of their own,
// so that the compiler keeps them behind a branch instead of evaluating them for every value (inlined, the
// widening's FP64 multiply and conversion ran unconditionally and bound its pass again).
QP_HD_COLD float narrow_pow2_slow(double x, int e) { return (float)(x * pow2(-e)); }
QP_HD_COLD double widen_pow2_slow(float c, int e) { return (double)c * pow2(e); }

// (float)(x 2^-e), round to nearest even. The 53-bit significand keeps its top 24 bits (hidden bit included); the
// 29 bits below decide the rounding, with ties to the even neighbour.
QP_HD float narrow_pow2(double x, int e) {
  const uint64_t u = f64_bits(x);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t sign = hi & 0x80000000u;
  const int ex = (int)((hi >> 20) & 0x7ffu);
  if (ex == 0 && (hi & 0xfffffu) == 0 && lo == 0) return f32_from(sign);   // signed zero
  const int fe = ex - 1023 - e + 127;                                      // the FP32 biased exponent
  if (ex == 0 || ex == 0x7ff || fe < 1 || fe > 253) return narrow_pow2_slow(x, e);
  uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);                      // 23 fraction bits
  const uint32_t rem = lo & 0x1fffffffu, half = 0x10000000u;
  uint32_t r = ((uint32_t)fe << 23) | m;
  if (rem > half || (rem == half && (m & 1u))) ++r;                        // a carry into the exponent is right
  return f32_from(sign | r);
}

// (double)c 2^e, exact.
QP_HD double widen_pow2(float c, int e) {
  const uint32_t u = f32_bits(c);
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  const int fe = (int)((u >> 23) & 0xffu);
  const uint32_t m = u & 0x7fffffu;
  if (fe == 0 && m == 0) return f64_from(sign);                             // signed zero
  const int de = fe - 127 + e + 1023;                                       // the FP64 biased exponent
  if (fe == 0 || fe == 255 || de < 1 || de > 2046) return widen_pow2_slow(c, e);
  return f64_from(sign | ((uint64_t)de << 52) | ((uint64_t)m << 29));
}

}  // namespace qp
