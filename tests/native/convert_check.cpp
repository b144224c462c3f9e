// Checks the refinement's power-of-two conversions (paper_2404_06841_gb300/csrc/qp_convert.cuh, host path) against
// the FP64 expressions they stand for, bit for bit: narrow_pow2(x, e) == (float)(x * 2^-e) and
// widen_pow2(c, e) == (double)c * 2^e, and refine_scale's bracket 2^e <= sqrt(s0) < 2^(e+1).
// Prints "ok <count>" or the first mismatch and exits non-zero.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "qp_convert.cuh"

static bool same_f(float a, float b) {
  if (std::isnan(a) || std::isnan(b)) return std::isnan(a) && std::isnan(b);
  uint32_t x, y;
  std::memcpy(&x, &a, 4);
  std::memcpy(&y, &b, 4);
  return x == y;
}
static bool same_d(double a, double b) {
  if (std::isnan(a) || std::isnan(b)) return std::isnan(a) && std::isnan(b);
  uint64_t x, y;
  std::memcpy(&x, &a, 8);
  std::memcpy(&y, &b, 8);
  return x == y;
}
static double dbits(uint64_t u) {
  double x;
  std::memcpy(&x, &u, 8);
  return x;
}
static float fbits(uint32_t u) {
  float x;
  std::memcpy(&x, &u, 4);
  return x;
}

int main() {
  std::mt19937_64 g(12345);
  long n = 0;
  auto narrow = [&](double x, int e) {
    const float want = (float)(x * std::ldexp(1.0, -e)), got = qp::narrow_pow2(x, e);
    ++n;
    if (!same_f(want, got)) {
      std::printf("narrow mismatch x=%a e=%d want=%a got=%a\n", x, e, (double)want, (double)got);
      return false;
    }
    return true;
  };
  auto widen = [&](float c, int e) {
    const double want = (double)c * std::ldexp(1.0, e), got = qp::widen_pow2(c, e);
    ++n;
    if (!same_d(want, got)) {
      std::printf("widen mismatch c=%a e=%d want=%a got=%a\n", (double)c, e, want, got);
      return false;
    }
    return true;
  };
  const int es[] = {0, 1, -1, 5, -7, 20, -20, 33, -40, 100, -100, 126, -126, 300, -300, 1000, -1000};
  // random bit patterns of every exponent, and random values around each scale
  for (int i = 0; i < 2000000; ++i) {
    const uint64_t u = g();
    const int e = es[i % 17];
    if (!narrow(dbits(u), e)) return 1;
    const double x = std::ldexp((double)(g() >> 11) * 0x1p-53 * ((g() & 1) ? 1 : -1), e + (int)(g() % 300) - 200);
    if (!narrow(x, e)) return 1;
    if (!widen(fbits((uint32_t)u), e)) return 1;
  }
  // ties and carries: 24 kept bits, the dropped 29 bits exactly half, just below and above; all-ones fractions
  for (int i = 0; i < 200000; ++i) {
    const int e = es[i % 17];
    const uint64_t frac = g() & ((1ull << 52) - 1);
    const uint64_t ex = (uint64_t)(1023 + e + (int)(g() % 250) - 125) & 0x7ff;
    const uint64_t sgn = (g() & 1) << 63;
    const uint64_t lows[] = {1ull << 28, (1ull << 28) - 1, (1ull << 28) + 1, 0, (1ull << 29) - 1};
    for (uint64_t lo : lows) {
      const uint64_t f2 = (frac & ~((1ull << 29) - 1)) | lo;
      if (!narrow(dbits(sgn | (ex << 52) | f2), e)) return 1;
      if (!narrow(dbits(sgn | (ex << 52) | ((1ull << 52) - 1 - ((1ull << 29) - 1)) | lo), e)) return 1;
    }
  }
  // zeros, FP64 subnormals, infinities, NaN; FP32 subnormal and overflowing results
  const double special[] = {0.0, -0.0, 4.9e-324, -4.9e-324, 2.2e-308, INFINITY, -INFINITY, NAN, 1.0, -1.0,
                            1.1754943508222875e-38, 1.1754942106924411e-38, 1.401298464324817e-45,
                            7.006492321624085e-46, 7.006492321624087e-46, 3.4028234663852886e+38,
                            3.4028235677973366e+38, 1e300};
  for (double x : special)
    for (int e : es)
      if (!narrow(x, e) || !narrow(x * 0x1p-3, e) || !narrow(std::ldexp(x, e), e)) return 1;
  const float fspecial[] = {0.f, -0.f, 1.4e-45f, -1.4e-45f, 1.17e-38f, 3.4e38f, INFINITY, -INFINITY, NAN, 1.f};
  for (float c : fspecial)
    for (int e : es)
      if (!widen(c, e)) return 1;
  // the scale: 2^e <= sqrt(s0) < 2^(e+1) and scale * inv == 1 for positive finite s0
  for (int i = 0; i < 1000000; ++i) {
    const double s0 = std::ldexp((double)(g() >> 11) * 0x1p-53 + 0x1p-60, (int)(g() % 2000) - 1000);
    double sc, inv;
    qp::refine_scale(s0, sc, inv);
    const double r = std::sqrt(s0);
    ++n;
    if (!(inv <= r && r < 2 * inv && sc * inv == 1.0)) {
      std::printf("scale mismatch s0=%a inv=%a sc=%a\n", s0, inv, sc);
      return 1;
    }
  }
  double sc = 1, inv = 1;
  qp::refine_scale(0.0, sc, inv);
  if (sc != 0.0 || inv != 0.0) return 1;
  qp::refine_scale(NAN, sc, inv);
  if (sc != 0.0 || inv != 0.0) return 1;
  qp::refine_scale(INFINITY, sc, inv);
  if (sc != 0.0 || inv != 0.0) return 1;
  std::printf("ok %ld\n", n);
  return 0;
}
