// Double transcendentals of the FP64 near field, written for this library.
//
//   dlog  natural logarithm of a positive, normal, finite double by the
//         table-driven reduction of P. T. P. Tang ("Table-driven
//         implementation of the logarithm function in IEEE floating-point
//         arithmetic", ACM TOMS 16(4), 1990): x = 2^e m with m in [1, 2); the
//         six leading fraction bits j of m pick c_j = 1 + (j + 1/2)/64;
//         r = m / c_j - 1 is formed as fma(m, ic_j, -1) with ic_j = 1/c_j
//         rounded to double, so that m ic_j = 1 + r up to one rounding of r;
//         then log x = e ln 2 + lc_j + log1p(r) with lc_j = -log(ic_j), and
//         log1p(r) from its Taylor series to r^9 (|r| < 2^-7, truncation
//         below 2^-73).  Absolute error a few units of 2^-53 times max(1,
//         |log x|).  The table of the 64 pairs (ic_j, lc_j) is built on the
//         device with CUDA's double division and logarithm.
//   datan2_ypos
//         atan2(y, x) for y >= 0 and finite arguments, in [0, pi], by octant
//         reduction to a = min(y, |x|) / max(y, |x|) in [0, 1] and a table of
//         64 breakpoints c_j = j/64: with j = floor(64 a) (from an
//         approximate reciprocal, so possibly one off at a breakpoint),
//         atan(a) = atan(c_j) + atan(z), z = (a - c_j)/(1 + a c_j) formed
//         from the numerator and denominator of a with one double division,
//         |z| < 2^-5; atan(z) from its Taylor series to z^11 (truncation
//         below 2^-65).  The addition theorem and the series are textbook;
//         the table of (c_j, atan(c_j)) is built on the device with CUDA's
//         double arctangent.  Relative error a few units of 2^-53 for
//         arguments of magnitude within [2^-1000, 2^1000] (the approximate
//         reciprocal flushes subnormals); x = y = 0 gives 0.
// The GPU tests compare dlog with CUDA's log and datan2_ypos with CUDA's atan2.
#pragma once
#include <cuda_runtime.h>

namespace bem {

constexpr int kDlogTab = 64;

__device__ __forceinline__ double dlog(double x, const double2* __restrict__ tab) {
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff) - 1023;
  const int j = (int)((bits >> 46) & (kDlogTab - 1));
  const double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  const double2 t = __ldg(tab + j);
  const double r = fma(m, t.x, -1.0);
  // log1p(r) = r (1 - r/2 + r^2/3 - ... + r^8/9)
  double p = 1.0 / 9.0;
  p = fma(p, r, -1.0 / 8.0);
  p = fma(p, r, 1.0 / 7.0);
  p = fma(p, r, -1.0 / 6.0);
  p = fma(p, r, 1.0 / 5.0);
  p = fma(p, r, -1.0 / 4.0);
  p = fma(p, r, 1.0 / 3.0);
  p = fma(p, r, -0.5);
  p = fma(p, r, 1.0);
  constexpr double kLn2d = 0.6931471805599453094;
  return fma((double)e, kLn2d, fma(r, p, t.y));
}

constexpr int kDatanTab = 64;

__device__ __forceinline__ double rcp_approx_f64(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}

__device__ __forceinline__ double datan2_ypos(double y, double x, const double2* __restrict__ tab) {
  constexpr double kPiD = 3.141592653589793116, kPi2D = 1.5707963267948965580;
  const double ax = fabs(x);
  const bool sw = y > ax;                 // the angle is within pi/4 of pi/2
  const double num = sw ? ax : y, den = sw ? y : ax;
  if (den == 0.0) return 0.0;
  // j = floor(64 a) from a + 1 in [1, 2): its six leading fraction bits
  const double a1 = fmin(num * rcp_approx_f64(den), 0.9999) + 1.0;
  const int j = (int)((__double_as_longlong(a1) >> 46) & (kDatanTab - 1));
  const double2 t = __ldg(tab + j);      // (c_j, atan(c_j))
  const double z = fma(-t.x, den, num) / fma(t.x, num, den);
  // atan(z) = z (1 - z^2/3 + z^4/5 - ... - z^10/11)
  const double s = z * z;
  double p = -1.0 / 11.0;
  p = fma(p, s, 1.0 / 9.0);
  p = fma(p, s, -1.0 / 7.0);
  p = fma(p, s, 1.0 / 5.0);
  p = fma(p, s, -1.0 / 3.0);
  const double at = fma(z * s, p, z) + t.y;     // atan(a) in [0, pi/4]
  if (sw) return x >= 0.0 ? kPi2D - at : kPi2D + at;
  return x >= 0.0 ? at : kPiD - at;
}

}  // namespace bem
