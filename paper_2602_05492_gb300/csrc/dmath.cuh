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
// The GPU tests compare dlog with CUDA's log.
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

}  // namespace bem
