// Float transcendentals of the hot pair loops, written for this library.
//
//   fm_atan2  octant reduction to a = min/max in [0, 1] (one approximate
//             division), atan(a) = a p(a^2) with p of degree 7 from a minimax
//             fit (Lawson's iteratively reweighted least squares,
//             fit_atan.py); |error| < 2e-7 in float
//   fm_log    the MUFU base-2 logarithm (__log2f) times ln 2
//   fm_log1p  |z| < 1/4: 2 atanh(s) with s = z/(2+z) from its odd Taylor
//             series to s^9 (truncation < 1e-10); otherwise fm_log(1+z)
// The GPU tests compare each against CUDA's accurate float functions.
#pragma once
#include <cuda_runtime.h>

namespace bem {

__device__ __forceinline__ float fm_atan01(float a) {
  const float s = a * a;
  float p = -4.054566845e-03f;
  p = fmaf(p, s, 2.186295576e-02f);
  p = fmaf(p, s, -5.591232330e-02f);
  p = fmaf(p, s, 9.642197192e-02f);
  p = fmaf(p, s, -1.390862912e-01f);
  p = fmaf(p, s, 1.994656622e-01f);
  p = fmaf(p, s, -3.332985938e-01f);
  p = fmaf(p, s, 9.999993443e-01f);
  return a * p;
}

// atan2(y, x), result in [-pi, pi]
__device__ __forceinline__ float fm_atan2(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  const float a = mx > 0.f ? __fdividef(mn, mx) : 0.f;
  float r = fm_atan01(a);
  r = ay > ax ? 1.57079637f - r : r;
  r = x < 0.f ? 3.14159274f - r : r;
  return copysignf(r, y);
}

__device__ __forceinline__ float fm_log(float x) { return __log2f(x) * 0.693147181f; }

__device__ __forceinline__ float fm_log1p(float z) {
  if (fabsf(z) < 0.25f) {
    const float s = __fdividef(z, 2.f + z);
    const float s2 = s * s;
    float p = fmaf(s2, 1.f / 9.f, 1.f / 7.f);
    p = fmaf(p, s2, 1.f / 5.f);
    p = fmaf(p, s2, 1.f / 3.f);
    return 2.f * fmaf(s * s2, p, s);
  }
  return fm_log(1.f + z);
}

}  // namespace bem
