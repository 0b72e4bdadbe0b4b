// Float transcendentals of the hot pair loops, written for this library.
//
//   fm_atan2       octant reduction to a = min/max in [0, 1] (one approximate
//                  reciprocal), atan(a) = a p(a^2) with p of degree 7 from a
//                  minimax fit (Lawson's iteratively reweighted least
//                  squares, fit_atan.py); |error| < 2e-7 in float
//   fm_atan2_ypos  the same for y >= 0 (result in [0, pi]); the layer
//                  integrals' angle atan2(h' L, h'^2 + t1 t2) always has y >= 0
//   mufu_lg2, mufu_rsqrt, mufu_rcp
//                  the MUFU approximations (PTX lg2/rsqrt/rcp.approx) in
//                  their flush-to-zero form: the pair loops never pass them
//                  a subnormal (every argument is at least eps^2, a floored
//                  maximum or a panel length), so the subnormal handling of
//                  the non-ftz forms is instructions spent on nothing
//   fm_log         the MUFU base-2 logarithm (__log2f) times ln 2
//   fm_log1p       |z| < 1/4: 2 atanh(s) with s = z/(2+z) from its odd Taylor
//                  series to s^9 (truncation < 1e-10); otherwise fm_log(1+z)
//   fm_log1p_half  (1/2) log1p(z), the form the folded layer formulas use
// The GPU tests compare each against CUDA's accurate float functions.
#pragma once
#include <cuda_runtime.h>

namespace bem {

constexpr float kLn2f = 0.693147181f;
constexpr float kLn2Halff = 0.346573591f;   // (ln 2)/2
constexpr float kFltMinNormal = 1.17549435e-38f;

__device__ __forceinline__ float mufu_lg2(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float mufu_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float mufu_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

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

// atan2(y, x), result in [-pi, pi].  max(|x|, |y|) is floored at the
// smallest normal float (x = y = 0 gives 0 without a branch).
__device__ __forceinline__ float fm_atan2(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(fmaxf(ax, ay), kFltMinNormal), mn = fminf(ax, ay);
  const float a = mn * mufu_rcp(mx);
  float r = fm_atan01(a);
  r = ay > ax ? 1.57079637f - r : r;
  r = x < 0.f ? 3.14159274f - r : r;
  return copysignf(r, y);
}

// atan2(y, x) for y >= 0, result in [0, pi].  max(|x|, y) is floored at the
// smallest normal float so that x = y = 0 gives 0 without a branch.
__device__ __forceinline__ float fm_atan2_ypos(float y, float x) {
  const float ax = fabsf(x);
  const float mx = fmaxf(fmaxf(ax, y), kFltMinNormal), mn = fminf(ax, y);
  float r = fm_atan01(mn * mufu_rcp(mx));
  r = y > ax ? 1.57079637f - r : r;
  return x < 0.f ? 3.14159274f - r : r;
}

__device__ __forceinline__ float fm_log(float x) { return __log2f(x) * kLn2f; }

// atanh(s) = (1/2) log1p(z) with s = z/(2+z), for |z| < 1/4, from the odd
// series s + s^3/3 + ... + s^9/9
__device__ __forceinline__ float fm_atanh_series(float z) {
  const float s = __fdividef(z, 2.f + z);
  const float s2 = s * s;
  float p = fmaf(s2, 1.f / 9.f, 1.f / 7.f);
  p = fmaf(p, s2, 1.f / 5.f);
  p = fmaf(p, s2, 1.f / 3.f);
  return fmaf(s * s2, p, s);
}

__device__ __forceinline__ float fm_log1p(float z) {
  if (fabsf(z) < 0.25f) return 2.f * fm_atanh_series(z);
  return fm_log(1.f + z);
}

__device__ __forceinline__ float fm_log1p_half(float z) {
  if (fabsf(z) < 0.25f) return fm_atanh_series(z);
  return __log2f(1.f + z) * kLn2Halff;
}

}  // namespace bem
