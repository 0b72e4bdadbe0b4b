// Device-side building blocks shared by the kernels of libbemgb.
//
// Notation (Sec. 3.1, Eq. (fundsol), (handleterm)):  a straight panel a->b of
// length L, unit tangent tau, right normal n = (tau_y, -tau_x).  Seen from a
// point x it has the frame coordinates
//     t1 = (a-x).tau,  t2 = t1 + L,  h = (a-x).n,  h'^2 = h^2 + eps^2
// and the regularised layer integrals (r -> sqrt(r^2+eps^2), Sec. 3.1.3)
//     S  = -(1/4pi) [ t2 log q2 - t1 log q1 - 2L + 2 h' Phi ],   qi = ti^2 + h'^2
//     Dl = -(1/2pi) (h/h') Phi,      Phi = atan2(h' L, h'^2 + t1 t2)
// S multiplies w_c and Dl multiplies -w_d in the handle term f.
//
// The double path evaluates t2 log q2 - t1 log q1 as L log q2 +
// t1 log1p(L (t1+t2)/q1), which has no cancellation when the panel is far
// from x (t1 ~ t2).  The float loops take both logarithms directly with the
// MUFU base-2 logarithm: the cancellation costs a few float ulps of log q
// times |t1|, far inside the mixed path's colour and gradient bounds.
//
// Endpoint derivatives go through the frame: with F(t1, t2, h)
//     dF/da = F_t1 tau + n [ -(h/L)(F_t1+F_t2) + (t2/L) F_h ]
//     dF/db = F_t2 tau + n [  (h/L)(F_t1+F_t2) - (t1/L) F_h ]
// and the partials
//     S_t1 = log q1/(4pi), S_t2 = -log q2/(4pi), S_h = -(1/2pi)(h/h')Phi
//     Dl_t1 = h/(2pi q1), Dl_t2 = -h/(2pi q2)
//     Dl_h = -(1/2pi)(1/h'^2) [ eps^2 Phi/h' - h^2 L (h'^2 - t1 t2)/(q1 q2) ]
// (each layer with its own eps).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fastmath.cuh"

namespace bem {

constexpr double kPi = 3.14159265358979323846;
constexpr double kInv2Pi = 0.15915494309189533577;   // 1/(2 pi)
constexpr double kInv4Pi = 0.07957747154594766788;   // 1/(4 pi)

// One straight panel as the kernels stage it (12 words, 16-byte aligned so
// that a float panel is three 128-bit loads).
template <typename T>
struct __align__(16) Panel {
  T ax, ay;      // start point a
  T tx, ty;      // unit tangent (0,0 for a zero-length panel)
  T L;           // length
  T wd[3];       // colour jump, Eq. (handleterm)
  T wc[3];       // normal-derivative jump
  T pad;
};

// 3-point Gauss-Legendre rule on [0,1] (Sec. 3.1.3)
__host__ __device__ inline double gauss_node(int q) {
  return q == 0 ? 0.11270166537925831148 : (q == 1 ? 0.5 : 0.88729833462074168852);
}
__host__ __device__ inline double gauss_weight(int q) {
  return q == 1 ? (8.0 / 18.0) : (5.0 / 18.0);
}

// cubic Bernstein weight j at t
template <typename T>
__host__ __device__ inline T bern3(int j, T t) {
  T s = T(1) - t;
  switch (j) {
    case 0: return s * s * s;
    case 1: return T(3) * t * s * s;
    case 2: return T(3) * t * t * s;
    default: return t * t * t;
  }
}

// math wrappers resolving to CUDA's float / double functions
__device__ inline float m_log(float x) { return logf(x); }
__device__ inline double m_log(double x) { return log(x); }
__device__ inline float m_log1p(float x) { return log1pf(x); }
__device__ inline double m_log1p(double x) { return log1p(x); }
__device__ inline float m_atan2(float y, float x) { return atan2f(y, x); }
__device__ inline double m_atan2(double y, double x) { return atan2(y, x); }
__device__ inline float m_sqrt(float x) { return sqrtf(x); }
__device__ inline double m_sqrt(double x) { return sqrt(x); }

// Frame of a panel seen from (x, y).
template <typename T>
struct Frame {
  T t1, t2, h, L;
};

template <typename T>
__device__ __forceinline__ Frame<T> frame(const Panel<T>& p, T x, T y) {
  Frame<T> f;
  T dax = p.ax - x, day = p.ay - y;
  f.t1 = dax * p.tx + day * p.ty;
  f.h = dax * p.ty - day * p.tx;
  f.L = p.L;
  f.t2 = f.t1 + p.L;
  return f;
}

// Near-field decision of the mixed-precision path: the distance from x to
// the panel segment is below near_factor * L (compared squared).  Every
// kernel that takes it (the float main loops that skip these pairs and the
// double near-field kernels that take them) computes the frame with the same
// explicitly rounded operations, so the decision agrees bit for bit.
__device__ __forceinline__ Frame<float> frame_rn(float ax, float ay, float tx, float ty, float L,
                                                 float x, float y) {
  Frame<float> f;
  const float dax = __fsub_rn(ax, x), day = __fsub_rn(ay, y);
  f.t1 = __fmaf_rn(dax, tx, __fmul_rn(day, ty));
  f.h = __fmaf_rn(dax, ty, -__fmul_rn(day, tx));
  f.t2 = __fadd_rn(f.t1, L);
  f.L = L;
  return f;
}

// near_factor^2 L^2
__device__ __forceinline__ float near_thr(float L, float near2) {
  return __fmul_rn(near2, __fmul_rn(L, L));
}

// hh = h*h of the frame.  The along-panel offset max(t1,0) + min(t2,0) is
// t1, t2 or 0 as x projects before, after or onto the panel (t1 <= t2).
__device__ __forceinline__ bool near_test(const Frame<float>& f, float hh, float thr) {
  const float dt = __fadd_rn(fmaxf(f.t1, 0.f), fminf(f.t2, 0.f));
  return __fmaf_rn(dt, dt, hh) < thr;
}

__device__ __forceinline__ bool near_pair(const Panel<float>& p, float x, float y, float near2) {
  const Frame<float> f = frame_rn(p.ax, p.ay, p.tx, p.ty, p.L, x, y);
  return near_test(f, __fmul_rn(f.h, f.h), near_thr(p.L, near2));
}

// Axis-aligned box (xmin, ymin, xmax, ymax) around every point whose pair
// with the panel near_test can call near: the segment grown by
// near_factor L, plus a margin far above the rounding of the frame.  A
// block of points whose box misses it has no near pair with the panel.
__device__ __forceinline__ float4 near_zone(const Panel<float>& p, float nfac) {
  const float R = fmaf(nfac * p.L, 1.001f, 1e-5f);
  const float bx = fmaf(p.L, p.tx, p.ax), by = fmaf(p.L, p.ty, p.ay);
  return make_float4(fminf(p.ax, bx) - R, fminf(p.ay, by) - R, fmaxf(p.ax, bx) + R,
                     fmaxf(p.ay, by) + R);
}

__device__ __forceinline__ bool boxes_meet(float4 a, float4 b) {
  return a.x <= b.z && b.x <= a.z && a.y <= b.w && b.y <= a.w;
}

// Bounding box of the points (x, y) held by the threads of a block of
// blockDim.x = 32 * nw threads (dead threads pass live = false); red: 4 nw floats
// of shared memory.  Every thread receives the box.  An empty set gives
// (+inf, +inf, -inf, -inf), which meets no box.
__device__ __forceinline__ float4 block_bbox(float x0, float y0, float x1, float y1, bool live,
                                             float* red) {
  float4 b = live ? make_float4(x0, y0, x1, y1)
                  : make_float4(__int_as_float(0x7f800000), __int_as_float(0x7f800000),
                                __int_as_float(0xff800000), __int_as_float(0xff800000));
  for (int o = 16; o; o >>= 1) {
    b.x = fminf(b.x, __shfl_xor_sync(0xffffffffu, b.x, o));
    b.y = fminf(b.y, __shfl_xor_sync(0xffffffffu, b.y, o));
    b.z = fmaxf(b.z, __shfl_xor_sync(0xffffffffu, b.z, o));
    b.w = fmaxf(b.w, __shfl_xor_sync(0xffffffffu, b.w, o));
  }
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[4 * w] = b.x; red[4 * w + 1] = b.y; red[4 * w + 2] = b.z; red[4 * w + 3] = b.w;
  }
  __syncthreads();
  b = make_float4(red[0], red[1], red[2], red[3]);
  for (int k = 1; k < nw; ++k) {
    b.x = fminf(b.x, red[4 * k]); b.y = fminf(b.y, red[4 * k + 1]);
    b.z = fmaxf(b.z, red[4 * k + 2]); b.w = fmaxf(b.w, red[4 * k + 3]);
  }
  return b;
}

// A float panel as the forward loops stage it in shared memory, with the
// constants of the layer integrals folded into the jumps:
//   wd' = w_d/(2 pi), wc' = -w_c/(2 pi), thr = near_thr(L, near_factor^2)
// so that -w_d Dl + w_c S = wd' Dh + wc' Sh with Dh, Sh of pair_fwd_f.
struct __align__(16) PanelF {
  float ax, ay, tx, ty;
  float L, thr, wd0, wd1;
  float wd2, wc0, wc1, wc2;
};

__device__ __forceinline__ PanelF stage_panel(const Panel<float>& p, float near2) {
  constexpr float k = 0.159154943f;   // 1/(2 pi)
  PanelF s;
  s.ax = p.ax; s.ay = p.ay; s.tx = p.tx; s.ty = p.ty;
  s.L = p.L;
  s.thr = near_thr(p.L, near2);
  s.wd0 = p.wd[0] * k; s.wd1 = p.wd[1] * k; s.wd2 = p.wd[2] * k;
  s.wc0 = -p.wc[0] * k; s.wc1 = -p.wc[1] * k; s.wc2 = -p.wc[2] * k;
  return s;
}

// One regularised layer pair: S with eps_c, Dl with eps_d.
template <typename T>
struct LayerVals {
  T S, Dl;
};

// Values only (forward evaluation).
template <typename T>
__device__ __forceinline__ LayerVals<T> layer_values(const Frame<T>& f, T eps_c2, T eps_d2,
                                                     bool same_eps) {
  LayerVals<T> v;
  T hc2 = f.h * f.h + eps_c2;
  T hc = m_sqrt(hc2);
  T tt = f.t1 * f.t2;
  T q1 = f.t1 * f.t1 + hc2;
  T q2 = f.t2 * f.t2 + hc2;
  T phic = m_atan2(hc * f.L, hc2 + tt);
  T lg2 = m_log(q2);
  T lp = m_log1p(f.L * (f.t1 + f.t2) / q1);
  v.S = -(f.L * (lg2 - T(2)) + f.t1 * lp + T(2) * hc * phic) * T(kInv4Pi);
  if (same_eps) {
    v.Dl = -(f.h / hc) * phic * T(kInv2Pi);
  } else {
    T hd2 = f.h * f.h + eps_d2;
    T hd = m_sqrt(hd2);
    T phid = m_atan2(hd * f.L, hd2 + tt);
    v.Dl = -(f.h / hd) * phid * T(kInv2Pi);
  }
  return v;
}

// Forward pair of the float loops, with the layer constants taken out
// (multiplied by -2 pi) so that they fold into the staged jumps of PanelF:
//   Dh = (h/h'_d) Phi_d                                        = -2 pi Dl
//   Sh = (1/2)(t2 log q2 - t1 log q1) - L + h'_c Phi_c          = -2 pi S
// hh = h*h.  Own arctangent (fastmath.cuh), both logarithms by the MUFU
// base-2 logarithm, one rsqrt for both h' and h/h'.  The difference of the
// two log terms loses to cancellation when t1 and t2 are far larger than L,
// but only about one float ulp of |t log q| (q <= 2 on the unit square)
// in absolute terms; pairs close to the panel, where it would matter
// relative to the value, are the near pairs evaluated in double.
__device__ __forceinline__ void pair_fwd_f(const Frame<float>& f, float hh, float eps_c2,
                                           float eps_d2, bool same_eps, float& Dh, float& Sh) {
  const float hc2 = hh + eps_c2;
  const float rc = mufu_rsqrt(hc2);
  const float hc = hc2 * rc;
  const float tt = f.t1 * f.t2;
  const float q1 = fmaf(f.t1, f.t1, hc2);
  const float q2 = fmaf(f.t2, f.t2, hc2);
  const float phic = fm_atan2_ypos(hc * f.L, hc2 + tt);
  const float d = fmaf(f.t2, mufu_lg2(q2), -f.t1 * mufu_lg2(q1));   // t2 lg q2 - t1 lg q1
  Sh = fmaf(hc, phic, fmaf(d, kLn2Halff, -f.L));
  if (same_eps) {
    Dh = f.h * rc * phic;
  } else {
    const float hd2 = hh + eps_d2;
    const float rd = mufu_rsqrt(hd2);
    Dh = f.h * rd * fm_atan2_ypos(hd2 * rd * f.L, hd2 + tt);
  }
}

// Values and frame partials of both layers.
template <typename T>
struct LayerGrad {
  T S, Dl;
  T S_t1, S_t2, S_h;
  T D_t1, D_t2, D_h;
};

template <typename T>
__device__ __forceinline__ LayerGrad<T> layer_grad(const Frame<T>& f, T eps_c2, T eps_d2,
                                                   bool same_eps) {
  LayerGrad<T> g;
  T tt = f.t1 * f.t2;
  T hh = f.h * f.h;
  // single layer, eps_c
  T hc2 = hh + eps_c2;
  T hc = m_sqrt(hc2);
  T q1 = f.t1 * f.t1 + hc2;
  T q2 = f.t2 * f.t2 + hc2;
  T phic = m_atan2(hc * f.L, hc2 + tt);
  T lg2 = m_log(q2);
  T lp = m_log1p(f.L * (f.t1 + f.t2) / q1);
  T lg1 = lg2 - lp;
  T hoc = f.h / hc;
  g.S = -(f.L * (lg2 - T(2)) + f.t1 * lp + T(2) * hc * phic) * T(kInv4Pi);
  g.S_t1 = lg1 * T(kInv4Pi);
  g.S_t2 = -lg2 * T(kInv4Pi);
  g.S_h = -hoc * phic * T(kInv2Pi);
  // double layer, eps_d
  T hd2, hd, phid, r1, r2;
  if (same_eps) {
    hd2 = hc2; hd = hc; phid = phic; r1 = q1; r2 = q2;
  } else {
    hd2 = hh + eps_d2;
    hd = m_sqrt(hd2);
    phid = m_atan2(hd * f.L, hd2 + tt);
    r1 = f.t1 * f.t1 + hd2;
    r2 = f.t2 * f.t2 + hd2;
  }
  T ir1 = T(1) / r1, ir2 = T(1) / r2;
  T ihd = T(1) / hd;
  g.Dl = -(f.h * ihd) * phid * T(kInv2Pi);
  g.D_t1 = f.h * ir1 * T(kInv2Pi);
  g.D_t2 = -f.h * ir2 * T(kInv2Pi);
  g.D_h = -(eps_d2 * phid * ihd - hh * f.L * (hd2 - tt) * ir1 * ir2) * (ihd * ihd) * T(kInv2Pi);
  return g;
}

// Values and frame partials of the float loops, each multiplied by -2 pi
// (the factor is applied once to the sums the loops accumulate):
//   S   = Sh of pair_fwd_f          D   = (h/h'_d) Phi_d
//   St1 = -(1/2) log q1             Dt1 = -h/q1
//   St2 =  (1/2) log q2             Dt2 =  h/q2
//   Sh_ = (h/h'_c) Phi_c            Dh_ = (1/h'^2)[eps_d^2 Phi_d/h' - h^2 L (h'^2 - t1 t2)/(q1 q2)]
// with both logarithms from the MUFU base-2 logarithm (mufu_lg2).
struct GradHat {
  float S, D;
  float St1, St2, Sh;
  float Dt1, Dt2, Dh;
};

__device__ __forceinline__ GradHat layer_grad_hat(const Frame<float>& f, float hh, float eps_c2,
                                                  float eps_d2, bool same_eps) {
  GradHat g;
  const float tt = f.t1 * f.t2;
  const float hc2 = hh + eps_c2;
  const float rc = mufu_rsqrt(hc2);
  const float hc = hc2 * rc;
  const float q1 = fmaf(f.t1, f.t1, hc2);
  const float q2 = fmaf(f.t2, f.t2, hc2);
  const float phic = fm_atan2_ypos(hc * f.L, hc2 + tt);
  const float lq1h = mufu_lg2(q1) * kLn2Halff;                 // (1/2) log q1
  const float lq2h = mufu_lg2(q2) * kLn2Halff;                 // (1/2) log q2
  g.S = fmaf(hc, phic, fmaf(f.t2, lq2h, fmaf(-f.t1, lq1h, -f.L)));
  g.St1 = -lq1h;
  g.St2 = lq2h;
  g.Sh = f.h * rc * phic;
  float hd2, rd, phid, r1, r2;
  if (same_eps) {
    hd2 = hc2; rd = rc; phid = phic; r1 = q1; r2 = q2;
    g.D = g.Sh;
  } else {
    hd2 = hh + eps_d2;
    rd = mufu_rsqrt(hd2);
    phid = fm_atan2_ypos(hd2 * rd * f.L, hd2 + tt);
    r1 = fmaf(f.t1, f.t1, hd2);
    r2 = fmaf(f.t2, f.t2, hd2);
    g.D = f.h * rd * phid;
  }
  const float ir1 = mufu_rcp(r1), ir2 = mufu_rcp(r2);
  g.Dt1 = -f.h * ir1;
  g.Dt2 = f.h * ir2;
  g.Dh = (eps_d2 * phid * rd - hh * f.L * (hd2 - tt) * ir1 * ir2) * (rd * rd);
  return g;
}

// Chain rule from frame partials (F_t1, F_t2, F_h) to d/da, d/db, out =
// (dF/dax, dF/day, dF/dbx, dF/dby).  iL = 1/L, or 0 for a zero-length panel
// (whose tangent is 0 too), which makes all four vanish without a branch.
template <typename T>
__device__ __forceinline__ void chain_endpoints(T tx, T ty, T iL, const Frame<T>& f, T Ft1, T Ft2,
                                                T Fh, T (&out)[4]) {
  const T s = f.h * (Ft1 + Ft2) * iL;
  const T na = fma(f.t2 * iL, Fh, -s);
  const T nb = fma(-f.t1 * iL, Fh, s);
  out[0] = fma(na, ty, Ft1 * tx);
  out[1] = fma(-na, tx, Ft1 * ty);
  out[2] = fma(nb, ty, Ft2 * tx);
  out[3] = fma(-nb, tx, Ft2 * ty);
}

// 1/L of a panel, 0 for a zero-length one (the float path with the MUFU reciprocal)
template <typename T>
__device__ __forceinline__ T inv_len(T L) {
  if constexpr (sizeof(T) == 4) {
    return L > 0.f ? mufu_rcp(L) : 0.f;
  } else {
    return L > T(0) ? T(1) / L : T(0);
  }
}

// Signed angle subtended at (x,y) by the segment a->b:
// atan2((a-x) x (b-x), (a-x).(b-x)).  The unregularised double-layer integral
// of a boundary segment is -phi/(2 pi) (Eq. (fundsol)).
template <typename T>
__device__ __forceinline__ T seg_angle(T ax, T ay, T bx, T by, T x, T y) {
  T dax = ax - x, day = ay - y, dbx = bx - x, dby = by - y;
  return m_atan2(dax * dby - day * dbx, dax * dbx + day * dby);
}
template <>
__device__ __forceinline__ float seg_angle<float>(float ax, float ay, float bx, float by, float x,
                                                  float y) {
  float dax = ax - x, day = ay - y, dbx = bx - x, dby = by - y;
  return fm_atan2(dax * dby - day * dbx, dax * dbx + day * dby);
}

}  // namespace bem
