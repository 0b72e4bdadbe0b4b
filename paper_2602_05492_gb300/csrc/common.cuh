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
// t2 log q2 - t1 log q1 is evaluated as L log q2 + t1 log1p(L (t1+t2)/q1),
// which has no cancellation when the panel is far from x (t1 ~ t2); this is
// what keeps single precision accurate in the far field.
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

// One straight panel as the kernels stage it (12 words).
template <typename T>
struct Panel {
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

// Near-field test of the mixed-precision path: the distance from x to the
// panel segment is below near_factor * L (compared squared).  The frame is
// recomputed here with explicitly rounded operations so that every kernel
// (the float main loops that skip these pairs and the double near-field
// kernels that take them) reaches the same decision bit for bit.
__device__ __forceinline__ bool near_pair(const Panel<float>& p, float x, float y, float near2) {
  const float dax = __fsub_rn(p.ax, x), day = __fsub_rn(p.ay, y);
  const float t1 = __fmaf_rn(dax, p.tx, __fmul_rn(day, p.ty));
  const float h = __fmaf_rn(dax, p.ty, -__fmul_rn(day, p.tx));
  const float t2 = __fadd_rn(t1, p.L);
  const float dt = t1 > 0.f ? t1 : (t2 < 0.f ? t2 : 0.f);
  const float d2 = __fmaf_rn(dt, dt, __fmul_rn(h, h));
  return d2 < __fmul_rn(near2, __fmul_rn(p.L, p.L));
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

// Float versions: own transcendentals (fastmath.cuh), one rsqrt for both
// h' and h/h', approximate divisions.
template <>
__device__ __forceinline__ LayerVals<float> layer_values<float>(const Frame<float>& f, float eps_c2,
                                                               float eps_d2, bool same_eps) {
  LayerVals<float> v;
  const float hh = f.h * f.h;
  const float hc2 = hh + eps_c2;
  const float rc = rsqrtf(hc2);
  const float hc = hc2 * rc;
  const float tt = f.t1 * f.t2;
  const float q1 = fmaf(f.t1, f.t1, hc2);
  const float q2 = fmaf(f.t2, f.t2, hc2);
  const float phic = fm_atan2(hc * f.L, hc2 + tt);
  const float lg2 = fm_log(q2);
  const float lp = fm_log1p(__fdividef(f.L * (f.t1 + f.t2), q1));
  v.S = -(f.L * (lg2 - 2.f) + f.t1 * lp + 2.f * hc * phic) * float(kInv4Pi);
  if (same_eps) {
    v.Dl = -(f.h * rc) * phic * float(kInv2Pi);
  } else {
    const float hd2 = hh + eps_d2;
    const float rd = rsqrtf(hd2);
    const float phid = fm_atan2(hd2 * rd * f.L, hd2 + tt);
    v.Dl = -(f.h * rd) * phid * float(kInv2Pi);
  }
  return v;
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

template <>
__device__ __forceinline__ LayerGrad<float> layer_grad<float>(const Frame<float>& f, float eps_c2,
                                                             float eps_d2, bool same_eps) {
  LayerGrad<float> g;
  const float tt = f.t1 * f.t2;
  const float hh = f.h * f.h;
  const float hc2 = hh + eps_c2;
  const float rc = rsqrtf(hc2);
  const float hc = hc2 * rc;
  const float q1 = fmaf(f.t1, f.t1, hc2);
  const float q2 = fmaf(f.t2, f.t2, hc2);
  const float phic = fm_atan2(hc * f.L, hc2 + tt);
  const float lg2 = fm_log(q2);
  const float lp = fm_log1p(__fdividef(f.L * (f.t1 + f.t2), q1));
  const float lg1 = lg2 - lp;
  g.S = -(f.L * (lg2 - 2.f) + f.t1 * lp + 2.f * hc * phic) * float(kInv4Pi);
  g.S_t1 = lg1 * float(kInv4Pi);
  g.S_t2 = -lg2 * float(kInv4Pi);
  g.S_h = -(f.h * rc) * phic * float(kInv2Pi);
  float hd2, rd, phid, r1, r2;
  if (same_eps) {
    hd2 = hc2; rd = rc; phid = phic; r1 = q1; r2 = q2;
  } else {
    hd2 = hh + eps_d2;
    rd = rsqrtf(hd2);
    phid = fm_atan2(hd2 * rd * f.L, hd2 + tt);
    r1 = fmaf(f.t1, f.t1, hd2);
    r2 = fmaf(f.t2, f.t2, hd2);
  }
  const float ir1 = __fdividef(1.f, r1), ir2 = __fdividef(1.f, r2);
  g.Dl = -(f.h * rd) * phid * float(kInv2Pi);
  g.D_t1 = f.h * ir1 * float(kInv2Pi);
  g.D_t2 = -f.h * ir2 * float(kInv2Pi);
  g.D_h = -(eps_d2 * phid * rd - hh * f.L * (hd2 - tt) * ir1 * ir2) * (rd * rd) * float(kInv2Pi);
  return g;
}

// Chain rule from frame partials (F_t1, F_t2, F_h) to d/da, d/db.
template <typename T>
__device__ __forceinline__ void frame_to_endpoints(const Panel<T>& p, const Frame<T>& f, T Ft1,
                                                   T Ft2, T Fh, T& dax, T& day, T& dbx, T& dby) {
  T iL = T(1) / f.L;
  T s = f.h * (Ft1 + Ft2) * iL;
  T na = -s + f.t2 * iL * Fh;
  T nb = s - f.t1 * iL * Fh;
  // n = (ty, -tx)
  dax = Ft1 * p.tx + na * p.ty;
  day = Ft1 * p.ty - na * p.tx;
  dbx = Ft2 * p.tx + nb * p.ty;
  dby = Ft2 * p.ty - nb * p.tx;
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
