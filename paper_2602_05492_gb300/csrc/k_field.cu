// Forward evaluation (Sec. 3.1.3, Eq. (bie) with alpha = 1):
//   u(x) = mean + sum_j phi_j(x)/(2 pi) u_b,j + sum_p [ -w_d,p Dl_p(x) + w_c,p S_p(x) ]
// One thread per point; panels (and boundary vertices) are staged block-wide
// in shared memory and broadcast to every warp.  In mixed precision the
// pair terms are float; pairs closer than near_factor panel lengths are
// skipped here and their double sum (k_near.cu) is added per point.
#include <algorithm>
#include <cmath>

#include "ctx.h"
#include "field_args.cuh"

namespace bem {

constexpr int kFB = 128;   // threads per block = panels per shared-memory tile

// Sum over one shared-memory tile of panels (double path).
template <typename T, bool SAME>
__device__ __forceinline__ void tile_accum(const Panel<T>* tile, int cnt, T x, T y,
                                           const FieldArgs<T>& a, T& s0, T& s1, T& s2) {
  for (int k = 0; k < cnt; ++k) {
    const Panel<T>& p = tile[k];
    Frame<T> f = frame(p, x, y);
    LayerVals<T> v = layer_values(f, a.ec2, a.ed2, SAME);
    s0 += -p.wd[0] * v.Dl + p.wc[0] * v.S;
    s1 += -p.wd[1] * v.Dl + p.wc[1] * v.S;
    s2 += -p.wd[2] * v.Dl + p.wc[2] * v.S;
  }
}

// Colour, residual and the block's loss partial from the handle sum s and the
// boundary angle sum b (without its 1/(2 pi)).
template <typename T>
__device__ __forceinline__ void field_epilogue(const FieldArgs<T>& a, int64_t i, bool live, T s0,
                                               T s1, T s2, T b0, T b1, T b2, double* red) {
  const int tid = threadIdx.x;
  double u0 = a.mean0 + double(b0) * kInv2Pi + double(s0);
  double u1 = a.mean1 + double(b1) * kInv2Pi + double(s1);
  double u2 = a.mean2 + double(b2) * kInv2Pi + double(s2);
  if (a.near_add && live) {
    u0 += a.near_add[3 * i];
    u1 += a.near_add[3 * i + 1];
    u2 += a.near_add[3 * i + 2];
  }
  double r2 = 0.0;
  if (live) {
    if (a.out) {
      a.out[3 * i] = T(u0);
      a.out[3 * i + 1] = T(u1);
      a.out[3 * i + 2] = T(u2);
    }
    if (a.target) {
      double r0 = u0 - fmin(double(a.target[3 * i]), 1.0);
      double r1 = u1 - fmin(double(a.target[3 * i + 1]), 1.0);
      double rr = u2 - fmin(double(a.target[3 * i + 2]), 1.0);
      if (a.resid) {
        a.resid[3 * i] = T(r0);
        a.resid[3 * i + 1] = T(r1);
        a.resid[3 * i + 2] = T(rr);
      }
      r2 = r0 * r0 + r1 * r1 + rr * rr;
    }
  }
  if (a.loss_part) {
    for (int o = 16; o; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);
    if ((tid & 31) == 0) red[tid >> 5] = r2;
    __syncthreads();
    if (tid == 0) {
      double s = 0;
      for (int w = 0; w < kFB / 32; ++w) s += red[w];
      a.loss_part[blockIdx.x] = s;
    }
  }
}

template <typename T, bool SAME>
__global__ void __launch_bounds__(kFB) k_field(FieldArgs<T> a) {
  __shared__ Panel<T> tile[kFB];
  __shared__ T sv[2 * (kFB + 1)];
  __shared__ T su[3 * kFB];
  __shared__ double red[kFB / 32];
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * kFB + tid;
  const bool live = i < a.n;
  T x = T(0.5), y = T(0.5);
  if (live) { x = a.xy[2 * i]; y = a.xy[2 * i + 1]; }
  T s0 = 0, s1 = 0, s2 = 0;
  const int p0 = a.split_out ? blockIdx.y * a.pchunk : 0;
  const int p1 = a.split_out ? min(a.P, p0 + a.pchunk) : a.P;
  for (int base = p0; base < p1; base += kFB) {
    __syncthreads();
    if (base + tid < p1) tile[tid] = a.pan[base + tid];
    __syncthreads();
    tile_accum<T, SAME>(tile, min(kFB, p1 - base), x, y, a, s0, s1, s2);
  }
  if (a.split_out) {
    if (live) {
      double* o = a.split_out + ((size_t)blockIdx.y * a.n + i) * 3;
      o[0] = double(s0);
      o[1] = double(s1);
      o[2] = double(s2);
    }
    return;
  }
  // boundary double layer with the (double) boundary solution
  T b0 = 0, b1 = 0, b2 = 0;
  if (a.ub) {
    for (int base = 0; base < a.Nb; base += kFB) {
      __syncthreads();
      int cnt = min(kFB, a.Nb - base);
      if (tid < cnt) {
        sv[2 * tid] = a.vert[2 * (base + tid)];
        sv[2 * tid + 1] = a.vert[2 * (base + tid) + 1];
        su[3 * tid] = T(a.ub[3 * (base + tid)]);
        su[3 * tid + 1] = T(a.ub[3 * (base + tid) + 1]);
        su[3 * tid + 2] = T(a.ub[3 * (base + tid) + 2]);
      }
      if (tid == 0) {
        sv[2 * cnt] = a.vert[2 * (base + cnt)];
        sv[2 * cnt + 1] = a.vert[2 * (base + cnt) + 1];
      }
      __syncthreads();
      for (int k = 0; k < cnt; ++k) {
        T phi = seg_angle(sv[2 * k], sv[2 * k + 1], sv[2 * k + 2], sv[2 * k + 3], x, y);
        b0 += phi * su[3 * k];
        b1 += phi * su[3 * k + 1];
        b2 += phi * su[3 * k + 2];
      }
    }
  }
  field_epilogue<T>(a, i, live, s0, s1, s2, b0, b1, b2, red);
}

// Float kernel of the mixed path.  Panels are staged as PanelF (three
// 128-bit shared-memory loads per panel, the layer constants folded into the
// jumps); one rounded frame per pair serves the near-field test and the layer
// formulas.  With NEAR, each tile puts first the panels whose near zone meets
// the block's bounding box; only those pairs take the near test, the rest
// cannot be near.  The boundary vertices are walked in order so that each
// vertex offset is formed once.
template <bool SAME>
__device__ __forceinline__ void pair_acc_f(const float4 A, const float4 B, const float4 C,
                                           const Frame<float>& f, float hh, float ec2, float ed2,
                                           float& s0, float& s1, float& s2) {
  // A = (ax, ay, tx, ty), B = (L, thr, wd0', wd1'), C = (wd2', wc0', wc1', wc2')
  float Dh, Sh;
  pair_fwd_f(f, hh, ec2, ed2, SAME, Dh, Sh);
  s0 = fmaf(B.z, Dh, fmaf(C.y, Sh, s0));
  s1 = fmaf(B.w, Dh, fmaf(C.z, Sh, s1));
  s2 = fmaf(C.x, Dh, fmaf(C.w, Sh, s2));
}

// Shared memory of one CTA of the float field kernels.
struct FieldSmemF {
  float4 tile[3 * kFB];
  float2 sv[kFB + 1];
  float4 su[kFB];
  double red[kFB / 32];
  float bred[4 * (kFB / 32)];
  int wcnt[kFB / 32];
};

// Handle sums of the points of a tile against the panels [p0, p1) of pan,
// added into s: the panels staged as PanelF kFB at a time; with NEAR, each
// staged tile puts first the panels whose near zone meets the block's
// bounding box bb, and only those pairs take the near test.  Every CTA-wide
// barrier is reached by all threads.
template <bool SAME, bool NEAR, int SPT>
__device__ __forceinline__ void tile_handle_sums(const FieldArgs<float>& a,
                                                 const Panel<float>* __restrict__ pan, int p0,
                                                 int p1, const float (&x)[SPT],
                                                 const float (&y)[SPT], float4 bb,
                                                 float (&s)[SPT][3], FieldSmemF& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int base = p0; base < p1; base += kFB) {
    const int cnt = min(kFB, p1 - base);
    int nf = 0;   // panels [0, nf) of the tile may have near pairs
    __syncthreads();
    if constexpr (NEAR) {
      Panel<float> p{};
      bool cand = false;
      if (tid < cnt) {
        p = pan[base + tid];
        cand = boxes_meet(near_zone(p, a.nfac), bb);
      }
      const unsigned m = __ballot_sync(0xffffffffu, cand);
      if (lane == 0) sm.wcnt[warp] = __popc(m);
      __syncthreads();
      int before = 0;
#pragma unroll
      for (int w = 0; w < kFB / 32; ++w) {
        before += w < warp ? sm.wcnt[w] : 0;
        nf += sm.wcnt[w];
      }
      if (tid < cnt) {
        const int below = __popc(m & ((1u << lane) - 1u));
        const int slot = cand ? before + below : nf + (warp * 32 - before) + (lane - below);
        reinterpret_cast<PanelF*>(sm.tile)[slot] = stage_panel(p, a.near2);
      }
    } else {
      if (tid < cnt) reinterpret_cast<PanelF*>(sm.tile)[tid] = stage_panel(pan[base + tid], 0.f);
    }
    __syncthreads();
    for (int k = 0; k < nf; ++k) {
      const float4 A = sm.tile[3 * k], B = sm.tile[3 * k + 1], C = sm.tile[3 * k + 2];
#pragma unroll
      for (int q = 0; q < SPT; ++q) {
        const Frame<float> f = frame_rn(A.x, A.y, A.z, A.w, B.x, x[q], y[q]);
        const float hh = __fmul_rn(f.h, f.h);
        if (!near_test(f, hh, B.y))
          pair_acc_f<SAME>(A, B, C, f, hh, a.ec2, a.ed2, s[q][0], s[q][1], s[q][2]);
      }
    }
    for (int k = nf; k < cnt; ++k) {
      const float4 A = sm.tile[3 * k], B = sm.tile[3 * k + 1], C = sm.tile[3 * k + 2];
#pragma unroll
      for (int q = 0; q < SPT; ++q) {
        const Frame<float> f = frame_rn(A.x, A.y, A.z, A.w, B.x, x[q], y[q]);
        pair_acc_f<SAME>(A, B, C, f, f.h * f.h, a.ec2, a.ed2, s[q][0], s[q][1], s[q][2]);
      }
    }
  }
}

// Boundary angle sums of the points of a tile for NT boundary solutions at
// once: b[t][q][c] += phi_j(x_q) u_t[j][c] over the segments j (without the
// 1/(2 pi)).  The angle of a segment does not depend on the handles, so the
// trials of one LM step share it.  su holds kFB entries per solution.
template <int SPT, int NT>
__device__ __forceinline__ void tile_boundary_sums(const float* __restrict__ vert, int Nb,
                                                   const double* const (&ub)[NT],
                                                   const float (&x)[SPT], const float (&y)[SPT],
                                                   float (&b)[NT][SPT][3], float2* sv, float4* su) {
  const int tid = threadIdx.x;
  for (int base = 0; base < Nb; base += kFB) {
    __syncthreads();
    const int cnt = min(kFB, Nb - base);
    if (tid < cnt) {
      const int j = base + tid;
      sv[tid] = make_float2(vert[2 * j], vert[2 * j + 1]);
#pragma unroll
      for (int t = 0; t < NT; ++t)
        su[t * kFB + tid] = make_float4(float(ub[t][3 * j]), float(ub[t][3 * j + 1]),
                                        float(ub[t][3 * j + 2]), 0.f);
    }
    if (tid == 0) sv[cnt] = make_float2(vert[2 * (base + cnt)], vert[2 * (base + cnt) + 1]);
    __syncthreads();
    float dax[SPT], day[SPT];
#pragma unroll
    for (int q = 0; q < SPT; ++q) { dax[q] = sv[0].x - x[q]; day[q] = sv[0].y - y[q]; }
    for (int k = 0; k < cnt; ++k) {
      const float2 w = sv[k + 1];
#pragma unroll
      for (int q = 0; q < SPT; ++q) {
        const float dbx = w.x - x[q], dby = w.y - y[q];
        const float phi = fm_atan2(dax[q] * dby - day[q] * dbx, dax[q] * dbx + day[q] * dby);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const float4 u = su[t * kFB + k];
          b[t][q][0] = fmaf(phi, u.x, b[t][q][0]);
          b[t][q][1] = fmaf(phi, u.y, b[t][q][1]);
          b[t][q][2] = fmaf(phi, u.z, b[t][q][2]);
        }
        dax[q] = dbx;
        day[q] = dby;
      }
    }
  }
}

// Colour, residual and the tile's loss partial (loss_part[tile]) from the
// handle sums s, the boundary angle sums b and the double near-field sums
// near_add (or null).
template <int SPT>
__device__ __forceinline__ void tile_finish(const FieldArgs<float>& a, int64_t tile,
                                            const int64_t (&i)[SPT], const bool (&live)[SPT],
                                            const float (&s)[SPT][3], const float (&b)[SPT][3],
                                            const double* __restrict__ near_add,
                                            double* __restrict__ loss_part, FieldSmemF& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double r2 = 0.0;
#pragma unroll
  for (int q = 0; q < SPT; ++q) {
    double u0 = a.mean0 + double(b[q][0]) * kInv2Pi + double(s[q][0]);
    double u1 = a.mean1 + double(b[q][1]) * kInv2Pi + double(s[q][1]);
    double u2 = a.mean2 + double(b[q][2]) * kInv2Pi + double(s[q][2]);
    if (!live[q]) continue;
    const int64_t ii = i[q];
    if (near_add) {
      u0 += near_add[3 * ii];
      u1 += near_add[3 * ii + 1];
      u2 += near_add[3 * ii + 2];
    }
    if (a.out) {
      a.out[3 * ii] = float(u0);
      a.out[3 * ii + 1] = float(u1);
      a.out[3 * ii + 2] = float(u2);
    }
    if (a.target) {
      const double r0 = u0 - fmin(double(a.target[3 * ii]), 1.0);
      const double r1 = u1 - fmin(double(a.target[3 * ii + 1]), 1.0);
      const double rr = u2 - fmin(double(a.target[3 * ii + 2]), 1.0);
      if (a.resid) {
        a.resid[3 * ii] = float(r0);
        a.resid[3 * ii + 1] = float(r1);
        a.resid[3 * ii + 2] = float(rr);
      }
      r2 += r0 * r0 + r1 * r1 + rr * rr;
    }
  }
  if (loss_part) {
    for (int o = 16; o; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);
    __syncthreads();
    if (lane == 0) sm.red[warp] = r2;
    __syncthreads();
    if (tid == 0) {
      double t = 0;
      for (int w = 0; w < kFB / 32; ++w) t += sm.red[w];
      loss_part[tile] = t;
    }
  }
}

// The points of tile `tile` (kFB * SPT of them, thread t owning points t,
// t + kFB, ...), their bounding box and their coordinates.
template <bool NEAR, int SPT>
__device__ __forceinline__ float4 tile_points(const FieldArgs<float>& a, int64_t tile,
                                              int64_t (&i)[SPT], bool (&live)[SPT], float (&x)[SPT],
                                              float (&y)[SPT], FieldSmemF& sm) {
  const int tid = threadIdx.x;
  float x0 = __int_as_float(0x7f800000), y0 = x0, x1 = -x0, y1 = -x0;
  bool any = false;
#pragma unroll
  for (int k = 0; k < SPT; ++k) {
    i[k] = tile * (kFB * SPT) + k * kFB + tid;
    live[k] = i[k] < a.n;
    x[k] = 0.5f; y[k] = 0.5f;
    if (live[k]) {
      x[k] = a.xy[2 * i[k]];
      y[k] = a.xy[2 * i[k] + 1];
      x0 = fminf(x0, x[k]); y0 = fminf(y0, y[k]); x1 = fmaxf(x1, x[k]); y1 = fmaxf(y1, y[k]);
      any = true;
    }
  }
  float4 bb = make_float4(0.f, 0.f, 0.f, 0.f);
  if constexpr (NEAR) bb = block_bbox(x0, y0, x1, y1, any, sm.bred);
  return bb;
}

// One tile of kFB * SPT points: handle sums with near-zone culling, the
// boundary term and the epilogue (colour, residual, the tile's loss partial
// in loss_part[tile]).  `ys` is the panel slice in split mode.  Every
// CTA-wide barrier is reached by all threads.
template <bool SAME, bool NEAR, int SPT>
__device__ __forceinline__ void field_tile_f32(const FieldArgs<float>& a, int64_t tile, int ys,
                                               FieldSmemF& sm) {
  int64_t i[SPT];
  bool live[SPT];
  float x[SPT], y[SPT];
  const float4 bb = tile_points<NEAR, SPT>(a, tile, i, live, x, y, sm);
  float s[SPT][3];
#pragma unroll
  for (int k = 0; k < SPT; ++k) s[k][0] = s[k][1] = s[k][2] = 0.f;
  const int p0 = a.split_out ? ys * a.pchunk : 0;
  const int p1 = a.split_out ? min(a.P, p0 + a.pchunk) : a.P;
  tile_handle_sums<SAME, NEAR, SPT>(a, a.pan, p0, p1, x, y, bb, s, sm);
  if (a.split_out) {
#pragma unroll
    for (int q = 0; q < SPT; ++q)
      if (live[q]) {
        double* o = a.split_out + ((size_t)ys * a.n + i[q]) * 3;
        o[0] = double(s[q][0]);
        o[1] = double(s[q][1]);
        o[2] = double(s[q][2]);
      }
    return;
  }
  float b[1][SPT][3];
#pragma unroll
  for (int q = 0; q < SPT; ++q) b[0][q][0] = b[0][q][1] = b[0][q][2] = 0.f;
  if (a.ub) {
    const double* const ub[1] = {a.ub};
    tile_boundary_sums<SPT, 1>(a.vert, a.Nb, ub, x, y, b, sm.sv, sm.su);
  }
  tile_finish<SPT>(a, tile, i, live, s, b[0], a.near_add, a.loss_part, sm);
}

// Several damping trials of one scene on one tile: the points and their
// boundary angles once, then per trial the handle sums against that
// trial's panels and the epilogue with that trial's boundary solution,
// near-field sums and loss partials (j.tloss[t][tile]).
template <bool SAME, bool NEAR, int SPT, int NT>
__device__ __forceinline__ void field_tile_trials_f32(const BatchJob& j, int64_t tile,
                                                      FieldSmemF& sm, float4* su) {
  const FieldArgs<float>& a = j.a;
  int64_t i[SPT];
  bool live[SPT];
  float x[SPT], y[SPT];
  const float4 bb = tile_points<NEAR, SPT>(a, tile, i, live, x, y, sm);
  float b[NT][SPT][3];
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int q = 0; q < SPT; ++q) b[t][q][0] = b[t][q][1] = b[t][q][2] = 0.f;
  double const* ub[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) ub[t] = j.tub[t];
  tile_boundary_sums<SPT, NT>(a.vert, a.Nb, ub, x, y, b, sm.sv, su);
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    float s[SPT][3];
#pragma unroll
    for (int q = 0; q < SPT; ++q) s[q][0] = s[q][1] = s[q][2] = 0.f;
    tile_handle_sums<SAME, NEAR, SPT>(a, j.tpan[t], 0, a.P, x, y, bb, s, sm);
    tile_finish<SPT>(a, tile, i, live, s, b[t], j.tnear[t], j.tloss[t], sm);
  }
}

template <bool SAME, bool NEAR, int SPT>
__global__ void __launch_bounds__(kFB) k_field_f32(const __grid_constant__ FieldArgs<float> a) {
  __shared__ FieldSmemF sm;
  field_tile_f32<SAME, NEAR, SPT>(a, blockIdx.x, blockIdx.y, sm);
}

// points per thread of the float evaluation (split mode: 1)
constexpr int kSptEval = 2;

// Batched evaluation: one persistent launch over the 128 * SPT-point tiles
// of every job (a job = one scene at one parameter vector).  CTAs take tiles
// from a global counter; a tile's job is found by binary search over the
// jobs' first-tile offsets.  Each tile runs the same code as k_field_f32, so
// with SPT = 1 a scene's colours, residuals and loss partials are those of a
// single-scene evaluation bit for bit.
template <bool SAME, bool NEAR, int SPT, int NT>
__global__ void __launch_bounds__(kFB) k_field_batch_f32(const BatchJob* __restrict__ jobs, int njobs,
                                                         const int64_t* __restrict__ total_p,
                                                         unsigned long long* __restrict__ counter) {
  __shared__ FieldSmemF sm;
  __shared__ float4 su_more[NT > 1 ? NT * kFB : 1];   // boundary solutions of NT trials
  __shared__ int64_t item_s;
  const int64_t total = *total_p;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) item_s = (int64_t)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t item = item_s;
    if (item >= total) return;
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].tile0 <= item) lo = mid; else hi = mid - 1;
    }
    if constexpr (NT > 1)
      field_tile_trials_f32<SAME, NEAR, SPT, NT>(jobs[lo], item - jobs[lo].tile0, sm, su_more);
    else
      field_tile_f32<SAME, NEAR, SPT>(jobs[lo].a, item - jobs[lo].tile0, 0, sm);
  }
}

// sum of per-block partials in fixed order -> out[0]
__global__ void k_sum_fixed(const double* __restrict__ part, int64_t m, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0;
  // each thread sums a contiguous range so the order is fixed
  int64_t per = (m + blockDim.x - 1) / blockDim.x;
  int64_t b = threadIdx.x * per, e = b + per < m ? b + per : m;
  for (int64_t k = b; k < e; ++k) s += part[k];
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    *out = t;
  }
}

// f_b,i = |G_i| sum_q w_q f(x_iq) from split partials (+ near-field sums)
__global__ void k_rhs_reduce(const double* __restrict__ part, int nsplit, int Nb,
                             const double* __restrict__ vert, const double* __restrict__ near_add,
                             double* __restrict__ fb) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * Nb) return;
  int i = t / 3, c = t % 3;
  double ex = vert[2 * (i + 1)] - vert[2 * i], ey = vert[2 * (i + 1) + 1] - vert[2 * i + 1];
  double ell = sqrt(ex * ex + ey * ey);
  int64_t n = 3 * (int64_t)Nb;
  double s = 0;
  for (int q = 0; q < 3; ++q) {
    double f = 0;
    for (int sp = 0; sp < nsplit; ++sp) f += part[((size_t)sp * n + 3 * i + q) * 3 + c];
    if (near_add) f += near_add[(3 * i + q) * 3 + c];
    s += gauss_weight(q) * f;
  }
  fb[3 * i + c] = ell * s;
}

template <typename T>
__global__ void k_mean_part(const T* __restrict__ t, int64_t n, double* __restrict__ part) {
  __shared__ double red[3][32];
  double s[3] = {0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < 3; ++c) s[c] += fmin(double(t[3 * i + c]), 1.0);
  for (int c = 0; c < 3; ++c)
    for (int o = 16; o; o >>= 1) s[c] += __shfl_down_sync(0xffffffffu, s[c], o);
  if ((threadIdx.x & 31) == 0)
    for (int c = 0; c < 3; ++c) red[c][threadIdx.x >> 5] = s[c];
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) v += red[threadIdx.x][w];
    part[blockIdx.x * 3 + threadIdx.x] = v;
  }
}

// ---------------------------------------------------------------------------

template <typename T>
static FieldArgs<T> make_args(bem_ctx* c) {
  FieldArgs<T> a{};
  a.pan = (const Panel<T>*)(sizeof(T) == 8 ? (const void*)c->d_pan64 : (const void*)c->d_pan32);
  a.pan64 = c->d_pan64;
  a.P = c->sc.P;
  a.pchunk = c->sc.P;
  a.vert = (const T*)(sizeof(T) == 8 ? (const void*)c->bd.d_vert : (const void*)c->bd.d_vert32);
  a.Nb = c->bd.Nb;
  a.ec2 = T(c->opts.eps_c * c->opts.eps_c);
  a.ed2 = T(c->opts.eps_d * c->opts.eps_d);
  a.ec2d = c->opts.eps_c * c->opts.eps_c;
  a.ed2d = c->opts.eps_d * c->opts.eps_d;
  a.near2 = T(c->opts.near_factor * c->opts.near_factor);
  a.nfac = float(c->opts.near_factor);
  return a;
}

template <typename T>
static void launch_field(bem_ctx* c, const FieldArgs<T>& a, dim3 grid, const char* name = nullptr) {
  ProfScope _ps(c, name ? name : a.split_out ? "k_field_rhs" : "k_field");
  const bool same = c->opts.eps_c == c->opts.eps_d;
  if constexpr (sizeof(T) == 4) {
    const bool near = c->opts.near_factor > 0;
#define BEM_FIELD_F32(SPT_)                                                  \
  do {                                                                       \
    if (same) {                                                              \
      if (near) k_field_f32<true, true, SPT_><<<grid, kFB, 0, S(c)>>>(a);    \
      else k_field_f32<true, false, SPT_><<<grid, kFB, 0, S(c)>>>(a);        \
    } else {                                                                 \
      if (near) k_field_f32<false, true, SPT_><<<grid, kFB, 0, S(c)>>>(a);   \
      else k_field_f32<false, false, SPT_><<<grid, kFB, 0, S(c)>>>(a);       \
    }                                                                        \
  } while (0)
    if (a.split_out) BEM_FIELD_F32(1);
    else BEM_FIELD_F32(kSptEval);
#undef BEM_FIELD_F32
  } else {
    if (same) k_field<T, true><<<grid, kFB, 0, S(c)>>>(a);
    else k_field<T, false><<<grid, kFB, 0, S(c)>>>(a);
  }
  BEM_LAUNCHED(c);
}

template <typename T>
static int field_eval_t(bem_ctx* c, int64_t n, const void* xy, void* out, const void* target,
                        void* resid, bool want_loss) {
  int rc;
  FieldArgs<T> a = make_args<T>(c);
  a.xy = (const T*)xy;
  a.n = n;
  a.ub = c->d_ub;
  a.mean0 = c->mean[0]; a.mean1 = c->mean[1]; a.mean2 = c->mean[2];
  a.target = (const T*)target;
  a.out = (T*)out;
  a.resid = (T*)resid;
  const int64_t per_block = sizeof(T) == 4 ? (int64_t)kFB * kSptEval : kFB;
  int64_t nblk = (n + per_block - 1) / per_block;
  if (sizeof(T) == 4 && c->opts.near_factor > 0 && n > 0) {
    if ((rc = grow(c, c->nearF, sizeof(double) * 3 * (size_t)n))) return rc;
    if ((rc = near_forward(c, n, (const float*)xy, (double*)c->nearF.p))) return rc;
    a.near_add = (const double*)c->nearF.p;
  }
  if (want_loss) {
    if ((rc = grow(c, c->loss, sizeof(double) * (nblk + 1)))) return rc;
    a.loss_part = (double*)c->loss.p;
  }
  if (nblk > 0) launch_field<T>(c, a, dim3((unsigned)nblk));
  if (want_loss) {
    if (nblk > 0) {
      k_sum_fixed<<<1, 1024, 0, S(c)>>>(a.loss_part, nblk, c->d_scal);
      BEM_LAUNCHED(c);
    } else if ((rc = cuda_check(c, cudaMemsetAsync(c->d_scal, 0, 8, S(c)), "memset"))) {
      return rc;
    }
  }
  return cuda_check(c, cudaGetLastError(), "k_field");
}

FieldArgs<float> field_args_f32(bem_ctx* c) { return make_args<float>(c); }

int64_t field_blocks(int64_t m) { return (m + (int64_t)kFB * kSptEval - 1) / ((int64_t)kFB * kSptEval); }

int field_finish_hand(bem_ctx* c, int64_t m, const float* xy, const double* hand,
                      const float* target, float* resid, double* loss_part) {
  FieldArgs<float> a = make_args<float>(c);
  a.P = 0;                 // no panel loop: the handle term comes in as hand
  a.xy = xy;
  a.n = m;
  a.ub = c->d_ub;
  a.mean0 = c->mean[0]; a.mean1 = c->mean[1]; a.mean2 = c->mean[2];
  a.target = target;
  a.resid = resid;
  a.near_add = hand;
  a.loss_part = loss_part;
  const int64_t nblk = field_blocks(m);
  if (nblk > 0) launch_field<float>(c, a, dim3((unsigned)nblk), "k_field_bnd");
  return cuda_check(c, cudaGetLastError(), "k_field boundary");
}

int field_sum_loss(bem_ctx* c, const double* loss_part, int64_t nblk) {
  if (nblk <= 0) return cuda_check(c, cudaMemsetAsync(c->d_scal, 0, 8, S(c)), "memset");
  k_sum_fixed<<<1, 1024, 0, S(c)>>>(loss_part, nblk, c->d_scal);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "loss sum");
}

int field_batch_launch(bem_ctx* c, const BatchJob* jobs, int njobs, const int64_t* total_tiles,
                       unsigned long long* counter, int spt, int blocks_per_sm, int nt) {
  int rc;
  if ((rc = cuda_check(c, cudaMemsetAsync(counter, 0, sizeof(unsigned long long), S(c)), "memset")))
    return rc;
  const unsigned grid = (unsigned)std::max(1, c->sms * blocks_per_sm);
  const bool same = c->opts.eps_c == c->opts.eps_d, near = c->opts.near_factor > 0;
#define BEM_BATCH_LAUNCH(SM_, NR_, SPT_, NT_) \
  k_field_batch_f32<SM_, NR_, SPT_, NT_><<<grid, kFB, 0, S(c)>>>(jobs, njobs, total_tiles, counter)
#define BEM_BATCH_NT(SPT_, NT_)                                                                 \
  do {                                                                                          \
    if (same) { if (near) BEM_BATCH_LAUNCH(true, true, SPT_, NT_); else BEM_BATCH_LAUNCH(true, false, SPT_, NT_); } \
    else { if (near) BEM_BATCH_LAUNCH(false, true, SPT_, NT_); else BEM_BATCH_LAUNCH(false, false, SPT_, NT_); }   \
  } while (0)
  // trial jobs of 2 to kJobTrials trials per scene, or one evaluation per job
  if (nt == 4) { if (spt == 2) BEM_BATCH_NT(2, 4); else BEM_BATCH_NT(1, 4); }
  else if (nt == 3) { if (spt == 2) BEM_BATCH_NT(2, 3); else BEM_BATCH_NT(1, 3); }
  else if (nt == 2) { if (spt == 2) BEM_BATCH_NT(2, 2); else BEM_BATCH_NT(1, 2); }
  else { if (spt == 2) BEM_BATCH_NT(2, 1); else BEM_BATCH_NT(1, 1); }
#undef BEM_BATCH_NT
#undef BEM_BATCH_LAUNCH
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "k_field_batch_f32");
}

int field_eval(bem_ctx* c, int64_t n, const void* xy, void* out, const void* target, void* resid,
               bool want_loss) {
  if (c->opts.precision == BEM_FP64)
    return field_eval_t<double>(c, n, xy, out, target, resid, want_loss);
  return field_eval_t<float>(c, n, xy, out, target, resid, want_loss);
}

template <typename T>
static int field_rhs_t(bem_ctx* c) {
  int rc;
  int Nb = c->bd.Nb, P = c->sc.P;
  int64_t n = 3 * (int64_t)Nb;
  int nsplit = (P + kFB - 1) / kFB;
  if (nsplit > 64) nsplit = 64;
  int pchunk = ((P + nsplit - 1) / nsplit + kFB - 1) / kFB * kFB;
  nsplit = (P + pchunk - 1) / pchunk;
  if ((rc = grow(c, c->gpart, sizeof(double) * (size_t)nsplit * n * 3))) return rc;
  FieldArgs<T> a = make_args<T>(c);
  a.xy = (const T*)(sizeof(T) == 8 ? (const void*)c->bd.d_gp : (const void*)c->bd.d_gp32);
  a.n = n;
  a.pchunk = pchunk;
  a.split_out = (double*)c->gpart.p;
  launch_field<T>(c, a, dim3((unsigned)((n + kFB - 1) / kFB), nsplit));
  const double* near_add = nullptr;
  if (sizeof(T) == 4 && c->opts.near_factor > 0) {
    if ((rc = grow(c, c->nearF, sizeof(double) * 3 * (size_t)n))) return rc;
    if ((rc = near_forward(c, n, (const float*)a.xy, (double*)c->nearF.p))) return rc;
    near_add = (const double*)c->nearF.p;
  }
  k_rhs_reduce<<<(3 * Nb + 255) / 256, 256, 0, S(c)>>>(a.split_out, nsplit, Nb, c->bd.d_vert,
                                                        near_add, c->d_fb);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "rhs");
}

int field_rhs(bem_ctx* c) {
  if (c->opts.precision == BEM_FP64) return field_rhs_t<double>(c);
  return field_rhs_t<float>(c);
}

int field_solve(bem_ctx* c) {
  if (c->opts.precision == BEM_FP64) return la_apply3(c, c->bd.d_W, c->d_fb, c->d_ub);
  return la_apply3_refined(c, c->bd.d_W32, c->bd.d_A, c->d_fb, c->d_ub, false);
}

int field_sample_mean(bem_ctx* c, int64_t n, const void* target, double* host_mean) {
  int rc;
  const int nb = 256;
  if ((rc = grow(c, c->loss, sizeof(double) * 3 * nb))) return rc;
  double* part = (double*)c->loss.p;
  if (c->opts.precision == BEM_FP64)
    k_mean_part<double><<<nb, 256, 0, S(c)>>>((const double*)target, n, part);
  else
    k_mean_part<float><<<nb, 256, 0, S(c)>>>((const float*)target, n, part);
  BEM_LAUNCHED(c);
  double h[3 * nb];
  if ((rc = cuda_check(c, cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, S(c)),
                       "mean")))
    return rc;
  if ((rc = cuda_check(c, cudaStreamSynchronize(S(c)), "mean sync"))) return rc;
  for (int k = 0; k < 3; ++k) {
    double s = 0;
    for (int b = 0; b < nb; ++b) s += h[3 * b + k];
    host_mean[k] = n > 0 ? s / double(n) : 0.0;
  }
  return BEM_OK;
}

}  // namespace bem
