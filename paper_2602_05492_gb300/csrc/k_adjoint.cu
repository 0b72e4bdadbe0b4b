// Reverse-mode gradient of sum_s r_s . u(x_s) (Sec. 3.2, Eq. (diffbie)).
//
//   sum_s r_s.u(x_s) = sum_s r_s.f(x_s) + q^T u_b,      q_j = sum_s phi_j(x_s)/(2pi) r_s
//   u_b = A^+ f_b  =>  q^T u_b = lambda^T f_b,           lambda = (A^+)^T q
//   f_b,i = |G_i| sum_k w_k f(x_ik)
// so the gradient is the handle-term adjoint over the samples (weights r_s)
// plus the same adjoint over the boundary Gauss points (weights
// lambda_i |G_i| w_k).  Kernel values are recomputed, nothing of size
// samples x panels is stored.
//
// Per (point, panel) pair the weighted handle term is
//   F = alpha Dl + beta S,  alpha = -r.w_d, beta = r.w_c,
// and its endpoint gradient is assembled from five per-panel sums of frame
// partials (see common.cuh):
//   A1 = sum F_t1, A2 = sum F_t2, A3 = sum h (F_t1+F_t2), A5 = sum t1 F_h, A6 = sum F_h
//   dF/da = tau A1 + n (-A3 + A5 + L A6)/L,   dF/db = tau A2 + n (A3 - A5)/L
// plus the jump derivatives sum -r_c Dl and sum r_c S: 11 sums per panel.
// One thread owns one panel and walks the points of its block's chunk, so
// these sums stay in registers (no cross-thread reduction per pair).
#include <algorithm>
#include <cmath>

#include "ctx.h"

namespace bem {

constexpr int kVB = 128;     // threads per block (panels per block)
constexpr int kNP = 11;      // sums per panel

template <typename T>
struct VjpArgs {
  const T* xy;
  const T* w;          // weights [n][3]
  int64_t n;
  const Panel<T>* pan;
  const Panel<double>* pan64;
  int P;
  const T* vert;
  int Nb;              // boundary segments handled by the extra blocks (0 = none)
  T ec2, ed2;
  double ec2d, ed2d;
  T near2;
  float nfac;          // near_factor (float path)
  int64_t chunk;       // points per blockIdx.y
  double* part;        // [gridDim.y][P][11]
  double* qpart;       // [gridDim.y][Nb][3]
};

template <typename T>
struct Acc11 {
  T v[kNP];
};

template <typename T, bool SAME>
__device__ __forceinline__ void pair_adj(const Panel<T>& p, T x, T y, T r0, T r1, T r2, T ec2,
                                         T ed2, T* acc) {
  Frame<T> f = frame(p, x, y);
  LayerGrad<T> g = layer_grad(f, ec2, ed2, SAME);
  T al = -(r0 * p.wd[0] + r1 * p.wd[1] + r2 * p.wd[2]);
  T be = r0 * p.wc[0] + r1 * p.wc[1] + r2 * p.wc[2];
  T gt1 = al * g.D_t1 + be * g.S_t1;
  T gt2 = al * g.D_t2 + be * g.S_t2;
  T gh = al * g.D_h + be * g.S_h;
  acc[0] += gt1;
  acc[1] += gt2;
  acc[2] += f.h * (gt1 + gt2);
  acc[3] += f.t1 * gh;
  acc[4] += gh;
  acc[5] -= r0 * g.Dl;
  acc[6] -= r1 * g.Dl;
  acc[7] -= r2 * g.Dl;
  acc[8] += r0 * g.S;
  acc[9] += r1 * g.S;
  acc[10] += r2 * g.S;
}

template <typename T, bool SAME, bool NEAR>
__global__ void __launch_bounds__(kVB) k_vjp(VjpArgs<T> a) {
  __shared__ T sx[kVB], sy[kVB], sr[3 * kVB];
  const int tid = threadIdx.x;
  const int ptiles = (a.P + kVB - 1) / kVB;
  const bool is_pan = (int)blockIdx.x < ptiles;
  const int idx = is_pan ? blockIdx.x * kVB + tid : (blockIdx.x - ptiles) * kVB + tid;
  const bool live = is_pan ? idx < a.P : idx < a.Nb;
  const int64_t s0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t s1 = min(a.n, s0 + a.chunk);

  Panel<T> p{};
  Panel<double> pd{};
  T bax = 0, bay = 0, bbx = 0, bby = 0;
  if (live) {
    if (is_pan) {
      p = a.pan[idx];
      if (NEAR) pd = a.pan64[idx];
    } else {
      bax = a.vert[2 * idx]; bay = a.vert[2 * idx + 1];
      bbx = a.vert[2 * idx + 2]; bby = a.vert[2 * idx + 3];
    }
  }
  double tot[kNP];
#pragma unroll
  for (int k = 0; k < kNP; ++k) tot[k] = 0.0;

  for (int64_t base = s0; base < s1; base += kVB) {
    int cnt = (int)min((int64_t)kVB, s1 - base);
    __syncthreads();
    if (tid < cnt) {
      sx[tid] = a.xy[2 * (base + tid)];
      sy[tid] = a.xy[2 * (base + tid) + 1];
      sr[3 * tid] = a.w[3 * (base + tid)];
      sr[3 * tid + 1] = a.w[3 * (base + tid) + 1];
      sr[3 * tid + 2] = a.w[3 * (base + tid) + 2];
    }
    __syncthreads();
    if (!live) continue;
    T acc[kNP];
#pragma unroll
    for (int k = 0; k < kNP; ++k) acc[k] = T(0);
    if (is_pan) {
      for (int k = 0; k < cnt; ++k) {
        T x = sx[k], y = sy[k];
        if (NEAR) {
          Frame<T> f = frame(p, x, y);
          T dt = f.t1 > T(0) ? f.t1 : (f.t2 < T(0) ? f.t2 : T(0));
          if (dt * dt + f.h * f.h < a.near2 * f.L * f.L) {
            double dacc[kNP];
#pragma unroll
            for (int q = 0; q < kNP; ++q) dacc[q] = 0.0;
            pair_adj<double, SAME>(pd, double(x), double(y), double(sr[3 * k]),
                                   double(sr[3 * k + 1]), double(sr[3 * k + 2]), a.ec2d, a.ed2d,
                                   dacc);
#pragma unroll
            for (int q = 0; q < kNP; ++q) tot[q] += dacc[q];
            continue;
          }
        }
        pair_adj<T, SAME>(p, x, y, sr[3 * k], sr[3 * k + 1], sr[3 * k + 2], a.ec2, a.ed2, acc);
      }
    } else {
      for (int k = 0; k < cnt; ++k) {
        T phi = seg_angle(bax, bay, bbx, bby, sx[k], sy[k]);
        acc[0] += phi * sr[3 * k];
        acc[1] += phi * sr[3 * k + 1];
        acc[2] += phi * sr[3 * k + 2];
      }
    }
#pragma unroll
    for (int k = 0; k < kNP; ++k) tot[k] += double(acc[k]);
  }
  if (!live) return;
  if (is_pan) {
    double* o = a.part + ((size_t)blockIdx.y * a.P + idx) * kNP;
#pragma unroll
    for (int k = 0; k < kNP; ++k) o[k] = tot[k];
  } else {
    double* o = a.qpart + ((size_t)blockIdx.y * a.Nb + idx) * 3;
    for (int k = 0; k < 3; ++k) o[k] = tot[k] * kInv2Pi;
  }
}

// Float pair of the adjoint with the -2 pi-scaled partials of
// layer_grad_hat: the 11 sums come out multiplied by -2 pi.
template <bool SAME>
__device__ __forceinline__ void pair_adj_f(const Panel<float>& p, const Frame<float>& f, float hh,
                                           float r0, float r1, float r2, float ec2, float ed2,
                                           float* acc) {
  const GradHat g = layer_grad_hat(f, hh, ec2, ed2, SAME);
  const float al = -(r0 * p.wd[0] + r1 * p.wd[1] + r2 * p.wd[2]);
  const float be = r0 * p.wc[0] + r1 * p.wc[1] + r2 * p.wc[2];
  const float gt1 = al * g.Dt1 + be * g.St1;
  const float gt2 = al * g.Dt2 + be * g.St2;
  const float gh = al * g.Dh + be * g.Sh;
  acc[0] += gt1;
  acc[1] += gt2;
  acc[2] += f.h * (gt1 + gt2);
  acc[3] += f.t1 * gh;
  acc[4] += gh;
  acc[5] -= r0 * g.D;
  acc[6] -= r1 * g.D;
  acc[7] -= r2 * g.D;
  acc[8] += r0 * g.S;
  acc[9] += r1 * g.S;
  acc[10] += r2 * g.S;
}

// Float adjoint of the mixed path: one thread per panel (or boundary
// segment), the block's points staged 256 at a time as (x, y, r0, r1), r2;
// float sums per tile are added to double totals kept in shared memory
// (thread-owned columns), so the registers hold only the panel, the tile sums
// and the pair's temporaries.  Near pairs are skipped (evaluated in double by
// k_near_adjoint); the rounded frame of the near test is the pair's frame.
constexpr int kVT = 256;

template <bool SAME, bool NEAR>
__global__ void __launch_bounds__(kVB) k_vjp_f32(VjpArgs<float> a) {
  __shared__ float4 sq[kVT];
  __shared__ float sr2[kVT];
  __shared__ double stot[kNP][kVB];
  __shared__ float bred[4 * (kVB / 32)];
  const int tid = threadIdx.x;
  const int ptiles = (a.P + kVB - 1) / kVB;
  const bool is_pan = (int)blockIdx.x < ptiles;
  const int idx = is_pan ? blockIdx.x * kVB + tid : (blockIdx.x - ptiles) * kVB + tid;
  const bool live = is_pan ? idx < a.P : idx < a.Nb;
  const int64_t s0 = (int64_t)blockIdx.y * a.chunk;
  const int64_t s1 = min(a.n, s0 + a.chunk);
  Panel<float> p{};
  float thr = 0.f;
  float4 zone = make_float4(0.f, 0.f, -1.f, -1.f);
  float bax = 0, bay = 0, bbx = 0, bby = 0;
  if (live) {
    if (is_pan) {
      p = a.pan[idx];
      thr = near_thr(p.L, a.near2);
      zone = near_zone(p, a.nfac);
    } else {
      bax = a.vert[2 * idx]; bay = a.vert[2 * idx + 1];
      bbx = a.vert[2 * idx + 2]; bby = a.vert[2 * idx + 3];
    }
  }
#pragma unroll
  for (int k = 0; k < kNP; ++k) stot[k][tid] = 0.0;
  for (int64_t base = s0; base < s1; base += kVT) {
    const int cnt = (int)min((int64_t)kVT, s1 - base);
    __syncthreads();
    float x0 = __int_as_float(0x7f800000), y0 = x0, x1 = -x0, y1 = -x0;
    for (int e = tid; e < cnt; e += kVB) {
      const int64_t i = base + e;
      const float x = a.xy[2 * i], y = a.xy[2 * i + 1];
      sq[e] = make_float4(x, y, a.w[3 * i], a.w[3 * i + 1]);
      sr2[e] = a.w[3 * i + 2];
      x0 = fminf(x0, x); y0 = fminf(y0, y); x1 = fmaxf(x1, x); y1 = fmaxf(y1, y);
    }
    // near pairs are possible only in warps with a panel whose near zone
    // meets the tile's bounding box
    bool tested = false;
    if (NEAR && is_pan) {
      const float4 bb = block_bbox(x0, y0, x1, y1, tid < cnt, bred);
      tested = __any_sync(0xffffffffu, live && boxes_meet(zone, bb));
    }
    __syncthreads();
    if (!live) continue;
    float acc[kNP];
#pragma unroll
    for (int k = 0; k < kNP; ++k) acc[k] = 0.f;
    if (is_pan) {
      if (tested) {
        for (int k = 0; k < cnt; ++k) {
          const float4 q = sq[k];
          const Frame<float> f = frame_rn(p.ax, p.ay, p.tx, p.ty, p.L, q.x, q.y);
          const float hh = __fmul_rn(f.h, f.h);
          if (near_test(f, hh, thr)) continue;
          pair_adj_f<SAME>(p, f, hh, q.z, q.w, sr2[k], a.ec2, a.ed2, acc);
        }
      } else {
        for (int k = 0; k < cnt; ++k) {
          const float4 q = sq[k];
          const Frame<float> f = frame_rn(p.ax, p.ay, p.tx, p.ty, p.L, q.x, q.y);
          pair_adj_f<SAME>(p, f, f.h * f.h, q.z, q.w, sr2[k], a.ec2, a.ed2, acc);
        }
      }
    } else {
      for (int k = 0; k < cnt; ++k) {
        const float4 q = sq[k];
        const float phi = seg_angle(bax, bay, bbx, bby, q.x, q.y);
        acc[0] += phi * q.z;
        acc[1] += phi * q.w;
        acc[2] += phi * sr2[k];
      }
    }
#pragma unroll
    for (int k = 0; k < kNP; ++k) stot[k][tid] += (double)acc[k];
  }
  if (!live) return;
  if (is_pan) {
    double* o = a.part + ((size_t)blockIdx.y * a.P + idx) * kNP;
#pragma unroll
    for (int k = 0; k < kNP; ++k) o[k] = stot[k][tid] * -kInv2Pi;
  } else {
    double* o = a.qpart + ((size_t)blockIdx.y * a.Nb + idx) * 3;
    for (int k = 0; k < 3; ++k) o[k] = stot[k][tid] * kInv2Pi;
  }
}

// out[m] (+)= sum over slices of part[slice][m], fixed order
__global__ void k_reduce_slices(const double* __restrict__ part, int slices, int64_t m,
                                double* __restrict__ out, int accumulate) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  double s = 0;
  for (int k = 0; k < slices; ++k) s += part[(size_t)k * m + t];
  out[t] = accumulate ? out[t] + s : s;
}

// weights of the boundary Gauss points: lambda_i |G_i| w_k
template <typename T>
__global__ void k_gauss_weights(const double* __restrict__ lam, int Nb,
                                const double* __restrict__ vert, T* __restrict__ w) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * Nb) return;
  int i = t / 3, q = t % 3;
  double ex = vert[2 * (i + 1)] - vert[2 * i], ey = vert[2 * (i + 1) + 1] - vert[2 * i + 1];
  double s = sqrt(ex * ex + ey * ey) * gauss_weight(q);
  for (int c = 0; c < 3; ++c) w[3 * t + c] = T(lam[3 * i + c] * s);
}

// Panel sums -> parameter gradient through the Bernstein maps.
__global__ void k_chain(const double* __restrict__ ps, const Panel<double>* __restrict__ pan,
                        const int* __restrict__ off, const int* __restrict__ Kc,
                        const uint8_t* __restrict__ closed, int C, double scale,
                        double* __restrict__ grad) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= 4 * C) return;
  int i = h / 4, j = h % 4, K = Kc[i];
  bool cl = closed[i];
  double gx = 0, gy = 0, gd[3] = {0, 0, 0}, gc[3] = {0, 0, 0};
  for (int k = 0; k < K; ++k) {
    int p = off[i] + k;
    const double* q = ps + (size_t)p * kNP;
    double t0 = double(k) / K, t1 = double(k + 1) / K;
    double wa = bern3(j, t0), wb = bern3(j, t1);
    if (cl && j == 0) { wa += bern3(3, t0); wb += bern3(3, t1); }
    if (cl && j == 3) { wa = 0; wb = 0; }
    double L = pan[p].L;
    if (L > 0 && (wa != 0 || wb != 0)) {
      double tx = pan[p].tx, ty = pan[p].ty, iL = 1.0 / L;
      double na = (-q[2] + q[3] + L * q[4]) * iL;
      double nb = (q[2] - q[3]) * iL;
      double dax = q[0] * tx + na * ty, day = q[0] * ty - na * tx;
      double dbx = q[1] * tx + nb * ty, dby = q[1] * ty - nb * tx;
      gx += wa * dax + wb * dbx;
      gy += wa * day + wb * dby;
    }
    double wm = bern3(j, (k + 0.5) / K);
    for (int c = 0; c < 3; ++c) {
      gd[c] += wm * q[5 + c];
      gc[c] += wm * q[8 + c];
    }
  }
  double* g = grad + (size_t)h * 8;
  g[0] = scale * gx;
  g[1] = scale * gy;
  for (int c = 0; c < 3; ++c) {
    g[2 + c] = scale * gd[c];
    g[5 + c] = scale * gc[c];
  }
}

// Panel sums -> parameter gradient of segment handles (panel h = handle h):
// a, b from the frame chain rule, the jumps directly.
__global__ void k_chain_seg(const double* __restrict__ ps, const Panel<double>* __restrict__ pan,
                            int H, double scale, double* __restrict__ grad) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  const double* q = ps + (size_t)h * kNP;
  double* g = grad + (size_t)h * 10;
  const double L = pan[h].L;
  double dax = 0, day = 0, dbx = 0, dby = 0;
  if (L > 0) {
    const double tx = pan[h].tx, ty = pan[h].ty, iL = 1.0 / L;
    const double na = (-q[2] + q[3] + L * q[4]) * iL;
    const double nb = (q[2] - q[3]) * iL;
    dax = q[0] * tx + na * ty; day = q[0] * ty - na * tx;
    dbx = q[1] * tx + nb * ty; dby = q[1] * ty - nb * tx;
  }
  g[0] = scale * dax; g[1] = scale * day; g[2] = scale * dbx; g[3] = scale * dby;
  for (int c = 0; c < 3; ++c) {
    g[4 + c] = scale * q[5 + c];
    g[7 + c] = scale * q[8 + c];
  }
}

// gradient from the panel sums for either parametrisation
static void launch_chain(bem_ctx* c, const double* sums, double* grad) {
  if (c->sc.pp == 4)
    k_chain_seg<<<(c->sc.NH + 127) / 128, 128, 0, S(c)>>>(sums, c->d_pan64, c->sc.NH, 1.0, grad);
  else
    k_chain<<<(4 * c->sc.C + 127) / 128, 128, 0, S(c)>>>(sums, c->d_pan64, c->sc.d_off, c->sc.d_K,
                                                        c->sc.d_closed, c->sc.C, 1.0, grad);
  BEM_LAUNCHED(c);
}

template <typename T>
static int vjp_pass(bem_ctx* c, int64_t n, const T* xy, const T* w, bool boundary, int accumulate) {
  int rc;
  const bool f32 = sizeof(T) == 4;
  const bool near = f32 && c->opts.near_factor > 0;
  int P = c->sc.P, Nb = boundary ? c->bd.Nb : 0;
  int ptiles = (P + kVB - 1) / kVB, btiles = (Nb + kVB - 1) / kVB;
  int tiles = ptiles + btiles;
  // double kernel: about four resident blocks per SM; float kernel: about
  // three waves of seven resident blocks per SM
  const int step = f32 ? kVT : kVB;
  const int64_t sms = c->sms;
  int64_t want = f32 ? (3 * 7 * sms + tiles - 1) / tiles : (4 * sms + tiles - 1) / tiles;
  int64_t maxs = (n + step - 1) / step;
  int slices = (int)std::max<int64_t>(1, std::min<int64_t>(want, maxs));
  int64_t chunk = ((n + slices - 1) / slices + step - 1) / step * step;
  slices = (int)std::max<int64_t>(1, (n + chunk - 1) / chunk);
  if (n <= 0) slices = 0;
  const int pslices = slices + (near && n > 0 ? 1 : 0);     // near sums in the last slice
  size_t pbytes = sizeof(double) * (size_t)std::max(pslices, 1) * P * kNP;
  size_t qbytes = sizeof(double) * (size_t)std::max(slices, 1) * (Nb > 0 ? Nb : 1) * 3;
  if ((rc = grow(c, c->part, pbytes + qbytes))) return rc;
  VjpArgs<T> a{};
  a.xy = xy;
  a.w = w;
  a.n = n;
  a.pan = (const Panel<T>*)(f32 ? (const void*)c->d_pan32 : (const void*)c->d_pan64);
  a.pan64 = c->d_pan64;
  a.P = P;
  a.vert = (const T*)(f32 ? (const void*)c->bd.d_vert32 : (const void*)c->bd.d_vert);
  a.Nb = Nb;
  a.ec2 = T(c->opts.eps_c * c->opts.eps_c);
  a.ed2 = T(c->opts.eps_d * c->opts.eps_d);
  a.ec2d = c->opts.eps_c * c->opts.eps_c;
  a.ed2d = c->opts.eps_d * c->opts.eps_d;
  a.near2 = T(c->opts.near_factor * c->opts.near_factor);
  a.nfac = float(c->opts.near_factor);
  a.chunk = chunk;
  a.part = (double*)c->part.p;
  a.qpart = (double*)((char*)c->part.p + pbytes);
  if (n > 0) {
    dim3 grid(tiles, slices);
    ProfScope _ps(c, Nb > 0 ? "k_vjp" : "k_vjp_gauss");
    bool same = c->opts.eps_c == c->opts.eps_d;
    if constexpr (sizeof(T) == 4) {
      if (same) {
        if (near) k_vjp_f32<true, true><<<grid, kVB, 0, S(c)>>>(a);
        else k_vjp_f32<true, false><<<grid, kVB, 0, S(c)>>>(a);
      } else {
        if (near) k_vjp_f32<false, true><<<grid, kVB, 0, S(c)>>>(a);
        else k_vjp_f32<false, false><<<grid, kVB, 0, S(c)>>>(a);
      }
    } else {
      if (same) k_vjp<T, true, false><<<grid, kVB, 0, S(c)>>>(a);
      else k_vjp<T, false, false><<<grid, kVB, 0, S(c)>>>(a);
    }
    BEM_LAUNCHED(c);
  }
  if (near && n > 0) {
    if ((rc = near_adjoint(c, n, (const float*)xy, (const float*)w,
                           a.part + (size_t)slices * P * kNP)))
      return rc;
  }
  // panel sums (accumulated into part2[P][11]) and q (into d_q)
  int64_t m = (int64_t)P * kNP;
  if (pslices > 0) {
    k_reduce_slices<<<(unsigned)((m + 255) / 256), 256, 0, S(c)>>>(a.part, pslices, m,
                                                                     (double*)c->part2.p,
                                                                     accumulate);
    BEM_LAUNCHED(c);
  } else if (!accumulate) {
    if ((rc = cuda_check(c, cudaMemsetAsync(c->part2.p, 0, sizeof(double) * m, S(c)), "memset")))
      return rc;
  }
  if (boundary) {
    if (slices > 0) {
      k_reduce_slices<<<(3 * Nb + 255) / 256, 256, 0, S(c)>>>(a.qpart, slices, 3 * (int64_t)Nb,
                                                               c->d_q, 0);
      BEM_LAUNCHED(c);
    } else if ((rc = cuda_check(c, cudaMemsetAsync(c->d_q, 0, sizeof(double) * 3 * Nb, S(c)),
                                "memset"))) {
      return rc;
    }
  }
  return cuda_check(c, cudaGetLastError(), "k_vjp");
}

template <typename T>
static int adj_vjp_t(bem_ctx* c, int64_t n, const T* xy, const T* resid, double* grad) {
  int rc;
  int P = c->sc.P, Nb = c->bd.Nb;
  if ((rc = grow(c, c->part2, sizeof(double) * (size_t)P * kNP))) return rc;
  // samples: panel sums and q
  if ((rc = vjp_pass<T>(c, n, xy, resid, true, 0))) return rc;
  // lambda = (A^+)^T q
  if (c->opts.precision == BEM_FP64) rc = la_apply3(c, c->bd.d_WT, c->d_q, c->d_lb);
  else rc = la_apply3_refined(c, c->bd.d_WT32, c->bd.d_A, c->d_q, c->d_lb, true);
  if (rc) return rc;
  // boundary Gauss points with weights lambda_i |G_i| w_k
  if ((rc = grow(c, c->g, sizeof(double) * 9 * (size_t)Nb))) return rc;
  T* gw = (T*)c->g.p;
  k_gauss_weights<T><<<(3 * Nb + 255) / 256, 256, 0, S(c)>>>(c->d_lb, Nb, c->bd.d_vert, gw);
  BEM_LAUNCHED(c);
  const T* gp = (const T*)(sizeof(T) == 8 ? (const void*)c->bd.d_gp : (const void*)c->bd.d_gp32);
  if ((rc = vjp_pass<T>(c, 3 * (int64_t)Nb, gp, gw, false, 1))) return rc;
  launch_chain(c, (const double*)c->part2.p, grad);
  return cuda_check(c, cudaGetLastError(), "vjp chain");
}

int adj_vjp(bem_ctx* c, int64_t n, const void* xy, const void* resid, double* grad) {
  if (c->opts.precision == BEM_FP64)
    return adj_vjp_t<double>(c, n, (const double*)xy, (const double*)resid, grad);
  return adj_vjp_t<float>(c, n, (const float*)xy, (const float*)resid, grad);
}

}  // namespace bem

// ---------------------------------------------------------------------------
// Allocation-free adjoint.
//
// For callers that may not allocate device memory while the hot path runs:
// real-time loops that must not enter the allocator (cudaMalloc/cudaFree can
// stall the whole device), and hosts whose own memory pool owns the GPU and
// hands out no more device memory once it is set up.  Every
// per-call buffer of the adjoint (per-slice partial sums, panel sums, Gauss
// weights, refinement residuals) lives in the static array below; the
// persistent state (panels, boundary factors) was allocated by bem_setup and
// bem_factor beforehand.  The array is shared by all calls on a device and
// keeps the previous call's contents; everything a call reads is written by
// that call first.  Calls whose work overlaps on the GPU race on it.

namespace bem {
namespace {

constexpr size_t kNoAllocBytes = 32u << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the static array on the current device.  It is looked
// up on every call (a host-side table lookup, no device work): a cached
// address would outlive a device reset or a released and re-created primary
// context.  The first lookup on a device loads the library's device code
// there, which must not happen inside a stream capture.
int noalloc_base(bem_ctx* c, unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_check(c, e, "cudaGetSymbolAddress of the static scratch");
  *out = (unsigned char*)p;
  return BEM_OK;
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

// one pass of the adjoint kernels over n points with explicit buffers:
// partial sums into part (slices x P x 11) and qpart, reduced into sums
// (added when accumulate) and q
template <typename T>
int noalloc_pass(bem_ctx* c, int64_t n, const T* xy, const T* w, bool boundary, int accumulate,
                 int max_slices, double* part, double* qpart, double* sums, double* q) {
  const int P = c->sc.P, Nb = boundary ? c->bd.Nb : 0;
  const int ptiles = (P + kVB - 1) / kVB, btiles = (Nb + kVB - 1) / kVB;
  const int tiles = ptiles + btiles;
  const bool f32 = sizeof(T) == 4;
  const int step = f32 ? kVT : kVB;
  const int64_t sms = c->sms;
  int64_t want = f32 ? (3 * 7 * sms + tiles - 1) / tiles : (4 * sms + tiles - 1) / tiles;
  want = std::min<int64_t>(want, max_slices);
  int64_t maxs = (n + step - 1) / step;
  int slices = (int)std::max<int64_t>(1, std::min<int64_t>(want, maxs));
  const int64_t chunk = ((n + slices - 1) / slices + step - 1) / step * step;
  slices = (int)std::max<int64_t>(1, (n + chunk - 1) / chunk);
  const int64_t m = (int64_t)P * kNP;
  if (n <= 0) {
    if (!accumulate)
      cudaMemsetAsync(sums, 0, sizeof(double) * m, S(c));
    if (boundary) cudaMemsetAsync(q, 0, sizeof(double) * 3 * Nb, S(c));
    return cuda_check(c, cudaGetLastError(), "noalloc pass");
  }
  VjpArgs<T> a{};
  a.xy = xy;
  a.w = w;
  a.n = n;
  a.pan = (const Panel<T>*)(f32 ? (const void*)c->d_pan32 : (const void*)c->d_pan64);
  a.pan64 = c->d_pan64;
  a.P = P;
  a.vert = (const T*)(f32 ? (const void*)c->bd.d_vert32 : (const void*)c->bd.d_vert);
  a.Nb = Nb;
  a.ec2 = T(c->opts.eps_c * c->opts.eps_c);
  a.ed2 = T(c->opts.eps_d * c->opts.eps_d);
  a.ec2d = c->opts.eps_c * c->opts.eps_c;
  a.ed2d = c->opts.eps_d * c->opts.eps_d;
  a.near2 = T(0);
  a.chunk = chunk;
  a.part = part;
  a.qpart = qpart;
  dim3 grid(tiles, slices);
  const bool same = c->opts.eps_c == c->opts.eps_d;
  if constexpr (sizeof(T) == 4) {
    if (same) k_vjp_f32<true, false><<<grid, kVB, 0, S(c)>>>(a);
    else k_vjp_f32<false, false><<<grid, kVB, 0, S(c)>>>(a);
  } else {
    if (same) k_vjp<T, true, false><<<grid, kVB, 0, S(c)>>>(a);
    else k_vjp<T, false, false><<<grid, kVB, 0, S(c)>>>(a);
  }
  k_reduce_slices<<<(unsigned)((m + 255) / 256), 256, 0, S(c)>>>(part, slices, m, sums, accumulate);
  c->launches += 2;
  if (boundary) {
    k_reduce_slices<<<(3 * Nb + 255) / 256, 256, 0, S(c)>>>(qpart, slices, 3 * (int64_t)Nb, q, 0);
    BEM_LAUNCHED(c);
  }
  return cuda_check(c, cudaGetLastError(), "noalloc pass");
}

template <typename T>
int noalloc_vjp(bem_ctx* c, int64_t n, const T* xy, const T* resid, double* grad,
                unsigned char* base) {
  const int P = c->sc.P, Nb = c->bd.Nb;
  // fixed part: panel sums, Gauss weights, refinement residuals
  const size_t sums_b = up256(sizeof(double) * (size_t)P * kNP);
  const size_t gw_b = up256(sizeof(T) * 9 * (size_t)Nb);
  const size_t ref_b = up256(sizeof(double) * 6 * (size_t)Nb);
  const size_t fixed = sums_b + gw_b + ref_b;
  const size_t per_slice = sizeof(double) * ((size_t)P * kNP + 3 * (size_t)Nb);
  if (fixed + per_slice > kNoAllocBytes) {
    char msg[200];
    snprintf(msg, sizeof(msg),
             "bem_vjp_noalloc: %d panels need more than its %zu-byte static scratch "
             "(limit about %zu panels at %d boundary segments)",
             P, kNoAllocBytes,
             (kNoAllocBytes - ref_b - 8 * 12 * (size_t)Nb) / (2 * 8 * kNP), Nb);
    return fail(c, BEM_EINVAL, msg);
  }
  const int max_slices = (int)std::min<size_t>(4096, (kNoAllocBytes - fixed) / per_slice);
  double* sums = (double*)base;
  T* gw = (T*)(base + sums_b);
  double* ref = (double*)(base + sums_b + gw_b);
  double* part = (double*)(base + fixed);
  double* qpart = part + (size_t)max_slices * P * kNP;
  int rc;
  if ((rc = geom_panelize(c, c->d_theta))) return rc;
  if ((rc = noalloc_pass<T>(c, n, xy, resid, true, 0, max_slices, part, qpart, sums, c->d_q))) return rc;
  if (c->opts.precision == BEM_FP64) rc = la_apply3(c, c->bd.d_WT, c->d_q, c->d_lb);
  else rc = la_apply3_refined_buf(c, c->bd.d_WT32, c->bd.d_A, c->d_q, c->d_lb, true, ref);
  if (rc) return rc;
  k_gauss_weights<T><<<(3 * Nb + 255) / 256, 256, 0, S(c)>>>(c->d_lb, Nb, c->bd.d_vert, gw);
  BEM_LAUNCHED(c);
  const T* gp = (const T*)(sizeof(T) == 8 ? (const void*)c->bd.d_gp : (const void*)c->bd.d_gp32);
  if ((rc = noalloc_pass<T>(c, 3 * (int64_t)Nb, gp, gw, false, 1, max_slices, part, qpart, sums,
                            nullptr)))
    return rc;
  launch_chain(c, sums, grad);
  return cuda_check(c, cudaGetLastError(), "noalloc vjp");
}

}  // namespace

}  // namespace bem

extern "C" int bem_vjp_noalloc(bem_ctx* c, int64_t n, const void* xy, const void* resid,
                               double* grad_out, void* stream) {
  using namespace bem;
  if (!c) return BEM_EINVAL;
  if (n < 0 || !grad_out || (n > 0 && (!xy || !resid)))
    return fail(c, BEM_EINVAL, "bem_vjp_noalloc: bad arguments");
  if (!c->have_scene) return fail(c, BEM_ESTATE, "bem_setup has not been called");
  if (!c->bd.factored) return fail(c, BEM_ESTATE, "bem_factor has not been called");
  int rc;
  if ((rc = cuda_check(c, cudaSetDevice(c->device), "cudaSetDevice"))) return rc;
  c->cur = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  if ((rc = noalloc_base(c, &base))) return rc;
  if (c->opts.precision == BEM_FP64)
    return noalloc_vjp<double>(c, n, (const double*)xy, (const double*)resid, grad_out, base);
  return noalloc_vjp<float>(c, n, (const float*)xy, (const float*)resid, grad_out, base);
}
