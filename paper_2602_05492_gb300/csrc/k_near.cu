// Near field of the mixed-precision path.
//
// The float main loops (forward evaluation, adjoint) skip every pair whose
// point lies closer than near_factor panel lengths to the panel (near_pair in
// common.cuh); the kernels here evaluate exactly those pairs in double:
//   near_forward  thread per point, candidate panels from a panel -> cell
//                 binning (each panel listed in every cell its near region
//                 touches); writes the double near sum of each point
//   near_adjoint  thread per panel, candidate points from a point -> cell
//                 binning; writes the 11 adjoint sums of each panel
// Cell lists are sorted by index, so every double sum has a fixed order.
#include <algorithm>
#include <cmath>

#include "ctx.h"
#include "dmath.cuh"

namespace bem {

// ---------------------------------------------------------------------------
// exclusive scan of int counts (in place), n up to a few million

__global__ void k_scan_block(int* __restrict__ v, int n, int* __restrict__ sums) {
  __shared__ int ws[32];
  const int base = blockIdx.x * 2048;
  const int i0 = base + 2 * threadIdx.x;
  int a = i0 < n ? v[i0] : 0, b = i0 + 1 < n ? v[i0 + 1] : 0;
  int t = a + b, x = t;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = ws[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  const int excl = x - t + (w > 0 ? ws[w - 1] : 0);
  if (i0 < n) v[i0] = excl;
  if (i0 + 1 < n) v[i0 + 1] = excl + a;
  if (threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = excl + t;
}

__global__ void k_scan_sums(int* __restrict__ sums, int nb, int* __restrict__ total) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int s = 0;
    for (int b = 0; b < nb; ++b) {
      int t = sums[b];
      sums[b] = s;
      s += t;
    }
    *total = s;
  }
}

__global__ void k_scan_add(int* __restrict__ v, int n, const int* __restrict__ sums) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] += sums[i / 2048];
}

// v[0..n) -> exclusive prefix sums; *total (device) = sum
static void scan(bem_ctx* c, int* v, int n, int* sums, int* total) {
  int nb = (n + 2047) / 2048;
  k_scan_block<<<nb, 1024, 0, S(c)>>>(v, n, sums);
  k_scan_sums<<<1, 32, 0, S(c)>>>(sums, nb, total);
  k_scan_add<<<(n + 255) / 256, 256, 0, S(c)>>>(v, n, sums);
  c->launches += 3;
}

__device__ __forceinline__ int cell_of(float v, int G) {
  int k = (int)floorf(v * G);
  return k < 0 ? 0 : (k >= G ? G - 1 : k);
}

// cells touched by the near region of panel p (its segment grown by
// near_factor L, plus a small margin for rounding)
__device__ __forceinline__ void panel_cells(const Panel<float>& p, float nf, int G, int& x0,
                                            int& x1, int& y0, int& y1) {
  const float bx = p.ax + p.tx * p.L, by = p.ay + p.ty * p.L;
  const float r = nf * p.L * 1.001f + 1e-6f;
  x0 = cell_of(fminf(p.ax, bx) - r, G);
  x1 = cell_of(fmaxf(p.ax, bx) + r, G);
  y0 = cell_of(fminf(p.ay, by) - r, G);
  y1 = cell_of(fmaxf(p.ay, by) + r, G);
}

// One warp per panel: the lanes take the cells of the panel's box in turn
// (a box spans tens of cells; one thread per panel would wait for each
// cell's atomic in sequence).
__global__ void k_pbin_count(const Panel<float>* __restrict__ pan, int P, float nf, int G,
                             int* __restrict__ cnt) {
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (p >= P) return;
  int x0, x1, y0, y1;
  panel_cells(pan[p], nf, G, x0, x1, y0, y1);
  const int w = x1 - x0 + 1, ncell = w * (y1 - y0 + 1);
  for (int k = lane; k < ncell; k += 32) atomicAdd(&cnt[(y0 + k / w) * G + x0 + k % w], 1);
}

__global__ void k_pbin_fill(const Panel<float>* __restrict__ pan, int P, float nf, int G,
                            const int* __restrict__ start, int* __restrict__ fill,
                            int* __restrict__ items) {
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (p >= P) return;
  int x0, x1, y0, y1;
  panel_cells(pan[p], nf, G, x0, x1, y0, y1);
  const int w = x1 - x0 + 1, ncell = w * (y1 - y0 + 1);
  for (int k = lane; k < ncell; k += 32) {
    const int cell = (y0 + k / w) * G + x0 + k % w;
    items[start[cell] + atomicAdd(&fill[cell], 1)] = p;
  }
}

__global__ void k_sbin_count(const float* __restrict__ xy, int64_t n, int G, int* __restrict__ cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  atomicAdd(&cnt[cell_of(xy[2 * i + 1], G) * G + cell_of(xy[2 * i], G)], 1);
}

__global__ void k_sbin_fill(const float* __restrict__ xy, int64_t n, int G,
                            const int* __restrict__ start, int* __restrict__ fill,
                            int* __restrict__ items) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cell = cell_of(xy[2 * i + 1], G) * G + cell_of(xy[2 * i], G);
  items[start[cell] + atomicAdd(&fill[cell], 1)] = (int)i;
}

// ascending order inside every cell list
__global__ void k_bin_sort(const int* __restrict__ start, int ncell, int* __restrict__ items) {
  int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= ncell) return;
  int b = start[cell], e = start[cell + 1];
  for (int i = b + 1; i < e; ++i) {
    int v = items[i], j = i - 1;
    while (j >= b && items[j] > v) {
      items[j + 1] = items[j];
      --j;
    }
    items[j + 1] = v;
  }
}

// buffers: [ncell+1] start, [ncell] fill, [nb] scan sums, [1] total, items
struct Bins {
  int G;
  int* start;
  int* items;
};

static int build_bins(bem_ctx* c, DevBuf& buf, bool panels, int64_t n, const float* xy, Bins& out) {
  int rc;
  const int P = c->sc.P;
  int G;
  if (panels) {
    G = 256;
  } else {
    G = 16;
    while (G < 2048 && (int64_t)(2 * G) * (2 * G) * 8 <= n) G *= 2;
  }
  const int ncell = G * G;
  const int nb = (ncell + 1 + 2047) / 2048;
  const size_t head = sizeof(int) * ((size_t)ncell + 1 + ncell + nb + 1);
  // item capacity: points -> n; panels -> counted on the device, bounded here by
  // the total cell coverage, which needs one synchronisation
  if ((rc = grow(c, buf, head + 64))) return rc;
  int* start = (int*)buf.p;
  int* fill = start + ncell + 1;
  int* sums = fill + ncell;
  int* total = sums + nb;
  if ((rc = cuda_check(c, cudaMemsetAsync(start, 0, sizeof(int) * (2 * (size_t)ncell + 1), S(c)),
                       "memset")))
    return rc;
  if (panels)
    k_pbin_count<<<(P + 7) / 8, 256, 0, S(c)>>>(c->d_pan32, P, (float)c->opts.near_factor, G,
                                                start);
  else
    k_sbin_count<<<(unsigned)((n + 255) / 256), 256, 0, S(c)>>>(xy, n, G, start);
  BEM_LAUNCHED(c);
  scan(c, start, ncell + 1, sums, total);
  int tot = 0;
  if ((rc = cuda_check(c, cudaMemcpyAsync(&tot, total, sizeof(int), cudaMemcpyDeviceToHost, S(c)),
                       "bins")) ||
      (rc = cuda_check(c, cudaStreamSynchronize(S(c)), "bins")))
    return rc;
  const size_t need = head + sizeof(int) * ((size_t)tot + 1);
  if (need > buf.cap) {
    // grow keeping the counts: copy the head aside
    DevBuf tmp;
    if ((rc = grow(c, tmp, head))) return rc;
    cudaMemcpyAsync(tmp.p, buf.p, head, cudaMemcpyDeviceToDevice, S(c));
    if ((rc = grow(c, buf, need))) { cudaFree(tmp.p); return rc; }
    cudaMemcpyAsync(buf.p, tmp.p, head, cudaMemcpyDeviceToDevice, S(c));
    cudaStreamSynchronize(S(c));
    cudaFree(tmp.p);
    start = (int*)buf.p;
    fill = start + ncell + 1;
  }
  int* items = (int*)((char*)buf.p + head);
  if (panels)
    k_pbin_fill<<<(P + 7) / 8, 256, 0, S(c)>>>(c->d_pan32, P, (float)c->opts.near_factor, G,
                                               start, fill, items);
  else
    k_sbin_fill<<<(unsigned)((n + 255) / 256), 256, 0, S(c)>>>(xy, n, G, start, fill, items);
  k_bin_sort<<<(ncell + 255) / 256, 256, 0, S(c)>>>(start, ncell, items);
  c->launches += 2;
  out.G = G;
  out.start = start;
  out.items = items;
  return cuda_check(c, cudaGetLastError(), "bins");
}

// ---------------------------------------------------------------------------
// double evaluation of the near pairs

// (ic_j, lc_j) of dlog and (c_j, atan(c_j)) of datan2_ypos, per device
__device__ double2 g_dlog_tab[kDlogTab];
__device__ double2 g_datan_tab[kDatanTab];

__global__ void k_dmath_init() {
  const int j = threadIdx.x;
  if (j < kDlogTab) {
    const double ic = 1.0 / (1.0 + (j + 0.5) / kDlogTab);
    g_dlog_tab[j] = make_double2(ic, -log(ic));
  }
  if (j < kDatanTab) {
    const double cj = (double)j / kDatanTab;
    g_datan_tab[j] = make_double2(cj, atan(cj));
  }
}

// The layer values of a near pair in double: the integrals of layer_values,
// with log(q2/q1) taken as the difference of two logarithms (dlog) instead of
// log1p of a quotient, and 1/h' from one reciprocal square root.  For a near
// pair q1 and q2 are of the scale of a few squared panel lengths, so the
// difference keeps an absolute accuracy of a few units of 2^-53 times
// |log q|, far below what the float far field carries.
template <bool SAME>
__device__ __forceinline__ LayerVals<double> layer_values_near(const Frame<double>& f, double ec2,
                                                              double ed2) {
  LayerVals<double> v;
  const double hh = f.h * f.h;
  const double hc2 = hh + ec2;
  const double rc = rsqrt(hc2);
  const double hc = hc2 * rc;
  const double tt = f.t1 * f.t2;
  const double q1 = fma(f.t1, f.t1, hc2), q2 = fma(f.t2, f.t2, hc2);
  const double phic = datan2_ypos(hc * f.L, hc2 + tt, g_datan_tab);
  const double lg1 = dlog(q1, g_dlog_tab), lg2 = dlog(q2, g_dlog_tab);
  v.S = -(f.L * (lg2 - 2.0) + f.t1 * (lg2 - lg1) + 2.0 * hc * phic) * kInv4Pi;
  if constexpr (SAME) {
    v.Dl = -(f.h * rc) * phic * kInv2Pi;
  } else {
    const double hd2 = hh + ed2;
    const double rd = rsqrt(hd2);
    v.Dl = -(f.h * rd) * datan2_ypos(hd2 * rd * f.L, hd2 + tt, g_datan_tab) * kInv2Pi;
  }
  return v;
}

// The layer values and frame partials of a near pair in double (the
// adjoint's near field): the integrals and derivatives of layer_grad, with
// both logarithms from dlog (log(q2/q1) as their difference), 1/h' from one
// reciprocal square root and 1/q1, 1/q2 from one reciprocal of q1 q2.
template <bool SAME>
__device__ __forceinline__ LayerGrad<double> layer_grad_near(const Frame<double>& f, double ec2,
                                                             double ed2) {
  LayerGrad<double> g;
  const double tt = f.t1 * f.t2, hh = f.h * f.h;
  // single layer, eps_c
  const double hc2 = hh + ec2;
  const double rc = rsqrt(hc2);
  const double hc = hc2 * rc;
  const double q1 = fma(f.t1, f.t1, hc2), q2 = fma(f.t2, f.t2, hc2);
  const double phic = datan2_ypos(hc * f.L, hc2 + tt, g_datan_tab);
  const double lg1 = dlog(q1, g_dlog_tab), lg2 = dlog(q2, g_dlog_tab);
  g.S = -(f.L * (lg2 - 2.0) + f.t1 * (lg2 - lg1) + 2.0 * hc * phic) * kInv4Pi;
  g.S_t1 = lg1 * kInv4Pi;
  g.S_t2 = -lg2 * kInv4Pi;
  g.S_h = -(f.h * rc) * phic * kInv2Pi;
  // double layer, eps_d
  double hd2, rd, phid, r1, r2;
  if constexpr (SAME) {
    hd2 = hc2; rd = rc; phid = phic; r1 = q1; r2 = q2;
  } else {
    hd2 = hh + ed2;
    rd = rsqrt(hd2);
    phid = datan2_ypos(hd2 * rd * f.L, hd2 + tt, g_datan_tab);
    r1 = fma(f.t1, f.t1, hd2);
    r2 = fma(f.t2, f.t2, hd2);
  }
  const double ir12 = 1.0 / (r1 * r2);
  const double ir1 = r2 * ir12, ir2 = r1 * ir12;
  g.Dl = -(f.h * rd) * phid * kInv2Pi;
  g.D_t1 = f.h * ir1 * kInv2Pi;
  g.D_t2 = -f.h * ir2 * kInv2Pi;
  g.D_h = -(ed2 * phid * rd - hh * f.L * (hd2 - tt) * ir12) * (rd * rd) * kInv2Pi;
  return g;
}

// SUBF: the sum of (double - float) pair values instead, the float value
// being the one the F rows hold (frame_rn, layer_grad_hat); added to the
// float handle term F w it gives the same near-field treatment as the
// evaluation kernel's skip-and-add.
template <bool SAME, bool SUBF>
__global__ void k_near_forward(const float* __restrict__ xy, int64_t n,
                               const Panel<float>* __restrict__ pan32,
                               const Panel<double>* __restrict__ pan64, Bins b, float near2,
                               double ec2, double ed2, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = xy[2 * i], y = xy[2 * i + 1];
  const int cell = cell_of(y, b.G) * b.G + cell_of(x, b.G);
  double s0 = 0, s1 = 0, s2 = 0;
  for (int k = b.start[cell]; k < b.start[cell + 1]; ++k) {
    const int p = b.items[k];
    if (!near_pair(pan32[p], x, y, near2)) continue;
    const Panel<double>& q = pan64[p];
    Frame<double> f = frame(q, double(x), double(y));
    const LayerVals<double> v = layer_values_near<SAME>(f, ec2, ed2);
    s0 += -q.wd[0] * v.Dl + q.wc[0] * v.S;
    s1 += -q.wd[1] * v.Dl + q.wc[1] * v.S;
    s2 += -q.wd[2] * v.Dl + q.wc[2] * v.S;
    if constexpr (SUBF) {
      const Panel<float>& pf = pan32[p];
      const Frame<float> ff = frame_rn(pf.ax, pf.ay, pf.tx, pf.ty, pf.L, x, y);
      const GradHat g = layer_grad_hat(ff, ff.h * ff.h, float(ec2), float(ed2), SAME);
      constexpr float kOut = float(-kInv2Pi);   // the hat values carry -2 pi
      s0 -= double(kOut * (-pf.wd[0] * g.D + pf.wc[0] * g.S));
      s1 -= double(kOut * (-pf.wd[1] * g.D + pf.wc[1] * g.S));
      s2 -= double(kOut * (-pf.wd[2] * g.D + pf.wc[2] * g.S));
    }
  }
  out[3 * i] = s0;
  out[3 * i + 1] = s1;
  out[3 * i + 2] = s2;
}

// One warp per panel.  The lanes test the candidate points of the panel's
// cells 32 at a time (float near test), append the near ones to a per-warp
// queue in shared memory (ballot + popcount, queue order = candidate order),
// and evaluate the queue in double 32 pairs at a time, so the double work
// runs on full warps.  The lanes' sums are combined by a fixed butterfly; the
// result does not depend on scheduling.
constexpr int kNearWarps = 4;

template <bool SAME>
__device__ __forceinline__ void near_adj_pair(const Panel<double>& q, float x, float y, double r0,
                                              double r1, double r2, double ec2, double ed2,
                                              double* acc) {
  Frame<double> f = frame(q, double(x), double(y));
  const LayerGrad<double> g = layer_grad_near<SAME>(f, ec2, ed2);
  const double al = -(r0 * q.wd[0] + r1 * q.wd[1] + r2 * q.wd[2]);
  const double be = r0 * q.wc[0] + r1 * q.wc[1] + r2 * q.wc[2];
  const double gt1 = al * g.D_t1 + be * g.S_t1;
  const double gt2 = al * g.D_t2 + be * g.S_t2;
  const double gh = al * g.D_h + be * g.S_h;
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

template <bool SAME>
__global__ void __launch_bounds__(32 * kNearWarps)
    k_near_adjoint(const float* __restrict__ xy, const float* __restrict__ w,
                   const Panel<float>* __restrict__ pan32, const Panel<double>* __restrict__ pan64,
                   int P, Bins b, float nf, float near2, double ec2, double ed2,
                   double* __restrict__ out) {
  __shared__ int queue[kNearWarps][64];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x * kNearWarps + wib;
  if (p >= P) return;          // whole warps exit together
  int* qu = queue[wib];
  const Panel<float> pf = pan32[p];
  const Panel<double> q = pan64[p];
  int x0, x1, y0, y1;
  panel_cells(pf, nf, b.G, x0, x1, y0, y1);
  double acc[11];
  for (int k = 0; k < 11; ++k) acc[k] = 0.0;
  int queued = 0;
  auto drain = [&](int cnt) {
    if (lane < cnt) {
      const int i = qu[lane];
      near_adj_pair<SAME>(q, xy[2 * i], xy[2 * i + 1], w[3 * i], w[3 * i + 1], w[3 * i + 2], ec2,
                          ed2, acc);
    }
  };
  for (int cy = y0; cy <= y1; ++cy)
    for (int cx = x0; cx <= x1; ++cx) {
      const int cell = cy * b.G + cx;
      const int beg = b.start[cell], end = b.start[cell + 1];
      for (int k0 = beg; k0 < end; k0 += 32) {
        const int k = k0 + lane;
        int i = -1;
        bool nr = false;
        if (k < end) {
          i = b.items[k];
          nr = near_pair(pf, xy[2 * i], xy[2 * i + 1], near2);
        }
        const unsigned m = __ballot_sync(0xffffffffu, nr);
        if (nr) qu[queued + __popc(m & ((1u << lane) - 1u))] = i;
        queued += __popc(m);
        __syncwarp();
        if (queued >= 32) {
          drain(32);
          __syncwarp();
          if (lane < queued - 32) qu[lane] = qu[32 + lane];
          queued -= 32;
          __syncwarp();
        }
      }
    }
  drain(queued);
  for (int o = 16; o; o >>= 1)
    for (int k = 0; k < 11; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  if (lane == 0)
    for (int k = 0; k < 11; ++k) out[(size_t)p * 11 + k] = acc[k];
}

// the tables of dlog and datan2_ypos on this context's device, built before
// their first use
static void dmath_ready(bem_ctx* c) {
  if (!c->dmath_ready) {
    k_dmath_init<<<1, kDlogTab > kDatanTab ? kDlogTab : kDatanTab, 0, S(c)>>>();
    BEM_LAUNCHED(c);
    c->dmath_ready = true;
  }
}

static int near_forward_t(bem_ctx* c, int64_t n, const float* xy, double* out, bool subf) {
  int rc;
  Bins b;
  if (!c->pbins_valid) {
    if ((rc = build_bins(c, c->nearP, true, 0, nullptr, b))) return rc;
    c->pbins_valid = true;
  }
  {
    // the panel bins live at the head of nearP with G = 256
    const int G = 256, ncell = G * G, nb = (ncell + 1 + 2047) / 2048;
    b.G = G;
    b.start = (int*)c->nearP.p;
    b.items = (int*)((char*)c->nearP.p + sizeof(int) * ((size_t)ncell + 1 + ncell + nb + 1));
  }

  dmath_ready(c);
  const float near2 = (float)(c->opts.near_factor * c->opts.near_factor);
  const double ec2 = c->opts.eps_c * c->opts.eps_c, ed2 = c->opts.eps_d * c->opts.eps_d;
  ProfScope _ps(c, "k_near_forward");
  const unsigned grid = (unsigned)((n + 127) / 128);
  const bool same = c->opts.eps_c == c->opts.eps_d;
#define BEM_NEAR_FW(SM_, SUB_) \
  k_near_forward<SM_, SUB_><<<grid, 128, 0, S(c)>>>(xy, n, c->d_pan32, c->d_pan64, b, near2, ec2, ed2, out)
  if (same) { if (subf) BEM_NEAR_FW(true, true); else BEM_NEAR_FW(true, false); }
  else { if (subf) BEM_NEAR_FW(false, true); else BEM_NEAR_FW(false, false); }
#undef BEM_NEAR_FW
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "near forward");
}

int near_forward(bem_ctx* c, int64_t n, const float* xy, double* out) {
  return near_forward_t(c, n, xy, out, false);
}

int near_forward_minus_float(bem_ctx* c, int64_t n, const float* xy, double* out) {
  return near_forward_t(c, n, xy, out, true);
}

int near_adjoint(bem_ctx* c, int64_t n, const float* xy, const float* w, double* out) {
  int rc;
  Bins b;
  if ((rc = build_bins(c, c->nearS, false, n, xy, b))) return rc;
  const int P = c->sc.P;
  const float nf = (float)c->opts.near_factor, near2 = nf * nf;
  const double ec2 = c->opts.eps_c * c->opts.eps_c, ed2 = c->opts.eps_d * c->opts.eps_d;
  dmath_ready(c);
  ProfScope _ps(c, "k_near_adjoint");
  if (c->opts.eps_c == c->opts.eps_d)
    k_near_adjoint<true><<<(P + kNearWarps - 1) / kNearWarps, 32 * kNearWarps, 0, S(c)>>>(
        xy, w, c->d_pan32, c->d_pan64, P, b, nf, near2, ec2, ed2, out);
  else
    k_near_adjoint<false><<<(P + kNearWarps - 1) / kNearWarps, 32 * kNearWarps, 0, S(c)>>>(
        xy, w, c->d_pan32, c->d_pan64, P, b, nf, near2, ec2, ed2, out);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "near adjoint");
}

__global__ void k_dlog_eval(int64_t n, const double* __restrict__ x, double* __restrict__ own,
                            double* __restrict__ ref) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    own[i] = dlog(x[i], g_dlog_tab);
    ref[i] = log(x[i]);
  }
}

__global__ void k_datan2_eval(int64_t n, const double* __restrict__ y, const double* __restrict__ x,
                              double* __restrict__ own, double* __restrict__ ref) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    own[i] = datan2_ypos(y[i], x[i], g_datan_tab);
    ref[i] = atan2(y[i], x[i]);
  }
}

}  // namespace bem

extern "C" int bem_datan2_eval(bem_ctx* c, int64_t n, const double* y, const double* x,
                               double* out_lib, double* out_ref, void* stream) {
  using namespace bem;
  if (!c) return BEM_EINVAL;
  if (n < 0 || (n > 0 && (!y || !x || !out_lib || !out_ref)))
    return fail(c, BEM_EINVAL, "bem_datan2_eval: bad arguments");
  int rc;
  if ((rc = ctx_set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  dmath_ready(c);
  if (n > 0) {
    k_datan2_eval<<<(unsigned)((n + 255) / 256), 256, 0, S(c)>>>(n, y, x, out_lib, out_ref);
    BEM_LAUNCHED(c);
  }
  return cuda_check(c, cudaGetLastError(), "k_datan2_eval");
}

extern "C" int bem_dlog_eval(bem_ctx* c, int64_t n, const double* x, double* out_lib,
                             double* out_ref, void* stream) {
  using namespace bem;
  if (!c) return BEM_EINVAL;
  if (n < 0 || (n > 0 && (!x || !out_lib || !out_ref)))
    return fail(c, BEM_EINVAL, "bem_dlog_eval: bad arguments");
  int rc;
  if ((rc = ctx_set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  dmath_ready(c);
  if (n > 0) {
    k_dlog_eval<<<(unsigned)((n + 255) / 256), 256, 0, S(c)>>>(n, x, out_lib, out_ref);
    BEM_LAUNCHED(c);
  }
  return cuda_check(c, cudaGetLastError(), "k_dlog_eval");
}
