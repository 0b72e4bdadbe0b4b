// Regularisers of segment handles (Sec. 4.4), pruning, and the quasi-random
// initialisation of Sec. 4.2.
//
// theta[h][10] = (a_x, a_y, b_x, b_y, w_d RGB, w_c RGB).  Endpoint e = 2h + s
// is a_h (s = 0) or b_h (s = 1), at theta[10h + 2s ..].  The three losses:
//   length    lw (|b - a| - lmax)^2 where |b - a| > lmax
//   snapping  sw |p - q|^2 over endpoint pairs of different handles closer
//             than r that choose each other by the lowest score
//             alpha |p - q| / r + (1 - alpha)(1 - |u_p . u_q|)
//             (u = unit handle direction; ties go to the lower index)
//   sparsity  lam t tanh(sqrt(w.w + eps^2) / t), w = w_d (lam_d), w_c (lam_c)
// Their analytic gradients and Hessians are added to the Gauss-Newton g and
// H of the LM step (Eq. (optimstep)); the snapping pairs are chosen once per
// step, at the current parameters.  The sparsity Hessian is taken with its
// saturation factor sech^2(rho/t) held fixed, lam s (I/rho - w w^T/rho^3):
// the exact Hessian adds -lam s (2 tanh(rho/t)/(t rho^2)) w w^T, negative
// curvature that can make diagonal entries of H negative, and then
// H + lambda diag(H) does not factor for any damping.
#include <cmath>
#include <vector>

#include "ctx.h"

namespace bem {

namespace {

__device__ __forceinline__ void handle_dir(const double* th, int h, double& ux, double& uy) {
  const double dx = th[10 * h + 2] - th[10 * h], dy = th[10 * h + 3] - th[10 * h + 1];
  const double ln = hypot(dx, dy);
  ux = ln > 0 ? dx / ln : 0.0;
  uy = ln > 0 ? dy / ln : 0.0;
}

// best[p] = the endpoint p chooses (or -1); one thread per endpoint, the
// candidates streamed through shared memory in blocks of 256
constexpr int kSnapTile = 256;

__global__ void __launch_bounds__(kSnapTile) k_snap_best(const double* __restrict__ th, int H,
                                                         double r, double alpha,
                                                         int* __restrict__ best) {
  __shared__ double sx[kSnapTile], sy[kSnapTile], su[kSnapTile], sv[kSnapTile];
  const int E = 2 * H;
  const int p = blockIdx.x * kSnapTile + threadIdx.x;
  double px = 0, py = 0, ux = 0, uy = 0;
  if (p < E) {
    px = th[10 * (p / 2) + 2 * (p % 2)];
    py = th[10 * (p / 2) + 2 * (p % 2) + 1];
    handle_dir(th, p / 2, ux, uy);
  }
  double bs = INFINITY;
  int bq = -1;
  for (int q0 = 0; q0 < E; q0 += kSnapTile) {
    __syncthreads();
    const int q = q0 + threadIdx.x;
    if (q < E) {
      sx[threadIdx.x] = th[10 * (q / 2) + 2 * (q % 2)];
      sy[threadIdx.x] = th[10 * (q / 2) + 2 * (q % 2) + 1];
      double a, b;
      handle_dir(th, q / 2, a, b);
      su[threadIdx.x] = a;
      sv[threadIdx.x] = b;
    }
    __syncthreads();
    if (p >= E) continue;
    const int n = min(kSnapTile, E - q0);
    for (int k = 0; k < n; ++k) {
      const int qq = q0 + k;
      if (qq / 2 == p / 2) continue;
      const double dist = hypot(px - sx[k], py - sy[k]);
      if (!(dist < r)) continue;
      const double cs = fabs(ux * su[k] + uy * sv[k]);
      const double s = alpha * dist / r + (1.0 - alpha) * (1.0 - cs);
      if (s < bs) { bs = s; bq = qq; }
    }
  }
  if (p < E) best[p] = bq;
}

// length and sparsity terms: one thread per handle, g and the handle's own
// 10 x 10 diagonal block of H (row stride n)
__global__ void k_reg_local(const double* __restrict__ th, int H, bem_reg rp, double* __restrict__ g,
                            double* __restrict__ Hm, int n) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  const double* t = th + 10 * (size_t)h;
  double* gh = g + 10 * (size_t)h;
  double* Hh = Hm + (size_t)(10 * h) * n + 10 * h;   // block origin
  if (rp.len_weight > 0) {
    const double ex = t[2] - t[0], ey = t[3] - t[1];
    const double ln = hypot(ex, ey), k = ln - rp.len_max;
    if (k > 0) {
      const double u[2] = {ex / ln, ey / ln};
      const double lam = rp.len_weight;
      for (int i = 0; i < 2; ++i) {
        const double gb = 2.0 * lam * k * u[i];
        gh[i] -= gb;
        gh[2 + i] += gb;
        for (int j = 0; j < 2; ++j) {
          const double M = 2.0 * lam * (u[i] * u[j] + (k / ln) * ((i == j ? 1.0 : 0.0) - u[i] * u[j]));
          Hh[(size_t)i * n + j] += M;
          Hh[(size_t)(2 + i) * n + 2 + j] += M;
          Hh[(size_t)i * n + 2 + j] -= M;
          Hh[(size_t)(2 + i) * n + j] -= M;
        }
      }
    }
  }
  for (int which = 0; which < 2; ++which) {
    const double lam = which == 0 ? rp.sparse_wd : rp.sparse_wc;
    if (!(lam > 0)) continue;
    const int off = which == 0 ? 4 : 7;
    const double* w = t + off;
    const double tt = rp.sparse_t;
    const double rho = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + rp.sparse_eps * rp.sparse_eps);
    const double th_ = tanh(rho / tt);
    const double s = 1.0 - th_ * th_;
    for (int i = 0; i < 3; ++i) {
      gh[off + i] += lam * s * w[i] / rho;
      for (int j = 0; j < 3; ++j) {
        const double ww = w[i] * w[j];
        Hh[(size_t)(off + i) * n + off + j] +=
            lam * s * ((i == j ? 1.0 : 0.0) / rho - ww / (rho * rho * rho));
      }
    }
  }
}

__device__ __forceinline__ bool snap_pair(const int* best, int p, int& q) {
  q = best[p];
  return q > p && best[q] == p;
}

// snapping terms: one thread per endpoint p that heads a mutual pair (p < q);
// an endpoint belongs to at most one pair, so no two threads share entries
__global__ void k_reg_snap(const double* __restrict__ th, int H, double lam,
                           const int* __restrict__ best, double* __restrict__ g,
                           double* __restrict__ Hm, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  int q;
  if (p >= 2 * H || !snap_pair(best, p, q)) return;
  const int ip = 10 * (p / 2) + 2 * (p % 2), iq = 10 * (q / 2) + 2 * (q % 2);
  for (int i = 0; i < 2; ++i) {
    const double d = 2.0 * lam * (th[ip + i] - th[iq + i]);
    g[ip + i] += d;
    g[iq + i] -= d;
    Hm[(size_t)(ip + i) * n + ip + i] += 2.0 * lam;
    Hm[(size_t)(iq + i) * n + iq + i] += 2.0 * lam;
    Hm[(size_t)(ip + i) * n + iq + i] -= 2.0 * lam;
    Hm[(size_t)(iq + i) * n + ip + i] -= 2.0 * lam;
  }
}

// total regulariser loss at th with the given pairs: one block, fixed order
__global__ void __launch_bounds__(1024) k_reg_loss(const double* __restrict__ th, int H, bem_reg rp,
                                                   const int* __restrict__ best,
                                                   double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0;
  for (int h = threadIdx.x; h < H; h += blockDim.x) {
    const double* t = th + 10 * (size_t)h;
    if (rp.len_weight > 0) {
      const double k = hypot(t[2] - t[0], t[3] - t[1]) - rp.len_max;
      if (k > 0) acc += rp.len_weight * k * k;
    }
    if (rp.snap_weight > 0 && best) {
      for (int s = 0; s < 2; ++s) {
        int q;
        if (snap_pair(best, 2 * h + s, q)) {
          const int iq = 10 * (q / 2) + 2 * (q % 2);
          const double dx = t[2 * s] - th[iq], dy = t[2 * s + 1] - th[iq + 1];
          acc += rp.snap_weight * (dx * dx + dy * dy);
        }
      }
    }
    for (int which = 0; which < 2; ++which) {
      const double lam = which == 0 ? rp.sparse_wd : rp.sparse_wc;
      if (!(lam > 0)) continue;
      const double* w = t + (which == 0 ? 4 : 7);
      const double rho = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + rp.sparse_eps * rp.sparse_eps);
      acc += lam * rp.sparse_t * tanh(rho / rp.sparse_t);
    }
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) *out = v;
  }
}

// keep[h] = 0 if |w_d,h| < thr and |w_c,h| < thr
__global__ void k_prune_flags(const double* __restrict__ th, int H, double thr, int* __restrict__ keep) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  const double* t = th + 10 * (size_t)h;
  const double nd = sqrt(t[4] * t[4] + t[5] * t[5] + t[6] * t[6]);
  const double nc = sqrt(t[7] * t[7] + t[8] * t[8] + t[9] * t[9]);
  keep[h] = (nd < thr && nc < thr) ? 0 : 1;
}

// order-preserving compaction of the kept handles: one block scans the flags
// in chunks of 1024; out receives the kept parameters, idx their old indices,
// count the number kept
__global__ void __launch_bounds__(1024) k_prune_compact(const double* __restrict__ th, int H,
                                                        const int* __restrict__ keep,
                                                        double* __restrict__ out,
                                                        int* __restrict__ idx, int* __restrict__ count) {
  __shared__ int wsum[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  for (int h0 = 0; h0 < H; h0 += 1024) {
    const int h = h0 + threadIdx.x;
    const int f = h < H ? keep[h] : 0;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    const int before = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < 32; ++w) {
      if (w < warp) off += wsum[w];
      tot += wsum[w];
    }
    if (f) {
      const int d = base + off + before;
      idx[d] = h;
      for (int e = 0; e < 10; ++e) out[10 * (size_t)d + e] = th[10 * (size_t)h + e];
    }
    __syncthreads();
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

}  // namespace

bool reg_active(const bem_ctx* c) {
  const bem_reg& r = c->reg;
  return c->sc.pp == 4 &&
         (r.len_weight > 0 || r.snap_weight > 0 || r.sparse_wd > 0 || r.sparse_wc > 0);
}

int reg_pairs(bem_ctx* c, const double* theta) {
  if (!(c->reg.snap_weight > 0)) return BEM_OK;
  const int H = c->sc.NH, E = 2 * H;
  int rc;
  if ((rc = grow(c, c->regw, sizeof(int) * (size_t)E))) return rc;
  k_snap_best<<<(E + kSnapTile - 1) / kSnapTile, kSnapTile, 0, S(c)>>>(
      theta, H, c->reg.snap_radius, c->reg.snap_alpha, (int*)c->regw.p);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "k_snap_best");
}

int reg_add(bem_ctx* c, const double* theta, double* H, double* g) {
  const int Hn = c->sc.NH, n = c->sc.nth;
  k_reg_local<<<(Hn + 127) / 128, 128, 0, S(c)>>>(theta, Hn, c->reg, g, H, n);
  BEM_LAUNCHED(c);
  if (c->reg.snap_weight > 0) {
    k_reg_snap<<<(2 * Hn + 127) / 128, 128, 0, S(c)>>>(theta, Hn, c->reg.snap_weight,
                                                       (const int*)c->regw.p, g, H, n);
    BEM_LAUNCHED(c);
  }
  return cuda_check(c, cudaGetLastError(), "k_reg_add");
}

int reg_loss(bem_ctx* c, const double* theta, double* d_out) {
  k_reg_loss<<<1, 1024, 0, S(c)>>>(theta, c->sc.NH, c->reg,
                                   c->reg.snap_weight > 0 ? (const int*)c->regw.p : nullptr, d_out);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "k_reg_loss");
}

int reg_prune(bem_ctx* c, double thr, std::vector<double>& kept_theta, std::vector<int>& kept_idx) {
  const int H = c->sc.NH;
  int rc;
  // flags [H] | indices [H] | count, then the compacted parameters
  const size_t ioff = 0, doff = ((sizeof(int) * (2 * (size_t)H + 1) + 255) / 256) * 256;
  if ((rc = grow(c, c->regw, doff + sizeof(double) * 10 * (size_t)H))) return rc;
  int* keep = (int*)c->regw.p + ioff;
  int* idx = keep + H;
  int* cnt = idx + H;
  double* out = (double*)((char*)c->regw.p + doff);
  k_prune_flags<<<(H + 255) / 256, 256, 0, S(c)>>>(c->d_theta, H, thr, keep);
  BEM_LAUNCHED(c);
  k_prune_compact<<<1, 1024, 0, S(c)>>>(c->d_theta, H, keep, out, idx, cnt);
  BEM_LAUNCHED(c);
  int n = 0;
  if ((rc = cuda_check(c, cudaGetLastError(), "prune")) ||
      (rc = cuda_check(c, cudaMemcpyAsync(&n, cnt, sizeof(int), cudaMemcpyDeviceToHost, S(c)), "count")) ||
      (rc = cuda_check(c, cudaStreamSynchronize(S(c)), "sync")))
    return rc;
  kept_theta.assign(10 * (size_t)n, 0.0);
  kept_idx.assign(n, 0);
  if (n == 0) return BEM_OK;
  if ((rc = cuda_check(c, cudaMemcpyAsync(kept_theta.data(), out, sizeof(double) * 10 * (size_t)n,
                                          cudaMemcpyDeviceToHost, S(c)), "theta")) ||
      (rc = cuda_check(c, cudaMemcpyAsync(kept_idx.data(), idx, sizeof(int) * (size_t)n,
                                          cudaMemcpyDeviceToHost, S(c)), "indices")))
    return rc;
  return cuda_check(c, cudaStreamSynchronize(S(c)), "sync");
}

}  // namespace bem

// ---- initialisation (host) --------------------------------------------------------

namespace {

// Point k of the two-dimensional Sobol sequence in Gray-code order: the XOR of
// the direction numbers of the set bits of k ^ (k >> 1).  Coordinate 1 has
// direction numbers 2^-j; coordinate 2 those of the primitive polynomial
// x + 1 with m_1 = 1, i.e. m_j = m_{j-1} xor 2 m_{j-1}.
void sobol2(uint64_t k, double& x, double& y) {
  const uint64_t g = k ^ (k >> 1);
  uint64_t X = 0, Y = 0, m = 1;
  for (int j = 1; j <= 52; ++j) {
    if (j > 1) m = m ^ (m << 1);
    if ((g >> (j - 1)) & 1u) {
      X ^= uint64_t(1) << (52 - j);
      Y ^= m << (52 - j);
    }
    if ((g >> j) == 0) break;
  }
  x = std::ldexp(double(X), -52);
  y = std::ldexp(double(Y), -52);
}

double radical_inverse3(uint64_t k) {
  double x = 0.0, f = 1.0 / 3.0;
  while (k > 0) {
    x += double(k % 3) * f;
    k /= 3;
    f /= 3.0;
  }
  return x;
}

bool inside(double x, double y, const double* poly, int V) {
  bool in = false;
  for (int i = 0; i < V; ++i) {
    const double x0 = poly[2 * i], y0 = poly[2 * i + 1];
    const double x1 = poly[2 * ((i + 1) % V)], y1 = poly[2 * ((i + 1) % V) + 1];
    if ((y0 > y) != (y1 > y)) {
      const double xc = x0 + (y - y0) * (x1 - x0) / (y1 - y0);
      if (x < xc) in = !in;
    }
  }
  return in;
}

double first_crossing(double ax, double ay, double bx, double by, const double* poly, int V) {
  double t_hit = 1.0;
  const double dx = bx - ax, dy = by - ay;
  for (int i = 0; i < V; ++i) {
    const double px = poly[2 * i], py = poly[2 * i + 1];
    const double ex = poly[2 * ((i + 1) % V)] - px, ey = poly[2 * ((i + 1) % V) + 1] - py;
    const double den = dx * ey - dy * ex;
    if (den == 0.0) continue;
    const double wx = px - ax, wy = py - ay;
    const double t = (wx * ey - wy * ex) / den, s = (wx * dy - wy * dx) / den;
    if (t > 0.0 && t <= t_hit && s >= 0.0 && s <= 1.0) t_hit = t;
  }
  return t_hit;
}

}  // namespace

extern "C" {

int bem_init_segments(int n_points, double length, int64_t first_index, int n_vertices,
                      const double* vertices, double* theta_out, int* n_handles) {
  if (n_points < 0 || !(length >= 0) || !std::isfinite(length) || first_index < 0 ||
      (vertices && n_vertices < 3) || (n_points > 0 && !theta_out) || !n_handles)
    return BEM_EINVAL;
  static const double sq[8] = {0, 0, 1, 0, 1, 1, 0, 1};
  const double* poly = vertices ? vertices : sq;
  const int V = vertices ? n_vertices : 4;
  int m = 0;
  for (int j = 0; j < n_points; ++j) {
    const uint64_t k = uint64_t(first_index) + uint64_t(j);
    double ax, ay;
    sobol2(k, ax, ay);
    if (!inside(ax, ay, poly, V)) continue;
    const double phi = 2.0 * M_PI * radical_inverse3(k);
    double bx = ax + length * std::cos(phi), by = ay + length * std::sin(phi);
    const double t = first_crossing(ax, ay, bx, by, poly, V);
    bx = ax + t * (bx - ax);
    by = ay + t * (by - ay);
    double* th = theta_out + 10 * (size_t)m;
    th[0] = ax; th[1] = ay; th[2] = bx; th[3] = by;
    for (int e = 4; e < 10; ++e) th[e] = 0.0;
    ++m;
  }
  *n_handles = m;
  return BEM_OK;
}

}  // extern "C"
