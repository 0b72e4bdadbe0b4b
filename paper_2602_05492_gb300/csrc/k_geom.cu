// Geometry kernels: curves -> panels, compatibility projection, the image
// boundary and its Galerkin matrix.
#include <cmath>

#include "ctx.h"

namespace bem {

// Panel p of curve i (index k of K) has endpoints B(k/K), B((k+1)/K) of the
// cubic Bezier through the curve's four control points (a closed curve uses
// its first point as its last) and jumps interpolated with the Bernstein
// weights at the mid-parameter (k+1/2)/K.
// Segment handles (pp = 4): panel p is handle p, (a, b, w_d, w_c) directly.
__global__ void k_panelize(const double* __restrict__ theta, const int* __restrict__ pcurve,
                           const int* __restrict__ pk, const int* __restrict__ Kc,
                           const uint8_t* __restrict__ closed, int P, int pp,
                           Panel<double>* out64, Panel<float>* out32) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double ax = 0, ay = 0, bx = 0, by = 0;
  double wd[3] = {0, 0, 0}, wc[3] = {0, 0, 0};
  if (pp == 4) {
    const double* th = theta + (size_t)p * 10;
    ax = th[0]; ay = th[1]; bx = th[2]; by = th[3];
    for (int c = 0; c < 3; ++c) { wd[c] = th[4 + c]; wc[c] = th[7 + c]; }
  } else {
    int i = pcurve[p], k = pk[p], K = Kc[i];
    const double* th = theta + (size_t)i * 32;
    double t0 = double(k) / K, t1 = double(k + 1) / K, tm = (k + 0.5) / K;
    for (int j = 0; j < 4; ++j) {
      int jg = (closed[i] && j == 3) ? 0 : j;
      double px = th[jg * 8 + 0], py = th[jg * 8 + 1];
      double w0 = bern3(j, t0), w1 = bern3(j, t1), wm = bern3(j, tm);
      ax += w0 * px; ay += w0 * py;
      bx += w1 * px; by += w1 * py;
      for (int c = 0; c < 3; ++c) {
        wd[c] += wm * th[j * 8 + 2 + c];
        wc[c] += wm * th[j * 8 + 5 + c];
      }
    }
  }
  double ex = bx - ax, ey = by - ay;
  double L = sqrt(ex * ex + ey * ey);
  Panel<double> q;
  q.ax = ax; q.ay = ay;
  q.L = L;
  q.tx = L > 0 ? ex / L : 0.0;
  q.ty = L > 0 ? ey / L : 0.0;
  for (int c = 0; c < 3; ++c) { q.wd[c] = wd[c]; q.wc[c] = wc[c]; }
  q.pad = 0;
  out64[p] = q;
  Panel<float> r;
  r.ax = float(ax); r.ay = float(ay);
  r.tx = float(q.tx); r.ty = float(q.ty); r.L = float(L);
  for (int c = 0; c < 3; ++c) { r.wd[c] = float(wd[c]); r.wc[c] = float(wc[c]); }
  r.pad = 0;
  out32[p] = r;
}

// a_h = sum_k length_k B_j((k+1/2)/K) over the panels of h's curve (a
// segment handle: its length), then w_c <- w_c - a (a.w_c)/(a.a) per
// channel (compatibility, Sec. 3.1.2 and the re-projection of Sec. 4.3).
// One block of up to 1,024 threads (a warp per owner for the panel sums);
// colour owner h has its w_c at theta[h (pp + 6) + pp + 3 + c].
__global__ void k_compat(double* __restrict__ theta, const Panel<double>* __restrict__ pan,
                         const int* __restrict__ off, const int* __restrict__ Kc, int C, int pp,
                         double* __restrict__ a_out, int project) {
  extern __shared__ double sh[];   // [owners] a
  const int H = pp == 4 ? C : 4 * C, stride = pp + 6, wco = pp + 3;
  double* a = sh;
  {
    const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int h = threadIdx.x >> 5; h < H; h += nwarp) {
      double s = 0;
      if (pp == 4) {
        s = lane == 0 ? pan[h].L : 0.0;
      } else {
        const int i = h / 4, j = h % 4, K = Kc[i];
        for (int k = lane; k < K; k += 32) s += pan[off[i] + k].L * bern3(j, (k + 0.5) / K);
      }
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        a[h] = s;
        if (a_out) a_out[h] = s;
      }
    }
  }
  __syncthreads();
  if (!project) return;
  __shared__ double red[4][32];
  double v[4] = {0, 0, 0, 0};
  for (int h = threadIdx.x; h < H; h += blockDim.x) {
    v[0] += a[h] * a[h];
    for (int c = 0; c < 3; ++c) v[1 + c] += a[h] * theta[h * stride + wco + c];
  }
  for (int o = 16; o; o >>= 1)
    for (int q = 0; q < 4; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  int w = threadIdx.x / 32, l = threadIdx.x % 32, nw = blockDim.x / 32;
  if (l == 0)
    for (int q = 0; q < 4; ++q) red[q][w] = v[q];
  __syncthreads();
  __shared__ double tot[4];
  if (threadIdx.x < 4) {
    double s = 0;
    for (int k = 0; k < nw; ++k) s += red[threadIdx.x][k];
    tot[threadIdx.x] = s;
  }
  __syncthreads();
  if (tot[0] <= 0) return;
  for (int h = threadIdx.x; h < H; h += blockDim.x)
    for (int c = 0; c < 3; ++c) theta[h * stride + wco + c] -= a[h] * tot[1 + c] / tot[0];
}

// A_ij = |G_i| sum_q w_q I_j(x_iq), A_ii = |G_i| / 2 (the coincident
// double-layer term of a straight segment vanishes), Eq. (bie_galerkin), with
// the inner integral I_j(x) of dG/dn_y over segment j
//   mode 0: exact, -phi_j(x)/(2 pi) (the signed angle of the segment at x);
//   mode 1: 3-point Gauss, -(|G_j|/2pi) sum_q' w_q' n_j.(y_jq' - x)/|y_jq' - x|^2
//           with n_j the right normal (the paper's 3 x 3 rule).
__global__ void k_assemble(const double* __restrict__ vert, const double* __restrict__ gp, int Nb,
                           int mode, double* __restrict__ A) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (j >= Nb) return;
  double ex = vert[2 * (i + 1)] - vert[2 * i], ey = vert[2 * (i + 1) + 1] - vert[2 * i + 1];
  double ell = sqrt(ex * ex + ey * ey);
  if (i == j) {
    A[(size_t)i * Nb + j] = 0.5 * ell;
    return;
  }
  double ax = vert[2 * j], ay = vert[2 * j + 1], bx = vert[2 * (j + 1)], by = vert[2 * (j + 1) + 1];
  double s = 0;
  if (mode == 0) {
    for (int q = 0; q < 3; ++q)
      s += gauss_weight(q) * seg_angle(ax, ay, bx, by, gp[2 * (3 * i + q)], gp[2 * (3 * i + q) + 1]);
    A[(size_t)i * Nb + j] = -ell * s * kInv2Pi;
    return;
  }
  const double lj = sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
  const double nx = (by - ay) / lj, ny = -(bx - ax) / lj;     // right normal
  for (int q = 0; q < 3; ++q) {
    const double x = gp[2 * (3 * i + q)], y = gp[2 * (3 * i + q) + 1];
    double in = 0;
    for (int p = 0; p < 3; ++p) {
      const double t = gauss_node(p);
      const double dx = ax + t * (bx - ax) - x, dy = ay + t * (by - ay) - y;
      const double r2 = dx * dx + dy * dy;
      if (r2 > 0) in += gauss_weight(p) * (nx * dx + ny * dy) / r2;
    }
    s += gauss_weight(q) * in;
  }
  A[(size_t)i * Nb + j] = -ell * lj * s * kInv2Pi;
}

int geom_panelize(bem_ctx* c, const double* d_theta) {
  int P = c->sc.P;
  c->pbins_valid = false;
  k_panelize<<<(P + 127) / 128, 128, 0, S(c)>>>(d_theta, c->sc.d_pcurve, c->sc.d_pk, c->sc.d_K,
                                                c->sc.d_closed, P, c->sc.pp, c->d_pan64,
                                                c->d_pan32);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "k_panelize");
}

int geom_compat(bem_ctx* c, double* d_theta, bool project) {
  int C = c->sc.C;
  size_t shm = sizeof(double) * c->sc.NH;
  if (shm > 48 * 1024) return fail(c, BEM_EINVAL, "too many handles for the compatibility kernel");
  // a re-projection leaves the step's weights (those of theta, which every
  // trial's constrained solve uses) as they are
  k_compat<<<1, 1024, shm, S(c)>>>(d_theta, c->d_pan64, c->sc.d_off, c->sc.d_K, C, c->sc.pp,
                                   project ? nullptr : c->d_compat, project ? 1 : 0);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "k_compat");
}

int geom_boundary_tables(bem_ctx* c) {
  // the unit square, or the context's polygon; each edge cut into M equal segments
  static const double sq[8] = {0, 0, 1, 0, 1, 1, 0, 1};
  const std::vector<double> poly =
      c->bd.poly.empty() ? std::vector<double>(sq, sq + 8) : c->bd.poly;
  const int V = (int)poly.size() / 2, M = c->bd.M, Nb = V * M;
  std::vector<double> v(2 * (Nb + 1)), g(2 * 3 * Nb);
  for (int e = 0; e < V; ++e) {
    const double ax = poly[2 * e], ay = poly[2 * e + 1];
    const double bx = poly[2 * ((e + 1) % V)], by = poly[2 * ((e + 1) % V) + 1];
    for (int m = 0; m < M; ++m) {
      const double t = double(m) / M;
      v[2 * (e * M + m)] = ax + (bx - ax) * t;
      v[2 * (e * M + m) + 1] = ay + (by - ay) * t;
    }
  }
  v[2 * Nb] = v[0];
  v[2 * Nb + 1] = v[1];
  for (int i = 0; i < Nb; ++i)
    for (int q = 0; q < 3; ++q) {
      double gq = gauss_node(q);
      g[2 * (3 * i + q)] = v[2 * i] + gq * (v[2 * (i + 1)] - v[2 * i]);
      g[2 * (3 * i + q) + 1] = v[2 * i + 1] + gq * (v[2 * (i + 1) + 1] - v[2 * i + 1]);
    }
  std::vector<float> v32(v.begin(), v.end()), g32(g.begin(), g.end());
  int rc;
  if ((rc = cuda_check(c, cudaMemcpy(c->bd.d_vert, v.data(), v.size() * 8, cudaMemcpyHostToDevice),
                       "vertices")))
    return rc;
  if ((rc = cuda_check(c, cudaMemcpy(c->bd.d_gp, g.data(), g.size() * 8, cudaMemcpyHostToDevice),
                       "gauss points")))
    return rc;
  if ((rc = cuda_check(c, cudaMemcpy(c->bd.d_vert32, v32.data(), v32.size() * 4,
                                     cudaMemcpyHostToDevice), "vertices")))
    return rc;
  return cuda_check(c, cudaMemcpy(c->bd.d_gp32, g32.data(), g32.size() * 4, cudaMemcpyHostToDevice),
                    "gauss points");
}

int geom_assemble(bem_ctx* c) {
  int Nb = c->bd.Nb;
  dim3 grid((Nb + 127) / 128, Nb);
  k_assemble<<<grid, 128, 0, S(c)>>>(c->bd.d_vert, c->bd.d_gp, Nb, c->opts.galerkin_mode,
                                     c->bd.d_A);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "k_assemble");
}

}  // namespace bem
