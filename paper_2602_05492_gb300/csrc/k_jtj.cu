// Gauss-Newton matrix H = (1/n) sum_s sum_c J_{s,c}^T J_{s,c} (Eq. (losshessian)).
//
// Colour channel c of the colour at x depends on the positions of all control
// points and on channel c's jumps only, so J_{s,c} has n_c = 16 C non-zero
// entries; H is assembled from three n_c x n_c blocks H_c.
//
// J_{s,c} = phi_s^T M_c + F_{s,c}  (Sec. 3.2.3):
//   phi_s[j]  = phi_j(x_s)/(2 pi)          boundary double layer at the sample
//   M_c       = A^+ df_b,c/dtheta          stacked right-hand sides, solved once per step
//   F_{s,c}   = df_c(x_s)/dtheta           handle-term derivatives (Bernstein chain rule)
// Samples are processed in chunks; J rows exist only for the current chunk.
// Column order inside a channel: position x, y of control handle h at 2h, 2h+1;
// w_d,c of h at 8C + h; w_c,c of h at 12C + h.
#include <algorithm>
#include <cmath>

#include "ctx.h"

namespace bem {

template <typename T>
__global__ void k_phi_rows(const T* __restrict__ xy, int ns, const T* __restrict__ vert, int Nb,
                           double* __restrict__ phi) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ns * Nb) return;
  int s = (int)(t / Nb), j = (int)(t % Nb);
  T x = xy[2 * s], y = xy[2 * s + 1];
  T a = seg_angle(vert[2 * j], vert[2 * j + 1], vert[2 * j + 2], vert[2 * j + 3], x, y);
  phi[(size_t)s * Nb + j] = double(a) * kInv2Pi;
}

// F rows of ns points for one curve per blockIdx.y: out F[c][s][nc].
template <typename T, bool SAME>
__global__ void k_frows(const T* __restrict__ xy, int ns, const Panel<T>* __restrict__ pan,
                        const int* __restrict__ off, const int* __restrict__ Kc,
                        const uint8_t* __restrict__ closed, int C, T ec2, T ed2,
                        double* __restrict__ F) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (s >= ns) return;
  int nc = 16 * C, K = Kc[i];
  T x = xy[2 * s], y = xy[2 * s + 1];
  T pos[4][2][3];
  T cd[4], cs[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    cd[j] = 0; cs[j] = 0;
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
      for (int c = 0; c < 3; ++c) pos[j][e][c] = 0;
  }
  for (int k = 0; k < K; ++k) {
    const Panel<T> p = pan[off[i] + k];
    T t0 = T(k) / T(K), t1 = T(k + 1) / T(K), tm = (T(k) + T(0.5)) / T(K);
    T wa[4], wb[4], wm[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) { wa[j] = bern3(j, t0); wb[j] = bern3(j, t1); wm[j] = bern3(j, tm); }
    Frame<T> f = frame(p, x, y);
    LayerGrad<T> g = layer_grad(f, ec2, ed2, SAME);
#pragma unroll
    for (int j = 0; j < 4; ++j) { cd[j] -= wm[j] * g.Dl; cs[j] += wm[j] * g.S; }
    if (!(p.L > T(0))) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T Ft1 = -p.wd[c] * g.D_t1 + p.wc[c] * g.S_t1;
      T Ft2 = -p.wd[c] * g.D_t2 + p.wc[c] * g.S_t2;
      T Fh = -p.wd[c] * g.D_h + p.wc[c] * g.S_h;
      T dax, day, dbx, dby;
      frame_to_endpoints(p, f, Ft1, Ft2, Fh, dax, day, dbx, dby);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        pos[j][0][c] += wa[j] * dax + wb[j] * dbx;
        pos[j][1][c] += wa[j] * day + wb[j] * dby;
      }
    }
  }
  if (closed[i]) {
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
      for (int c = 0; c < 3; ++c) { pos[0][e][c] += pos[3][e][c]; pos[3][e][c] = 0; }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double* row = F + ((size_t)c * ns + s) * nc;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int h = 4 * i + j;
      row[2 * h] = double(pos[j][0][c]);
      row[2 * h + 1] = double(pos[j][1][c]);
      row[8 * C + h] = double(cd[j]);
      row[12 * C + h] = double(cs[j]);
    }
  }
}

// Df[c][i][col] = |G_i| sum_k w_k Fg[c][3i+k][col]
__global__ void k_df_reduce(const double* __restrict__ Fg, int Nb, int nc,
                            const double* __restrict__ vert, double* __restrict__ Df) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y, c = blockIdx.z;
  if (col >= nc) return;
  double ex = vert[2 * (i + 1)] - vert[2 * i], ey = vert[2 * (i + 1) + 1] - vert[2 * i + 1];
  double ell = sqrt(ex * ex + ey * ey);
  size_t n3 = 3 * (size_t)Nb;
  double s = 0;
  for (int q = 0; q < 3; ++q) s += gauss_weight(q) * Fg[((size_t)c * n3 + 3 * i + q) * nc + col];
  Df[((size_t)c * Nb + i) * nc + col] = ell * s;
}

// H[a][b] = scale * sum_c Hc[c][col_c(a)][col_c(b)] over channels where both are active
__global__ void k_h_assemble(const double* __restrict__ Hc, int C, double scale,
                             double* __restrict__ H) {
  int nth = 32 * C, nc = 16 * C;
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  int a = blockIdx.y;
  if (b >= nth) return;
  auto col = [&](int t, int c) {
    int h = t / 8, comp = t % 8;
    if (comp < 2) return 2 * h + comp;
    if (comp < 5) return comp - 2 == c ? 8 * C + h : -1;
    return comp - 5 == c ? 12 * C + h : -1;
  };
  double s = 0;
  for (int c = 0; c < 3; ++c) {
    int ca = col(a, c), cb = col(b, c);
    if (ca >= 0 && cb >= 0) s += Hc[((size_t)c * nc + ca) * nc + cb];
  }
  H[(size_t)a * nth + b] = scale * s;
}

template <typename T>
static void launch_frows(bem_ctx* c, const T* xy, int ns, double* F) {
  int C = c->sc.C;
  dim3 grid((ns + 127) / 128, C);
  const Panel<T>* pan =
      (const Panel<T>*)(sizeof(T) == 8 ? (const void*)c->d_pan64 : (const void*)c->d_pan32);
  T ec2 = T(c->opts.eps_c * c->opts.eps_c), ed2 = T(c->opts.eps_d * c->opts.eps_d);
  ProfScope _ps(c, "k_frows");
  if (c->opts.eps_c == c->opts.eps_d)
    k_frows<T, true><<<grid, 128, 0, S(c)>>>(xy, ns, pan, c->sc.d_off, c->sc.d_K, c->sc.d_closed,
                                             C, ec2, ed2, F);
  else
    k_frows<T, false><<<grid, 128, 0, S(c)>>>(xy, ns, pan, c->sc.d_off, c->sc.d_K, c->sc.d_closed,
                                              C, ec2, ed2, F);
  BEM_LAUNCHED(c);
}

template <typename T>
static int jtj_t(bem_ctx* c, int64_t n, const T* xy, double* Hout) {
  int rc;
  int C = c->sc.C, nc = 16 * C, Nb = c->bd.Nb, nth = c->sc.nth;
  // stacked right-hand sides: F at the boundary Gauss points -> Df -> M_c = A^+ Df_c
  int n3 = 3 * Nb;
  if ((rc = grow(c, c->Fg, sizeof(double) * 3 * (size_t)n3 * nc))) return rc;
  if ((rc = grow(c, c->Dfc, sizeof(double) * 3 * (size_t)Nb * nc))) return rc;
  if ((rc = grow(c, c->Mc, sizeof(double) * 3 * (size_t)Nb * nc))) return rc;
  if ((rc = grow(c, c->Hc, sizeof(double) * 3 * (size_t)nc * nc))) return rc;
  const T* gp = (const T*)(sizeof(T) == 8 ? (const void*)c->bd.d_gp : (const void*)c->bd.d_gp32);
  launch_frows<T>(c, gp, n3, (double*)c->Fg.p);
  k_df_reduce<<<dim3((nc + 127) / 128, Nb, 3), 128, 0, S(c)>>>((const double*)c->Fg.p, Nb, nc,
                                                                c->bd.d_vert, (double*)c->Dfc.p);
  BEM_LAUNCHED(c);
  double* Mc = (double*)c->Mc.p;
  double* Df = (double*)c->Dfc.p;
  for (int ch = 0; ch < 3; ++ch)
    la_dgemm(c, false, false, Nb, nc, Nb, 1.0, c->bd.d_W, Nb, Df + (size_t)ch * Nb * nc, nc, 0.0,
             Mc + (size_t)ch * Nb * nc, nc);
  // chunks of samples
  size_t per = sizeof(double) * ((size_t)Nb + 3 * (size_t)nc);
  int64_t ns = std::max<int64_t>(128, std::min<int64_t>(n, (int64_t)((512u << 20) / per)));
  ns = std::min<int64_t>(ns, 32768);
  if ((rc = grow(c, c->jrow, per * (size_t)ns))) return rc;
  double* phi = (double*)c->jrow.p;
  double* F = phi + (size_t)ns * Nb;
  double* Hc = (double*)c->Hc.p;
  const T* vert = (const T*)(sizeof(T) == 8 ? (const void*)c->bd.d_vert : (const void*)c->bd.d_vert32);
  if ((rc = cuda_check(c, cudaMemsetAsync(Hc, 0, sizeof(double) * 3 * (size_t)nc * nc, S(c)),
                       "memset")))
    return rc;
  for (int64_t s0 = 0; s0 < n; s0 += ns) {
    int m = (int)std::min<int64_t>(ns, n - s0);
    {
      ProfScope _pp(c, "k_phi_rows");
      k_phi_rows<T><<<(unsigned)(((int64_t)m * Nb + 255) / 256), 256, 0, S(c)>>>(xy + 2 * s0, m,
                                                                                    vert, Nb, phi);
      BEM_LAUNCHED(c);
    }
    launch_frows<T>(c, xy + 2 * s0, m, F);
    ProfScope _pg(c, "jtj_gemm");
    for (int ch = 0; ch < 3; ++ch) {
      double* Fc = F + (size_t)ch * m * nc;
      la_dgemm(c, false, false, m, nc, Nb, 1.0, phi, Nb, Mc + (size_t)ch * Nb * nc, nc, 1.0, Fc,
               nc);
      la_dgemm(c, true, false, nc, nc, m, 1.0, Fc, nc, Fc, nc, 1.0, Hc + (size_t)ch * nc * nc, nc);
    }
  }
  k_h_assemble<<<dim3((nth + 127) / 128, nth), 128, 0, S(c)>>>(Hc, C, n > 0 ? 1.0 / double(n) : 0.0,
                                                                Hout);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "jtj");
}

int jtj_build(bem_ctx* c, int64_t n, const void* xy, double* H) {
  if (c->opts.precision == BEM_FP64) return jtj_t<double>(c, n, (const double*)xy, H);
  return jtj_t<float>(c, n, (const float*)xy, H);
}

}  // namespace bem
