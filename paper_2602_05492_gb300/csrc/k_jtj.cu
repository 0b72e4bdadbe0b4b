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
#include <cuda_bf16.h>

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

// F rows of ns points for one curve per blockIdx.y.  TR = false: double
// F[c][s][nc]; TR = true: float F^T[c*nc + col][s] with row stride ldf.
template <typename T, bool SAME, bool TR>
__global__ void k_frows(const T* __restrict__ xy, int ns, const Panel<T>* __restrict__ pan,
                        const int* __restrict__ off, const int* __restrict__ Kc,
                        const uint8_t* __restrict__ closed, int C, T ec2, T ed2,
                        void* __restrict__ Fout, int ldf) {
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
  if (TR) {
    float* F = (float*)Fout;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float* base = F + (size_t)c * nc * ldf + s;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int h = 4 * i + j;
        base[(size_t)(2 * h) * ldf] = float(pos[j][0][c]);
        base[(size_t)(2 * h + 1) * ldf] = float(pos[j][1][c]);
        base[(size_t)(8 * C + h) * ldf] = float(cd[j]);
        base[(size_t)(12 * C + h) * ldf] = float(cs[j]);
      }
    }
    return;
  }
  double* F = (double*)Fout;
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

// bf16 rows phi_j(x_s)/(2 pi): Phi[s][j], row stride Nb
__global__ void k_phi_rows_bf16(const float* __restrict__ xy, int ns, const float* __restrict__ vert,
                                int Nb, __nv_bfloat16* __restrict__ phi) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ns * Nb) return;
  int s = (int)(t / Nb), j = (int)(t % Nb);
  float a = seg_angle(vert[2 * j], vert[2 * j + 1], vert[2 * j + 2], vert[2 * j + 3], xy[2 * s],
                      xy[2 * s + 1]);
  phi[t] = __float2bfloat16_rn(a * float(kInv2Pi));
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// tf32 hi/lo split of phi_j(x_s)/(2 pi): hi[s][j], lo[s][j]
__global__ void k_phi_rows_x3(const float* __restrict__ xy, int ns, const float* __restrict__ vert,
                              int Nb, float* __restrict__ hi, float* __restrict__ lo) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ns * Nb) return;
  int s = (int)(t / Nb), j = (int)(t % Nb);
  float a = seg_angle(vert[2 * j], vert[2 * j + 1], vert[2 * j + 2], vert[2 * j + 3], xy[2 * s],
                      xy[2 * s + 1]) *
            float(kInv2Pi);
  float h = tf32_round(a);
  hi[t] = h;
  lo[t] = tf32_round(a - h);
}

// tf32 hi/lo split of Mt[c*nc + col][j] = Mc[c][j][col]
__global__ void k_mt_x3(const double* __restrict__ Mc, int Nb, int nc, float* __restrict__ hi,
                        float* __restrict__ lo) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int row = blockIdx.y;
  if (j >= Nb) return;
  int c = row / nc, col = row % nc;
  double v = Mc[((size_t)c * Nb + j) * nc + col];
  float h = tf32_round((float)v);
  hi[(size_t)row * Nb + j] = h;
  lo[(size_t)row * Nb + j] = tf32_round((float)(v - (double)h));
}

// Mt[c*nc + col][j] = bf16(Mc[c][j][col])
__global__ void k_mt_bf16(const double* __restrict__ Mc, int Nb, int nc,
                          __nv_bfloat16* __restrict__ Mt) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int row = blockIdx.y;             // c*nc + col
  if (j >= Nb) return;
  int c = row / nc, col = row % nc;
  Mt[(size_t)row * Nb + j] = __float2bfloat16_rn((float)Mc[((size_t)c * Nb + j) * nc + col]);
}

// Hc[c][i][j] = sum over splits of part[split][c][i][j] (upper blocks) in
// fixed order, mirrored to the lower triangle
__global__ void k_syrk_reduce(const float* __restrict__ part, int splits, int nc,
                              double* __restrict__ Hc) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y, c = blockIdx.z;
  if (j >= nc) return;
  int a = min(i, j), b = max(i, j);
  // a block (ti, tj) with ti <= tj holds entry (a, b) when a's tile <= b's tile
  size_t off = ((size_t)c * nc + a) * nc + b;
  if ((a / 128) > (b / 128)) off = ((size_t)c * nc + b) * nc + a;
  double s = 0;
  size_t stride = (size_t)3 * nc * nc;
  for (int k = 0; k < splits; ++k) s += (double)part[k * stride + off];
  Hc[((size_t)c * nc + i) * nc + j] = s;
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

template <typename T, bool TR = false>
static void launch_frows(bem_ctx* c, const T* xy, int ns, void* F, int ldf = 0) {
  int C = c->sc.C;
  dim3 grid((ns + 127) / 128, C);
  const Panel<T>* pan =
      (const Panel<T>*)(sizeof(T) == 8 ? (const void*)c->d_pan64 : (const void*)c->d_pan32);
  T ec2 = T(c->opts.eps_c * c->opts.eps_c), ed2 = T(c->opts.eps_d * c->opts.eps_d);
  ProfScope _ps(c, "k_frows");
  if (c->opts.eps_c == c->opts.eps_d)
    k_frows<T, true, TR><<<grid, 128, 0, S(c)>>>(xy, ns, pan, c->sc.d_off, c->sc.d_K,
                                                 c->sc.d_closed, C, ec2, ed2, F, ldf);
  else
    k_frows<T, false, TR><<<grid, 128, 0, S(c)>>>(xy, ns, pan, c->sc.d_off, c->sc.d_K,
                                                  c->sc.d_closed, C, ec2, ed2, F, ldf);
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

// Stacked right-hand sides M_c = A^+ df_b,c/dtheta in double (shared by both paths).
template <typename T>
static int jtj_stacked_rhs(bem_ctx* c) {
  int rc;
  int C = c->sc.C, nc = 16 * C, Nb = c->bd.Nb, n3 = 3 * Nb;
  if ((rc = grow(c, c->Fg, sizeof(double) * 3 * (size_t)n3 * nc))) return rc;
  if ((rc = grow(c, c->Dfc, sizeof(double) * 3 * (size_t)Nb * nc))) return rc;
  if ((rc = grow(c, c->Mc, sizeof(double) * 3 * (size_t)Nb * nc))) return rc;
  const T* gp = (const T*)(sizeof(T) == 8 ? (const void*)c->bd.d_gp : (const void*)c->bd.d_gp32);
  launch_frows<T>(c, gp, n3, c->Fg.p);
  k_df_reduce<<<dim3((nc + 127) / 128, Nb, 3), 128, 0, S(c)>>>((const double*)c->Fg.p, Nb, nc,
                                                                c->bd.d_vert, (double*)c->Dfc.p);
  BEM_LAUNCHED(c);
  double* Mc = (double*)c->Mc.p;
  double* Df = (double*)c->Dfc.p;
  for (int ch = 0; ch < 3; ++ch)
    la_dgemm(c, false, false, Nb, nc, Nb, 1.0, c->bd.d_W, Nb, Df + (size_t)ch * Nb * nc, nc, 0.0,
             Mc + (size_t)ch * Nb * nc, nc);
  return cuda_check(c, cudaGetLastError(), "stacked rhs");
}

// Mixed precision: J^T rows and the Gram blocks on the tensor cores, either
// in bf16 (fp32 accumulate) or in the 3xtf32 split; Gram blocks accumulate
// per K slice in fp32 and the slices are summed in double.
static int jtj_tc(bem_ctx* c, int64_t n, const float* xy, double* Hout, bool x3) {
  int rc;
  int C = c->sc.C, nc = 16 * C, Nb = c->bd.Nb, nth = c->sc.nth;
  if ((rc = jtj_stacked_rhs<float>(c))) return rc;
  const size_t es = x3 ? 2 * sizeof(float) : sizeof(__nv_bfloat16);   // bytes per element (all parts)
  // M_c^T, [3 nc][Nb]
  const size_t mt_part = (x3 ? 4 : 2) * 3 * (size_t)nc * Nb;
  if ((rc = grow(c, c->tcMt, es * 3 * (size_t)nc * Nb))) return rc;
  const void* Mt[2] = {c->tcMt.p, (char*)c->tcMt.p + mt_part};
  if (x3)
    k_mt_x3<<<dim3((Nb + 127) / 128, 3 * nc), 128, 0, S(c)>>>((const double*)c->Mc.p, Nb, nc,
                                                               (float*)Mt[0], (float*)Mt[1]);
  else
    k_mt_bf16<<<dim3((Nb + 127) / 128, 3 * nc), 128, 0, S(c)>>>((const double*)c->Mc.p, Nb, nc,
                                                                 (__nv_bfloat16*)Mt[0]);
  BEM_LAUNCHED(c);
  // per-chunk buffers: Phi [m][Nb], F^T f32 [3nc][ld], J^T [3nc][ld]
  const int64_t chunk = std::min<int64_t>(std::max<int64_t>(n, 1), 262144);
  const int ld = (int)((chunk + 63) / 64 * 64);
  const size_t phi_part = (x3 ? 4 : 2) * (size_t)chunk * Nb;
  const size_t phi_b = (x3 ? 2 : 1) * phi_part;
  const size_t f_b = sizeof(float) * 3 * (size_t)nc * ld;
  const size_t j_part = (x3 ? 4 : 2) * 3 * (size_t)nc * ld;
  const size_t j_b = (x3 ? 2 : 1) * j_part;
  if ((rc = grow(c, c->jrow, phi_b + 256 + f_b + 256))) return rc;
  if ((rc = grow(c, c->tcJ, j_b))) return rc;
  const int splits = tc_syrk_splits(nc, x3);
  const size_t part_b = sizeof(float) * (size_t)splits * 3 * nc * nc;
  if ((rc = grow(c, c->tcPart, part_b))) return rc;
  if ((rc = grow(c, c->Hc, sizeof(double) * 3 * (size_t)nc * nc))) return rc;
  const void* phi[2] = {c->jrow.p, (char*)c->jrow.p + phi_part};
  float* F = (float*)((char*)c->jrow.p + (phi_b + 255) / 256 * 256);
  void* J[2] = {c->tcJ.p, (char*)c->tcJ.p + j_part};
  float* part = (float*)c->tcPart.p;
  if ((rc = cuda_check(c, cudaMemsetAsync(part, 0, part_b, S(c)), "memset"))) return rc;
  if ((rc = cuda_check(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), S(c)), "memset"))) return rc;
  for (int64_t s0 = 0; s0 < n; s0 += chunk) {
    const int m = (int)std::min<int64_t>(chunk, n - s0);
    {
      ProfScope _pp(c, "k_phi_rows");
      const unsigned blocks = (unsigned)(((int64_t)m * Nb + 255) / 256);
      if (x3)
        k_phi_rows_x3<<<blocks, 256, 0, S(c)>>>(xy + 2 * s0, m, c->bd.d_vert32, Nb,
                                                (float*)phi[0], (float*)phi[1]);
      else
        k_phi_rows_bf16<<<blocks, 256, 0, S(c)>>>(xy + 2 * s0, m, c->bd.d_vert32, Nb,
                                                  (__nv_bfloat16*)phi[0]);
      BEM_LAUNCHED(c);
    }
    launch_frows<float, true>(c, xy + 2 * s0, m, F, ld);
    if ((rc = tc_jrows(c, x3, 3 * nc, m, Nb, Mt, Nb, phi, Nb, F, ld, J, ld))) return rc;
    const void* Jc[2] = {J[0], J[1]};
    if ((rc = tc_syrk(c, x3, nc, m, Jc, ld, part, splits))) return rc;
  }
  k_syrk_reduce<<<dim3((nc + 127) / 128, nc, 3), 128, 0, S(c)>>>(part, splits, nc,
                                                                  (double*)c->Hc.p);
  k_h_assemble<<<dim3((nth + 127) / 128, nth), 128, 0, S(c)>>>((const double*)c->Hc.p, C,
                                                                n > 0 ? 1.0 / double(n) : 0.0, Hout);
  c->launches += 2;
  if ((rc = cuda_check(c, cudaGetLastError(), "jtj tc"))) return rc;
  int st = 0;
  if ((rc = cuda_check(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                                          S(c)), "status")) ||
      (rc = cuda_check(c, cudaStreamSynchronize(S(c)), "sync")))
    return rc;
  if (st) return fail(c, BEM_ETIMEDOUT, "tensor-core J^T J: a bounded device wait ran out");
  return BEM_OK;
}

int jtj_build(bem_ctx* c, int64_t n, const void* xy, double* H) {
  if (c->opts.precision == BEM_FP64) return jtj_t<double>(c, n, (const double*)xy, H);
  if (c->opts.jtj_mode == BEM_JTJ_BF16) return jtj_tc(c, n, (const float*)xy, H, false);
  if (c->opts.jtj_mode == BEM_JTJ_3XTF32) return jtj_tc(c, n, (const float*)xy, H, true);
  return jtj_t<float>(c, n, (const float*)xy, H);
}

}  // namespace bem
