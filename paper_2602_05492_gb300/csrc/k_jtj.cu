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

// Channel and per-channel column of J^T row r of the J-row layout, or -1 for
// a padding row: position rows belong to their channel, the jump rows (the
// same in every channel) are taken from channel 0.
__device__ __forceinline__ int jrow_col(const JLayout& L, int r, int& ch) {
  if (r < 3 * L.Pp) {
    ch = r / L.Pp;
    const int col = r - ch * L.Pp;
    return col < L.npos ? col : -1;
  }
  ch = 0;
  const int w = r - 3 * L.Pp;
  return w < 2 * L.nh ? L.npos + w : -1;
}

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
// F[c][s][nc]; TR = true: float F^T rows in the J-row layout (JLayout: the
// position columns per channel at rows c Pp + col, the jump columns once, at
// rows 3 Pp + h and 3 Pp + NH + h), row stride ldf.
// Panel k of the curve runs from vertex k to vertex k+1 (vertex v = B(v/K)),
// so the endpoint derivatives are first summed per vertex (panel k's start
// plus panel k-1's end) and then spread to the control points with the
// Bernstein weights B_j(v/K).  Each block stages its curve's panels, with
// these weights and the mid-parameter ones, in shared memory, kFrowsTable
// panels at a time.
constexpr int kFrowsTable = 128;

// One (point, panel) pair of the F rows: the two layer values and the
// endpoint derivatives (a then b, x then y) of Dl and S.  iL as in
// chain_endpoints.  The double path returns them as they are; the float
// path returns them multiplied by -2 pi (layer_grad_hat), which the kernels
// undo once per output entry.
template <typename T, bool SAME>
__device__ __forceinline__ void frows_pair(T ax, T ay, T tx, T ty, T L, T iL, T x, T y, T ec2,
                                           T ed2, T& Dl, T& S, T (&Dd)[4], T (&Sd)[4]) {
  if constexpr (sizeof(T) == 4) {
    const Frame<float> f = frame_rn(ax, ay, tx, ty, L, x, y);
    const GradHat g = layer_grad_hat(f, f.h * f.h, ec2, ed2, SAME);
    Dl = g.D;
    S = g.S;
    chain_endpoints(tx, ty, iL, f, g.Dt1, g.Dt2, g.Dh, Dd);
    chain_endpoints(tx, ty, iL, f, g.St1, g.St2, g.Sh, Sd);
  } else {
    Frame<T> f;
    const T dax = ax - x, day = ay - y;
    f.t1 = dax * tx + day * ty;
    f.h = dax * ty - day * tx;
    f.L = L;
    f.t2 = f.t1 + L;
    const LayerGrad<T> g = layer_grad(f, ec2, ed2, SAME);
    Dl = g.Dl;
    S = g.S;
    chain_endpoints(tx, ty, iL, f, g.D_t1, g.D_t2, g.D_h, Dd);
    chain_endpoints(tx, ty, iL, f, g.S_t1, g.S_t2, g.S_h, Sd);
  }
}

// A panel of the block's curve as k_frows stages it in shared memory: the
// frame data, iL, the jumps with the handle term's signs folded in
// (a = -w_d, b = w_c) and the Bernstein weights of the panel's start vertex
// (wv) and midpoint (wm).
template <typename T>
struct __align__(16) FrowsPanel {
  T ax, ay, tx, ty;
  T L, iL, a[3], b[3];
  T wv[4], wm[4];
};

// With hw (float path only) the block also writes its curve's share of the
// handle term at theta, hw[(c C + i) ldh + s] = sum over the curve's four
// colour owners of F_c[s][w_d col] w_d,c + F_c[s][w_c col] w_c,c, from the
// float values it stores in F^T and the jumps of theta (owner h at
// theta[8 h + 2 .. 8 h + 7]).  The colour is linear in the jumps, so these
// shares summed over the curves are the handle term of the colour.
template <typename T, bool SAME, bool TR>
__global__ void __launch_bounds__(128, 6) k_frows(const T* __restrict__ xy, int ns, const Panel<T>* __restrict__ pan,
                        const int* __restrict__ off, const int* __restrict__ Kc,
                        const uint8_t* __restrict__ closed, int C, T ec2, T ed2,
                        void* __restrict__ Fout, int ldf, int Pp, const double* __restrict__ theta,
                        float* __restrict__ hw, int ldh) {
  __shared__ FrowsPanel<T> tab[kFrowsTable];
  // the float pair values carry a factor -2 pi (frows_pair)
  constexpr T kOut = sizeof(T) == 4 ? T(-kInv2Pi) : T(1);
  const int i = blockIdx.y;
  const int K = Kc[i];
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = s < ns;
  const int nc = 16 * C;
  const T x = live ? xy[2 * s] : T(0), y = live ? xy[2 * s + 1] : T(0);
  T pos[4][2][3];
  T cd[4], cs[4];
  T carry[2][3];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    cd[j] = 0; cs[j] = 0;
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
      for (int c = 0; c < 3; ++c) pos[j][e][c] = 0;
  }
#pragma unroll
  for (int e = 0; e < 2; ++e)
#pragma unroll
    for (int c = 0; c < 3; ++c) carry[e][c] = 0;
  const Panel<T>* cp = pan + off[i];
  for (int k0 = 0; k0 < K; k0 += kFrowsTable) {
    const int cnt = min(K - k0, kFrowsTable);
    __syncthreads();   // every thread is done with the previous table
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const Panel<T> p = cp[k0 + e];
      const int k = k0 + e;
      FrowsPanel<T> r;
      r.ax = p.ax; r.ay = p.ay; r.tx = p.tx; r.ty = p.ty;
      r.L = p.L;
      r.iL = inv_len(p.L);
#pragma unroll
      for (int c = 0; c < 3; ++c) { r.a[c] = -p.wd[c]; r.b[c] = p.wc[c]; }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        r.wv[j] = bern3(j, T(k) / T(K));
        r.wm[j] = bern3(j, (T(k) + T(0.5)) / T(K));
      }
      tab[e] = r;
    }
    __syncthreads();
    if (!live) continue;
#pragma unroll (sizeof(T) == 4 ? 2 : 1)
    for (int e = 0; e < cnt; ++e) {
      const FrowsPanel<T>& r = tab[e];
      T Dl, S, Dd[4], Sd[4];
      frows_pair<T, SAME>(r.ax, r.ay, r.tx, r.ty, r.L, r.iL, x, y, ec2, ed2, Dl, S, Dd, Sd);
#pragma unroll
      for (int j = 0; j < 4; ++j) { cd[j] = fma(-r.wm[j], Dl, cd[j]); cs[j] = fma(r.wm[j], S, cs[j]); }
      // vertex k: start of panel k and end of panel k-1
#pragma unroll
      for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
          const T v = fma(r.a[c], Dd[e2], fma(r.b[c], Sd[e2], carry[e2][c]));
          carry[e2][c] = fma(r.a[c], Dd[2 + e2], r.b[c] * Sd[2 + e2]);
#pragma unroll
          for (int j = 0; j < 4; ++j) pos[j][e2][c] = fma(r.wv[j], v, pos[j][e2][c]);
        }
      }
    }
  }
  if (!live) return;
  // vertex K = B(1) = control point 3
#pragma unroll
  for (int e = 0; e < 2; ++e)
#pragma unroll
    for (int c = 0; c < 3; ++c) pos[3][e][c] += carry[e][c];
  if (closed[i]) {
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
      for (int c = 0; c < 3; ++c) { pos[0][e][c] += pos[3][e][c]; pos[3][e][c] = 0; }
  }
  if (TR) {
    float* F = (float*)Fout + s;
    float fd[4], fs[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int h = 4 * i + j;
      fd[j] = float(kOut * cd[j]);
      fs[j] = float(kOut * cs[j]);
      F[(size_t)(3 * Pp + h) * ldf] = fd[j];            // jump columns, once for all channels
      F[(size_t)(3 * Pp + 4 * C + h) * ldf] = fs[j];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float* base = F + (size_t)c * Pp * ldf;
      float t = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int h = 4 * i + j;
        base[(size_t)(2 * h) * ldf] = float(kOut * pos[j][0][c]);
        base[(size_t)(2 * h + 1) * ldf] = float(kOut * pos[j][1][c]);
        if (hw) {
          t = fmaf(fd[j], float(theta[8 * h + 2 + c]), t);
          t = fmaf(fs[j], float(theta[8 * h + 5 + c]), t);
        }
      }
      if (hw) hw[((size_t)c * C + i) * ldh + s] = t;
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
      row[2 * h] = double(kOut * pos[j][0][c]);
      row[2 * h + 1] = double(kOut * pos[j][1][c]);
      row[8 * C + h] = double(kOut * cd[j]);
      row[12 * C + h] = double(kOut * cs[j]);
    }
  }
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// One operand value in the scheme's format at element o: bf16; or the high
// part rounded to tf32 (fp32 storage) or bf16 and the low part the rounded
// rest, x = hi + lo
template <int SCH>
__device__ __forceinline__ void put_operand(void* p0, void* p1, size_t o, float x) {
  if constexpr (SCH == SCH_TF32X3) {
    const float h = tf32_round(x);
    ((float*)p0)[o] = h;
    ((float*)p1)[o] = tf32_round(x - h);
  } else if constexpr (SCH == SCH_BF16X3) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    ((__nv_bfloat16*)p0)[o] = h;
    ((__nv_bfloat16*)p1)[o] = __float2bfloat16_rn(x - __bfloat162float(h));
  } else {
    ((__nv_bfloat16*)p0)[o] = __float2bfloat16_rn(x);
  }
}

// Phi rows of a chunk of samples written from the segment side: thread j
// (boundary segment) walks the block's sample slice, writes phi_j(x_s)/(2 pi)
// into row s (in the scheme's operand format) and, when residuals are given, sums
// q_j += phi_j(x_s)/(2 pi) r_s into a per-slice double partial qpart[slice][j][3].
template <int SCH>
__global__ void __launch_bounds__(128) k_phi_q(const float* __restrict__ xy, const float* __restrict__ r,
                                               int m, int slice_len, const float* __restrict__ vert,
                                               int Nb, void* __restrict__ phi0,
                                               void* __restrict__ phi1, double* __restrict__ qpart) {
  __shared__ float4 sxr[128];   // x, y, r0, r1 of the slice's samples
  __shared__ float sr2[128];     // r2
  const int j = blockIdx.x * 128 + threadIdx.x;
  const int s0 = blockIdx.y * slice_len, s1 = min(m, s0 + slice_len);
  const bool live = j < Nb;
  float ax = 0, ay = 0, bx = 0, by = 0;
  if (live) { ax = vert[2 * j]; ay = vert[2 * j + 1]; bx = vert[2 * j + 2]; by = vert[2 * j + 3]; }
  double q0 = 0, q1 = 0, q2 = 0;
  for (int base = s0; base < s1; base += 128) {
    const int cnt = min(128, s1 - base);
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const int s = base + threadIdx.x;
      sxr[threadIdx.x] = make_float4(xy[2 * s], xy[2 * s + 1], r ? r[3 * s] : 0.f,
                                     r ? r[3 * s + 1] : 0.f);
      sr2[threadIdx.x] = r ? r[3 * s + 2] : 0.f;
    }
    __syncthreads();
    if (!live) continue;
    float a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 4
    for (int k = 0; k < cnt; ++k) {
      const float4 p = sxr[k];
      const float phi = seg_angle(ax, ay, bx, by, p.x, p.y) * float(kInv2Pi);
      put_operand<SCH>(phi0, phi1, (size_t)(base + k) * Nb + j, phi);
      if (r) { a0 = fmaf(phi, p.z, a0); a1 = fmaf(phi, p.w, a1); a2 = fmaf(phi, sr2[k], a2); }
    }
    q0 += a0; q1 += a1; q2 += a2;
  }
  if (live && r && qpart) {
    double* o = qpart + ((size_t)blockIdx.y * Nb + j) * 3;
    o[0] = q0; o[1] = q1; o[2] = q2;
  }
}

constexpr int kGemvSegs = 16;   // sample segments per row in k_ft_gemv

// out[t] = sum over k of part[k][t] (fixed order)
// out[t] = sum over k < nparts of part[k m + t]: 32 outputs per block of 32 x
// 32 threads, thread row ty summing k = ty, ty + 32, ...; the 32 row sums
// are added in a fixed order
__global__ void __launch_bounds__(1024) k_sum_rows(const double* __restrict__ part, int nparts,
                                                   int m, double* __restrict__ out) {
  __shared__ double acc[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int t = blockIdx.x * 32 + tx;
  double s = 0;
  if (t < m)
    for (int k = ty; k < nparts; k += 32) s += part[(size_t)k * m + t];
  acc[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && t < m) {
    double v = 0;
    for (int y = 0; y < 32; ++y) v += acc[y][tx];
    out[t] = v;
  }
}

// out[row] = sum over k of part[row][k] (fixed order; one warp per row)
// out[row] (+)= sum of the float partials part[row stride + k], k < nparts,
// one warp per row in a fixed order: with 16-byte aligned rows, each lane
// adds four consecutive partials in float ((a + b) + (c + d)) and those sums
// in double (a quarter of the double additions, which bound this kernel on
// the FP64 pipe); otherwise every partial in double
__global__ void k_row_sums(const float* __restrict__ part, int rows, int64_t nparts,
                           int64_t stride, bool add, double* __restrict__ out) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const float* p = part + (size_t)row * stride;
  double s = 0;
  int64_t k0 = 0;
  if ((stride & 3) == 0 && ((uintptr_t)part & 15) == 0) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
    const int64_t n4 = nparts >> 2;
    for (int64_t k = lane; k < n4; k += 32) {
      const float4 v = p4[k];
      s += (double)((v.x + v.y) + (v.z + v.w));
    }
    k0 = 4 * n4;
  }
  for (int64_t k = k0 + lane; k < nparts; k += 32) s += (double)p[k];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[row] = add ? out[row] + s : s;
}

// The handle part of the gradient over segment seg of the chunk's samples:
// gpart[seg][c nc + col] = sum_s F^T[row][s] r[s][c] for every J^T row of
// the J-row layout and each channel c whose column col it holds (position
// rows: their channel; jump rows: all three), double accumulation; one warp
// per (row, segment), gridDim.y segments.
__global__ void k_ft_gemv(const float* __restrict__ F, int ldf, JLayout L, int nc, int m,
                          const float* __restrict__ r, double* __restrict__ gpart) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= L.rows()) return;
  int c0 = 0;
  const int col = jrow_col(L, row, c0);
  if (col < 0) return;
  const bool jump = row >= 3 * L.Pp;
  const int seg = (m + gridDim.y - 1) / gridDim.y;
  const int sb = blockIdx.y * seg, se = min(m, sb + seg);
  const float* f = F + (size_t)row * ldf;
  double acc[3] = {0, 0, 0};
  for (int s0 = sb; s0 < se; s0 += 32 * 8) {
    float a[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int s = s0 + u * 32 + lane;
      if (s < se) {
        const float v = f[s];
        if (jump) {
          a[0] += v * r[3 * s]; a[1] += v * r[3 * s + 1]; a[2] += v * r[3 * s + 2];
        } else {
          a[0] += v * r[3 * s + c0];
        }
      }
    }
    for (int k = 0; k < 3; ++k) acc[k] += a[k];
  }
  for (int k = 0; k < 3; ++k)
    for (int o = 16; o; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  if (lane) return;
  double* out = gpart + (size_t)blockIdx.y * 3 * nc;
  if (jump) {
    for (int k = 0; k < 3; ++k) out[(size_t)k * nc + col] = acc[k];
  } else {
    out[(size_t)c0 * nc + col] = acc[0];
  }
}

// g[theta] = scale * sum over channels of (handle part + boundary part) of
// channel-local column col_c(theta); gh[c*nc + col] summed over chunks,
// boundary part gb[c*nc + col] = sum_i Df[c][i][col] lambda[i][c]
__global__ void k_g_boundary(const double* __restrict__ Df, int Nb, int nc,
                             const double* __restrict__ lam, double* __restrict__ gb) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;   // c*nc + col
  const int lane = threadIdx.x & 31;
  if (row >= 3 * nc) return;
  const int c = row / nc, col = row % nc;
  double acc = 0;
  for (int i = lane; i < Nb; i += 32) acc += Df[((size_t)c * Nb + i) * nc + col] * lam[3 * i + c];
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) gb[row] = acc;
}

// Column of parameter t in channel c's block of J (or -1): colour owner
// h = t / (pp + 6) has its pp position entries at pp h + comp (every channel),
// w_d,c at pp NH + h and w_c,c at (pp + 1) NH + h.
__device__ __forceinline__ int param_col(int t, int c, int pp, int NH) {
  const int stride = pp + 6, h = t / stride, comp = t % stride;
  if (comp < pp) return pp * h + comp;
  if (comp < pp + 3) return comp - pp == c ? pp * NH + h : -1;
  return comp - pp - 3 == c ? (pp + 1) * NH + h : -1;
}

__global__ void k_g_assemble(const double* __restrict__ gparts, int nparts, int stride,
                             const double* __restrict__ gb, int pp, int NH, double scale,
                             double* __restrict__ g) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = (pp + 6) * NH, nc = (pp + 2) * NH;
  if (t >= nth) return;
  double s = 0;
  for (int c = 0; c < 3; ++c) {
    const int col = param_col(t, c, pp, NH);
    if (col < 0) continue;
    const int row = c * nc + col;
    double v = gb[row];
    for (int k = 0; k < nparts; ++k) v += gparts[(size_t)k * stride + row];
    s += v;
  }
  g[t] = scale * s;
}

// Hc[c][i][j] (per-channel column order, nc x nc) = sum over splits of the
// Gram entry of channel-order indices (i', j') of channel c (upper blocks,
// part[split][c][cdim][cdim]) in fixed order, mirrored to the lower
// triangle; the jump-jump entries of every channel are channel 0's.
__global__ void k_syrk_reduce(const float* __restrict__ part, int splits, int nc, JLayout L,
                              double* __restrict__ Hc) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y, c = blockIdx.z;
  if (j >= nc) return;
  const int ci = i < L.npos ? i : L.Pp + (i - L.npos);
  const int cj = j < L.npos ? j : L.Pp + (j - L.npos);
  const int a = min(ci, cj), b = max(ci, cj);
  const int D = L.cdim();
  const int src = (a >= L.Pp) ? 0 : c;       // jump-jump blocks: channel 0
  const size_t off = ((size_t)src * D + a) * D + b;
  double s = 0;
  const size_t stride = (size_t)3 * D * D;
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
__global__ void k_h_assemble(const double* __restrict__ Hc, int pp, int NH, double scale,
                             double* __restrict__ H) {
  const int nth = (pp + 6) * NH, nc = (pp + 2) * NH;
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  int a = blockIdx.y;
  if (b >= nth) return;
  double s = 0;
  for (int c = 0; c < 3; ++c) {
    const int ca = param_col(a, c, pp, NH), cb = param_col(b, c, pp, NH);
    if (ca >= 0 && cb >= 0) s += Hc[((size_t)c * nc + ca) * nc + cb];
  }
  H[(size_t)a * nth + b] = scale * s;
}

// F rows of segment handles (the paper's parametrisation, one panel per
// handle): thread = point, blockIdx.y = a run of kSegRun handles.  Columns of
// channel c: a, b of handle h at 4h .. 4h+3, w_d,c at 4H + h, w_c,c at 5H + h.
constexpr int kSegRun = 8;

template <typename T, bool SAME, bool TR>
__global__ void __launch_bounds__(128) k_frows_seg(const T* __restrict__ xy, int ns,
                                                   const Panel<T>* __restrict__ pan, int H, T ec2,
                                                   T ed2, void* __restrict__ Fout, int ldf, int Pp) {
  constexpr T kOut = sizeof(T) == 4 ? T(-kInv2Pi) : T(1);
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const int nc = 6 * H;
  const T x = xy[2 * s], y = xy[2 * s + 1];
  const int h0 = blockIdx.y * kSegRun, h1 = min(H, h0 + kSegRun);
  for (int h = h0; h < h1; ++h) {
    const Panel<T> p = pan[h];
    T Dl, S, Dd[4], Sd[4];
    frows_pair<T, SAME>(p.ax, p.ay, p.tx, p.ty, p.L, inv_len(p.L), x, y, ec2, ed2, Dl, S, Dd, Sd);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T a = -p.wd[c], b = p.wc[c];
      T v[6];
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = kOut * (a * Dd[e] + b * Sd[e]);
      v[4] = -kOut * Dl;
      v[5] = kOut * S;
      const int cols[6] = {4 * h, 4 * h + 1, 4 * h + 2, 4 * h + 3, 4 * H + h, 5 * H + h};
      if (TR) {
        // J-row layout: positions per channel, the jump columns once
        float* F = (float*)Fout + s;
#pragma unroll
        for (int e = 0; e < 4; ++e) F[(size_t)(c * Pp + cols[e]) * ldf] = float(v[e]);
        if (c == 0) {
          F[(size_t)(3 * Pp + h) * ldf] = float(v[4]);
          F[(size_t)(3 * Pp + H + h) * ldf] = float(v[5]);
        }
      } else {
        double* row = (double*)Fout + ((size_t)c * ns + s) * nc;
#pragma unroll
        for (int e = 0; e < 6; ++e) row[cols[e]] = double(v[e]);
      }
    }
  }
}

template <typename T, bool TR = false>
static void launch_frows(bem_ctx* c, const T* xy, int ns, void* F, int ldf = 0,
                         float* hw = nullptr, int ldh = 0) {
  const int Pp = jlayout(c->sc.pp, c->sc.NH).Pp;
  int C = c->sc.C;
  dim3 grid((ns + 127) / 128, C);
  const Panel<T>* pan =
      (const Panel<T>*)(sizeof(T) == 8 ? (const void*)c->d_pan64 : (const void*)c->d_pan32);
  T ec2 = T(c->opts.eps_c * c->opts.eps_c), ed2 = T(c->opts.eps_d * c->opts.eps_d);
  ProfScope _ps(c, "k_frows");
  if (c->sc.pp == 4) {
    const int H = c->sc.NH;
    dim3 gs((ns + 127) / 128, (H + kSegRun - 1) / kSegRun);
    if (c->opts.eps_c == c->opts.eps_d)
      k_frows_seg<T, true, TR><<<gs, 128, 0, S(c)>>>(xy, ns, pan, H, ec2, ed2, F, ldf, Pp);
    else
      k_frows_seg<T, false, TR><<<gs, 128, 0, S(c)>>>(xy, ns, pan, H, ec2, ed2, F, ldf, Pp);
    BEM_LAUNCHED(c);
    return;
  }
  if (c->opts.eps_c == c->opts.eps_d)
    k_frows<T, true, TR><<<grid, 128, 0, S(c)>>>(xy, ns, pan, c->sc.d_off, c->sc.d_K,
                                                 c->sc.d_closed, C, ec2, ed2, F, ldf, Pp,
                                                 c->d_theta, hw, ldh);
  else
    k_frows<T, false, TR><<<grid, 128, 0, S(c)>>>(xy, ns, pan, c->sc.d_off, c->sc.d_K,
                                                  c->sc.d_closed, C, ec2, ed2, F, ldf, Pp,
                                                  c->d_theta, hw, ldh);
  BEM_LAUNCHED(c);
}

template <typename T>
static int jtj_t(bem_ctx* c, int64_t n, const T* xy, double* Hout) {
  int rc;
  int nc = c->sc.nc, Nb = c->bd.Nb, nth = c->sc.nth;
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
  ns = std::min<int64_t>(ns, c->opts.gn_chunk > 0 ? c->opts.gn_chunk : 32768);
  bem_ctx* w = c->scratch ? c->scratch : c;   // owner of the chunk buffers
  if ((rc = grow(c, w->jrow, per * (size_t)ns))) return rc;
  double* phi = (double*)w->jrow.p;
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
  k_h_assemble<<<dim3((nth + 127) / 128, nth), 128, 0, S(c)>>>(Hc, c->sc.pp, c->sc.NH, n > 0 ? 1.0 / double(n) : 0.0,
                                                                Hout);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "jtj");
}

// The A operand of the tensor-core J-row contraction straight from Df:
//   Mt[row][j] = M_c[j][col] = sum_i W[j][i] Df_c[i][col]
// for the channel and column of each J^T row (jrow_col; padding rows 0), in
// fp32 (W = A^+ as float, Df converted on load), 64 x 64 tiles of 4 x 4
// outputs per thread, written in the scheme's operand format.  The result is
// rounded to bf16 / tf32 (or split into two such parts) at once, so fp32
// accumulation loses nothing the J rows keep.
template <int SCH>
__global__ void __launch_bounds__(256) k_mt_sgemm(const float* __restrict__ W,
                                                  const double* __restrict__ Df, int Nb, int nc,
                                                  JLayout L, void* __restrict__ out0,
                                                  void* __restrict__ out1) {
  __shared__ float As[16][64 + 4];   // [k][row of Mt]
  __shared__ float Bs[16][64 + 4];   // [k][j]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int j0 = blockIdx.x * 64, r0 = blockIdx.y * 64;
  const int rows = L.rows();
  float acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
  for (int i0 = 0; i0 < Nb; i0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int kk = e >> 6, rr = e & 63;
      const int r = r0 + rr, i = i0 + kk;
      float v = 0.f;
      int ch = 0;
      const int col = r < rows ? jrow_col(L, r, ch) : -1;
      if (col >= 0 && i < Nb) v = (float)Df[((size_t)ch * Nb + i) * nc + col];
      As[kk][rr] = v;
    }
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int jj = e >> 4, kk = e & 15;
      const int j = j0 + jj, i = i0 + kk;
      Bs[kk][jj] = (j < Nb && i < Nb) ? W[(size_t)j * Nb + i] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int r = r0 + ty * 4 + p;
    if (r >= rows) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + tx * 4 + q;
      if (j >= Nb) continue;
      put_operand<SCH>(out0, out1, (size_t)r * Nb + j, acc[p][q]);
    }
  }
}

// Stacked right-hand sides M_c = A^+ df_b,c/dtheta (Sec. 3.2.3): the F rows
// at the boundary Gauss points reduced to Df_c, then, when `solve` is set,
// the double products M_c = A^+ Df_c (the tensor-core path forms its
// rounded M_c^T itself, k_mt_sgemm).
template <typename T>
static int jtj_stacked_rhs(bem_ctx* c, bool solve = true) {
  int rc;
  int nc = c->sc.nc, Nb = c->bd.Nb, n3 = 3 * Nb;
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
  if (!solve) return cuda_check(c, cudaGetLastError(), "stacked rhs");
  if (!solve) return cuda_check(c, cudaGetLastError(), "stacked rhs");
  for (int ch = 0; ch < 3; ++ch)
    la_dgemm(c, false, false, Nb, nc, Nb, 1.0, c->bd.d_W, Nb, Df + (size_t)ch * Nb * nc, nc, 0.0,
             Mc + (size_t)ch * Nb * nc, nc);
  return cuda_check(c, cudaGetLastError(), "stacked rhs");
}

// Mixed precision: J^T rows and the Gram blocks on the tensor cores, either
// in bf16 (fp32 accumulate) or in the 3xtf32 split; Gram blocks accumulate
// per K slice in fp32 and the slices are summed in double.
// With residuals r (float [n][3]) it also forms the gradient g = (1/n) J^T r
// from the same J rows (Eq. (lossjacobian)): the handle part as a double
// GEMV over F^T per chunk, the boundary part as q^T M_c = (A^+T q)^T Df_c
// with q = sum_s phi_s r_s summed while the Phi rows are written.
// hand[s][c] += sum over the curves i (fixed order) of hw[(c C + i) ldh + s],
// the curves' shares of the handle term at theta that k_frows wrote (hand
// already holds the near-field correction).  Thread = point.
__global__ void __launch_bounds__(256) k_hand_sum(const float* __restrict__ hw, int ldh, int C,
                                                  int m, double* __restrict__ hand) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= m) return;
  for (int c = 0; c < 3; ++c) {
    const float* p = hw + (size_t)c * C * ldh + s;
    // eight independent float partial sums keep eight loads in flight (a
    // partial adds C / 8 shares, a few float roundings of a colour), and
    // only the eight partials are added in double: double adds run at a
    // small fraction of the float rate here
    float t[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int i = 0;
    for (; i + 8 <= C; i += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = p[(size_t)(i + u) * ldh];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] += v[u];
    }
    for (; i < C; ++i) t[0] += p[(size_t)i * ldh];
    double d = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) d += double(t[u]);
    hand[3 * (size_t)s + c] += d;
  }
}

// The residual comes out of the J-row pass when forming the handle term from
// the colour columns of the F rows (a few flops per colour owner and point)
// is cheaper than evaluating every pair again (about 63 flops per panel):
// with more than six panels per colour owner, i.e. Bezier curves of more
// than 24 panels, not for one-panel segment handles.
bool jtj_fuses_eval(const bem_ctx* c) {
  return jtj_gives_gradient(c) && c->sc.P > 6 * c->sc.NH;
}

static int jtj_tc(bem_ctx* c, int64_t n, const float* xy, double* Hout, int sch,
                  const float* resid, double* gout, const float* target) {
  int rc;
  int C = c->sc.C, nc = c->sc.nc, Nb = c->bd.Nb, nth = c->sc.nth;
  const bool want_g = resid && gout;
  // with target the residual at theta is formed here, chunk by chunk, from
  // the F rows (handle term F w), the near-field correction and the
  // boundary term, before the chunk's Phi rows and J rows need it
  const bool fuse_r = want_g && target;
  if (target && !want_g) return fail(c, BEM_EINVAL, "jtj: a target needs the residual and gradient outputs");
  if ((rc = jtj_stacked_rhs<float>(c, false))) return rc;
  // J^T rows: the position columns per channel, the jump columns once (JLayout)
  const JLayout L = jlayout(c->sc.pp, c->sc.NH);
  const int rows = L.rows();
  const bool x3 = sch != SCH_BF16;                  // split operands, three products
  const size_t pb = sch == SCH_TF32X3 ? 4 : 2;      // bytes per element of one part
  const size_t es = (x3 ? 2 : 1) * pb;              // bytes per element (all parts)
  // M^T in the J-row layout, [rows][Nb]
  const size_t mt_part = pb * (size_t)rows * Nb;
  if ((rc = grow(c, c->tcMt, es * (size_t)rows * Nb))) return rc;
  const void* Mt[2] = {c->tcMt.p, (char*)c->tcMt.p + mt_part};
  {
    ProfScope _pm(c, "k_mt_sgemm");
    dim3 grid((Nb + 63) / 64, (rows + 63) / 64);
    const double* Df = (const double*)c->Dfc.p;
    if (sch == SCH_TF32X3)
      k_mt_sgemm<SCH_TF32X3><<<grid, 256, 0, S(c)>>>(c->bd.d_W32, Df, Nb, nc, L, (void*)Mt[0],
                                                     (void*)Mt[1]);
    else if (sch == SCH_BF16X3)
      k_mt_sgemm<SCH_BF16X3><<<grid, 256, 0, S(c)>>>(c->bd.d_W32, Df, Nb, nc, L, (void*)Mt[0],
                                                     (void*)Mt[1]);
    else
      k_mt_sgemm<SCH_BF16><<<grid, 256, 0, S(c)>>>(c->bd.d_W32, Df, Nb, nc, L, (void*)Mt[0],
                                                   nullptr);
    BEM_LAUNCHED(c);
  }
  // per-chunk buffers: Phi [m][Nb], F^T f32 [rows][ld], J^T [rows][ld]
  const int64_t chunk = gn_chunk_tc(c, n);
  const int nchunks = (int)((n + chunk - 1) / chunk);
  const int ld = (int)((chunk + 63) / 64 * 64);
  const size_t phi_part = pb * (size_t)chunk * Nb;
  const size_t phi_b = (x3 ? 2 : 1) * phi_part;
  const size_t f_b = sizeof(float) * (size_t)rows * ld;
  const size_t j_part = pb * (size_t)rows * ld;
  const size_t j_b = (x3 ? 2 : 1) * j_part;
  // gradient work: per chunk handle partial [3nc], q partials per slice
  // sample slices of the Phi-row pass: 1,024 samples each, up to 256 (a
  // 262,144-sample chunk gives 8 x 256 CTAs, enough to fill the SMs to the
  // kernel's register limit of 12 CTAs)
  const int qslices = (int)std::max<int64_t>(1, std::min<int64_t>(256, (chunk + 1023) / 1024));
  // handle part of the gradient: the bf16 and compensated-bf16 J rows form
  // it per 64-sample block of a chunk in their epilogue ([3nc][blocks of the
  // chunk]), summed into [3nc] after each chunk; 3xtf32 runs a GEMV per
  // chunk ([chunks x segs][3nc])
  const bool fused_g = want_g && sch != SCH_TF32X3;
  const int64_t cblk = (chunk + 63) / 64;   // 64-sample blocks of a chunk
  const size_t gh_b = sizeof(double) * (fused_g ? (size_t)cblk * 3 * nc + 3 * (size_t)nc
                                                : (size_t)std::max(nchunks, 1) * kGemvSegs * 3 * nc);
  const size_t q_b = sizeof(double) * (size_t)std::max(nchunks, 1) * qslices * Nb * 3;
  const size_t gb_b = sizeof(double) * 3 * (size_t)nc;
  bem_ctx* w = c->scratch ? c->scratch : c;   // owner of the chunk buffers
  // the curves' shares of the handle term at theta, [3][C][ld]
  const size_t hw_b = fuse_r ? sizeof(float) * 3 * (size_t)C * ld : 0;
  if ((rc = grow(c, w->jrow, phi_b + 256 + f_b + 256 + hw_b + 256))) return rc;
  if ((rc = grow(c, w->tcJ, j_b))) return rc;
  if (want_g && (rc = grow(c, w->gwork, gh_b + q_b + gb_b + 256))) return rc;
  const int splits = tc_syrk_splits(L, x3, c->sms);
  const size_t part_b = sizeof(float) * (size_t)splits * 3 * L.cdim() * L.cdim();
  if ((rc = grow(c, w->tcPart, part_b))) return rc;
  if ((rc = grow(c, c->Hc, sizeof(double) * 3 * (size_t)nc * nc))) return rc;
  const void* phi[2] = {w->jrow.p, (char*)w->jrow.p + phi_part};
  float* F = (float*)((char*)w->jrow.p + (phi_b + 255) / 256 * 256);
  float* hw = fuse_r ? (float*)((char*)F + (f_b + 255) / 256 * 256) : nullptr;
  void* J[2] = {w->tcJ.p, (char*)w->tcJ.p + j_part};
  float* part = (float*)w->tcPart.p;
  double* gh = (double*)w->gwork.p;
  double* qp = gh + gh_b / sizeof(double);
  double* gb = qp + (size_t)std::max(nchunks, 1) * qslices * Nb * 3;
  double* hand = nullptr;
  double* lossp = nullptr;
  int64_t lblk = 0;
  // host inputs (lm_step_host): nothing above reads the samples
  if (c->hin_on && (rc = cuda_check(c, cudaStreamWaitEvent(S(c), c->hin_xy_ready, 0), "wait")))
    return rc;
  if (fuse_r) {
    // the near-field correction of every sample in one launch before the
    // chunks (one launch balances the uneven near pairs across the SMs);
    // each chunk then adds its F-row shares into its slice
    if ((rc = grow(c, c->nearF, sizeof(double) * 3 * (size_t)n))) return rc;
    if ((rc = grow(c, c->loss, sizeof(double) * (size_t)(field_blocks(n) + nchunks + 1)))) return rc;
    hand = (double*)c->nearF.p;
    lossp = (double*)c->loss.p;
    if (c->opts.near_factor > 0) {
      if ((rc = near_forward_minus_float(c, n, xy, hand))) return rc;
    } else if ((rc = cuda_check(c, cudaMemsetAsync(hand, 0, sizeof(double) * 3 * (size_t)n, S(c)),
                                "memset"))) {
      return rc;
    }
  }
  if ((rc = cuda_check(c, cudaMemsetAsync(part, 0, part_b, S(c)), "memset"))) return rc;
  if ((rc = cuda_check(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), S(c)), "memset"))) return rc;
  // the padding rows of F^T (never written by the F rows) hold zeros, so
  // that the J rows of the padding are zero
  for (int k = 0; k < 4; ++k) {
    const int r0 = k < 3 ? k * L.Pp + L.npos : 3 * L.Pp + 2 * L.nh;
    const int r1 = k < 3 ? (k + 1) * L.Pp : rows;
    if (r1 > r0 &&
        (rc = cuda_check(c, cudaMemsetAsync(F + (size_t)r0 * ld, 0, sizeof(float) * (size_t)(r1 - r0) * ld,
                                            S(c)), "memset")))
      return rc;
  }
  int ci = 0;
  float* ghf = reinterpret_cast<float*>(gh);                          // fp32 partials of a chunk
  double* ghr = fused_g ? gh + (size_t)cblk * 3 * nc : nullptr;   // [3nc] running sums
  if (fused_g &&
      (rc = cuda_check(c, cudaMemsetAsync(ghr, 0, sizeof(double) * 3 * (size_t)nc, S(c)), "memset")))
    return rc;
  for (int64_t s0 = 0; s0 < n; s0 += chunk, ++ci) {
    const int m = (int)std::min<int64_t>(chunk, n - s0);
    launch_frows<float, true>(c, xy + 2 * s0, m, F, ld, hw, ld);
    if (fuse_r) {
      double* hs = hand + 3 * s0;
      if (c->hin_on && (rc = cuda_check(c, cudaStreamWaitEvent(S(c), c->hin_t_ready[ci], 0), "wait")))
        return rc;
      {
        ProfScope _ph(c, "k_hand_sum");
        k_hand_sum<<<(m + 255) / 256, 256, 0, S(c)>>>(hw, ld, C, m, hs);
        BEM_LAUNCHED(c);
      }
      if ((rc = field_finish_hand(c, m, xy + 2 * s0, hs, target + 3 * s0,
                                  const_cast<float*>(resid) + 3 * s0, lossp + lblk)))
        return rc;
      lblk += field_blocks(m);
    }
    {
      ProfScope _pp(c, "k_phi_rows");
      const int sl = want_g ? qslices : (int)std::max<int64_t>(1, std::min<int64_t>(256, (m + 1023) / 1024));
      const int len = (m + sl - 1) / sl;
      dim3 grid((Nb + 127) / 128, (m + len - 1) / len);
      double* q = want_g ? qp + (size_t)ci * qslices * Nb * 3 : nullptr;
      const float* rr = want_g ? resid + 3 * s0 : nullptr;
      if (want_g && (int)grid.y < qslices)      // unused slices of a short chunk hold zeros
        cudaMemsetAsync(q, 0, sizeof(double) * qslices * Nb * 3, S(c));
      if (sch == SCH_TF32X3)
        k_phi_q<SCH_TF32X3><<<grid, 128, 0, S(c)>>>(xy + 2 * s0, rr, m, len, c->bd.d_vert32, Nb,
                                                    (void*)phi[0], (void*)phi[1], q);
      else if (sch == SCH_BF16X3)
        k_phi_q<SCH_BF16X3><<<grid, 128, 0, S(c)>>>(xy + 2 * s0, rr, m, len, c->bd.d_vert32, Nb,
                                                    (void*)phi[0], (void*)phi[1], q);
      else
        k_phi_q<SCH_BF16><<<grid, 128, 0, S(c)>>>(xy + 2 * s0, rr, m, len, c->bd.d_vert32, Nb,
                                                  (void*)phi[0], nullptr, q);
      BEM_LAUNCHED(c);
    }
    if (want_g && !fused_g) {
      ProfScope _pg(c, "k_ft_gemv");
      k_ft_gemv<<<dim3((rows + 7) / 8, kGemvSegs), 256, 0, S(c)>>>(
          F, ld, L, nc, m, resid + 3 * s0, gh + (size_t)ci * kGemvSegs * 3 * nc);
      BEM_LAUNCHED(c);
    }
    if ((rc = tc_jrows(c, sch, L, m, Nb, Mt, Nb, phi, Nb, F, ld, J, ld,
                       fused_g ? resid + 3 * s0 : nullptr, nc, fused_g ? ghf : nullptr, cblk)))
      return rc;
    if (fused_g) {
      // every (channel, column) row of the chunk's blocks is written by the
      // J-row epilogue; their sums are added in a fixed order
      k_row_sums<<<(3 * nc + 7) / 8, 256, 0, S(c)>>>(ghf, 3 * nc, (m + 63) / 64, cblk, true, ghr);
      BEM_LAUNCHED(c);
    }
    const void* Jc[2] = {J[0], J[1]};
    if ((rc = tc_syrk(c, sch, L, m, Jc, ld, part, splits))) return rc;
  }
  if (fuse_r && (rc = field_sum_loss(c, lossp, lblk))) return rc;
  k_syrk_reduce<<<dim3((nc + 127) / 128, nc, 3), 128, 0, S(c)>>>(part, splits, nc, L,
                                                                  (double*)c->Hc.p);
  k_h_assemble<<<dim3((nth + 127) / 128, nth), 128, 0, S(c)>>>((const double*)c->Hc.p, c->sc.pp, c->sc.NH,
                                                                n > 0 ? 1.0 / double(n) : 0.0, Hout);
  c->launches += 2;
  if (want_g) {
    // q = sum over chunks and slices (fixed order) -> lambda = (A^+)^T q
    const int nq = nchunks * qslices;
    k_sum_rows<<<(3 * Nb + 31) / 32, 1024, 0, S(c)>>>(qp, nq, 3 * Nb, c->d_q);
    BEM_LAUNCHED(c);
    if ((rc = la_apply3_refined(c, c->bd.d_WT32, c->bd.d_A, c->d_q, c->d_lb, true))) return rc;
    k_g_boundary<<<(3 * nc + 7) / 8, 256, 0, S(c)>>>((const double*)c->Dfc.p, Nb, nc, c->d_lb, gb);
    if (fused_g) {
      k_g_assemble<<<(nth + 127) / 128, 128, 0, S(c)>>>(ghr, 1, 3 * nc, gb, c->sc.pp, c->sc.NH,
                                                         n > 0 ? 1.0 / double(n) : 0.0, gout);
      c->launches += 2;
    } else {
      k_g_assemble<<<(nth + 127) / 128, 128, 0, S(c)>>>(gh, nchunks * kGemvSegs, 3 * nc, gb, c->sc.pp, c->sc.NH,
                                                         n > 0 ? 1.0 / double(n) : 0.0, gout);
      c->launches += 2;
    }
  }
  if ((rc = cuda_check(c, cudaGetLastError(), "jtj tc"))) return rc;
  int st = 0;
  if ((rc = cuda_check(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                                          S(c)), "status")) ||
      (rc = cuda_check(c, cudaStreamSynchronize(S(c)), "sync")))
    return rc;
  if (st) return fail(c, BEM_ETIMEDOUT, "tensor-core J^T J: a bounded device wait ran out");
  return BEM_OK;
}

int jtj_build(bem_ctx* c, int64_t n, const void* xy, double* H, const void* resid, double* g,
              const void* target) {
  if (target && !jtj_fuses_eval(c))
    return fail(c, BEM_EINVAL, "jtj: residual formed in the pass only in the tensor-core modes");
  if (c->opts.precision == BEM_FP64) return jtj_t<double>(c, n, (const double*)xy, H);
  if (c->opts.jtj_mode == BEM_JTJ_BF16)
    return jtj_tc(c, n, (const float*)xy, H, SCH_BF16, (const float*)resid, g, (const float*)target);
  if (c->opts.jtj_mode == BEM_JTJ_3XTF32)
    return jtj_tc(c, n, (const float*)xy, H, SCH_TF32X3, (const float*)resid, g,
                  (const float*)target);
  if (c->opts.jtj_mode == BEM_JTJ_BF16X3)
    return jtj_tc(c, n, (const float*)xy, H, SCH_BF16X3, (const float*)resid, g,
                  (const float*)target);
  return jtj_t<float>(c, n, (const float*)xy, H);
}

bool jtj_gives_gradient(const bem_ctx* c) {
  return c->opts.precision == BEM_MIXED &&
         (c->opts.jtj_mode == BEM_JTJ_BF16 || c->opts.jtj_mode == BEM_JTJ_3XTF32 ||
          c->opts.jtj_mode == BEM_JTJ_BF16X3);
}

}  // namespace bem
