// Float Cholesky factor and triangular solves of the equilibrated LM matrix
// for large systems (n_theta >= kBlockedMinN, e.g. the 5,000 parameters of
// 500 segment handles).  The solve around them (equilibration, iterative
// refinement in double, the double fallback) is la_lm_solve's.
//
// Factor, right-looking in 64-column steps, three launches per step:
//   (1) one CTA factors the 64 x 64 diagonal block and inverts the factor;
//   (2) the panel below it, L_21 L_11^T = A_21, by forward substitution, one
//       thread per row;
//   (3) the trailing lower triangle, A_22 -= L_21 L_21^T, in 128 x 128 tiles.
// Kf holds the trailing updates, Lf the factor (lower), Linv64 the inverses of
// its 64 x 64 diagonal blocks ([n/64][64][64], zero-padded).
//
// Solve: a cluster of kTrsvCluster CTAs shares the forward and backward
// substitution through distributed shared memory (see k_trsv_cluster).
#include <cooperative_groups.h>

#include <algorithm>

#include "ctx.h"

namespace bem {

namespace {

// Cholesky of the 32 x 32 block S (row stride 65) in warp-register form:
// lane r holds row r; column j takes its pivot from lane j, l_rj = a_rj /
// sqrt(pivot) for r > j, then a_rq -= l_rj l_qj with l_qj shuffled from lane
// q.  nb valid rows; rows and columns beyond nb come out zero.  The inverse
// of the factor goes to X (lane c computes column c).  A pivot that is not
// positive is replaced by 1 and the first one is reported.
__device__ void warp_chol32(float (*S)[65], int nb, float (*X)[65], int* status, float* bad_pivot) {
  const int r = threadIdx.x & 31;
  float a[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) a[q] = S[r][q];
  float rd = 0.f;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    if (j < nb) {
      float d = __shfl_sync(0xffffffffu, a[j], j);
      if (!(d > 0.f)) {
        if (r == 0 && atomicCAS(status, 0, 1) == 0) *bad_pivot = d;
        d = 1.f;
      }
      const float rs = rsqrtf(d);
      const float l = r > j ? a[j] * rs : 0.f;
      if (r == j) { a[j] = d * rs; rd = rs; }
      if (r > j) a[j] = l;
#pragma unroll
      for (int q = j + 1; q < 32; ++q) a[q] = fmaf(-l, __shfl_sync(0xffffffffu, l, q), a[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 32; ++q) S[r][q] = (q <= r && r < nb) ? a[q] : 0.f;
  // X_rc = (delta_rc - sum_{k=c}^{r-1} L_rk X_kc) / L_rr, L_rk shuffled from lane r
  float x[32];
#pragma unroll
  for (int rr = 0; rr < 32; ++rr) {
    float sacc = rr == r ? 1.f : 0.f;
#pragma unroll
    for (int k = 0; k < rr; ++k) sacc = fmaf(-__shfl_sync(0xffffffffu, a[k], rr), x[k], sacc);
    const float rdr = __shfl_sync(0xffffffffu, rd, rr);
    x[rr] = (rr >= r && rr < nb) ? sacc * rdr : 0.f;
  }
#pragma unroll
  for (int rr = 0; rr < 32; ++rr) X[rr][r] = x[rr];
}

// (1) the diagonal block at (k0, k0), nb = min(64, n - k0): 2 x 2 blocks of
// 32 (L11; L21 from L21 L11^T = A21 by forward substitution; A22 - L21
// L21^T; L22) and the inverse X = [[X11, 0], [-X22 L21 X11, X22]].
__global__ void __launch_bounds__(256) k_chol_diag64(const float* __restrict__ Kf, float* __restrict__ Lf,
                                                     int n, int k0, float* __restrict__ Linv64,
                                                     int* __restrict__ status,
                                                     float* __restrict__ bad_pivot) {
  __shared__ float S[64][65];
  __shared__ float X[64][65];
  __shared__ float W[32][65];
  const int tid = threadIdx.x;
  const int nb = min(64, n - k0), nb1 = min(nb, 32), nb2 = nb - nb1;
  {
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * u, r = e >> 6, q = e & 63;
      v[u] = (r < nb && q <= r) ? Kf[(size_t)(k0 + r) * n + k0 + q] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * u;
      S[e >> 6][e & 63] = v[u];
      X[e >> 6][e & 63] = 0.f;
    }
  }
  __syncthreads();
  if (tid < 32) warp_chol32(S, nb1, X, status, bad_pivot);
  __syncthreads();
  if (nb2 > 0) {
    // L21, one thread per row: x_q = (a_q - sum_{l<q} x_l L_ql) / L_qq (nb1 = 32 here)
    if (tid < 32) {
      const int r = tid;
      float x[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        float v = S[32 + r][q];
#pragma unroll
        for (int l = 0; l < q; ++l) v = fmaf(-x[l], S[q][l], v);
        x[q] = r < nb2 ? v / S[q][q] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 32; ++q) W[r][q] = x[q];
    }
    __syncthreads();
    // A22 -= L21 L21^T (lower part), L21 into S
    for (int e = tid; e < 1024; e += 256) {
      const int r = e >> 5, q = e & 31;
      if (q <= r) {
        float v = S[32 + r][32 + q];
        for (int l = 0; l < 32; ++l) v = fmaf(-W[r][l], W[q][l], v);
        S[32 + r][32 + q] = v;
      }
      S[32 + r][q] = W[r][q];
    }
    __syncthreads();
    if (tid < 32)
      warp_chol32(reinterpret_cast<float (*)[65]>(&S[32][32]), nb2,
                  reinterpret_cast<float (*)[65]>(&X[32][32]), status, bad_pivot);
    __syncthreads();
    // X21 = -X22 (L21 X11): W <- L21 X11 (X11 lower), then X21
    float y[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u, r = e >> 5, q = e & 31;
      float v = 0.f;
      for (int l = q; l < 32; ++l) v = fmaf(S[32 + r][l], X[l][q], v);
      y[u] = v;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u;
      W[e >> 5][e & 31] = y[u];
    }
    __syncthreads();
    for (int e = tid; e < 1024; e += 256) {
      const int r = e >> 5, q = e & 31;
      float v = 0.f;
      for (int l = 0; l <= r; ++l) v = fmaf(-X[32 + r][32 + l], W[l][q], v);
      X[32 + r][q] = r < nb2 ? v : 0.f;
    }
    __syncthreads();
  }
  float* Xo = Linv64 + (size_t)(k0 / 64) * 4096;
  for (int e = tid; e < 64 * 64; e += 256) {
    const int r = e >> 6, q = e & 63;
    if (r < nb && q < nb) Lf[(size_t)(k0 + r) * n + k0 + q] = q <= r ? S[r][q] : 0.f;
    Xo[e] = X[r][q];
  }
}

// (2) panel rows i >= k0 + 64, 64 per CTA, one thread per row: forward
// substitution with the diagonal factor L_11 (read back from Lf), the row
// held in registers.  Called only when the whole block exists (n >= k0 + 64).
__global__ void __launch_bounds__(64) k_chol_panel64(const float* __restrict__ Kf, float* __restrict__ Lf,
                                                     int n, int k0) {
  __shared__ float L[64][65];
  __shared__ float rdiag[64];
  const int tid = threadIdx.x;
  {
    float v[64];
#pragma unroll
    for (int u = 0; u < 64; ++u) v[u] = tid <= u ? Lf[(size_t)(k0 + u) * n + k0 + tid] : 0.f;
#pragma unroll
    for (int u = 0; u < 64; ++u) L[u][tid] = v[u];
  }
  __syncthreads();
  rdiag[tid] = 1.f / L[tid][tid];
  __syncthreads();
  const int gi = k0 + 64 + 64 * blockIdx.x + tid;
  if (gi >= n) return;
  const float* row = Kf + (size_t)gi * n + k0;
  float x[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) x[q] = row[q];
#pragma unroll
  for (int q = 0; q < 64; ++q) {
    float v = x[q];
#pragma unroll
    for (int l = 0; l < q; ++l) v = fmaf(-x[l], L[q][l], v);
    x[q] = v * rdiag[q];
  }
  float* out = Lf + (size_t)gi * n + k0;
#pragma unroll
  for (int q = 0; q < 64; ++q) out[q] = x[q];
}

// (3) trailing update: tile (bi, bj), bj <= bi, of the rows/columns >= r0 =
// k0 + 64: Kf[i][j] -= sum_l L[i][k0 + l] L[j][k0 + l].  256 threads, each an
// 8 x 8 block (rows 4 ty.. and 64 + 4 ty.., columns likewise with tx), the
// panel rows staged transposed in 32-column chunks.  Diagonal tiles are
// updated whole (the strict upper triangle of Kf is never read).
constexpr int kSyrkLd = 132;
__global__ void __launch_bounds__(256) k_chol_syrk128(float* __restrict__ Kf, const float* __restrict__ Lf,
                                                      int n, int k0) {
  __shared__ __align__(16) float Pa[32][kSyrkLd];
  __shared__ __align__(16) float Pb[32][kSyrkLd];
  int t = blockIdx.x, bi = 0;
  while (t > bi) { t -= bi + 1; ++bi; }
  const int bj = t, r0 = k0 + 64;
  const int i0 = r0 + 128 * bi, j0 = r0 + 128 * bj;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  for (int l0 = 0; l0 < 64; l0 += 32) {
    float va[16], vb[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * u, rr = e >> 5, l = e & 31;
      const int gi = i0 + rr, gj = j0 + rr;
      va[u] = gi < n ? Lf[(size_t)gi * n + k0 + l0 + l] : 0.f;
      vb[u] = gj < n ? Lf[(size_t)gj * n + k0 + l0 + l] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * u, rr = e >> 5, l = e & 31;
      Pa[l][rr] = va[u];
      Pb[l][rr] = vb[u];
    }
    __syncthreads();
#pragma unroll 4
    for (int l = 0; l < 32; ++l) {
      const float4 a0 = *reinterpret_cast<const float4*>(&Pa[l][4 * ty]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Pa[l][64 + 4 * ty]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Pb[l][4 * tx]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Pb[l][64 + 4 * tx]);
      const float pa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float pb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(pa[a], pb[b], acc[a][b]);
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int gi = i0 + (a < 4 ? 4 * ty + a : 64 + 4 * ty + a - 4);
    if (gi >= n) continue;
    float* rowp = Kf + (size_t)gi * n;
    float cur[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int gj = j0 + (b < 4 ? 4 * tx + b : 64 + 4 * tx + b - 4);
      cur[b] = gj < n ? rowp[gj] : 0.f;
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int gj = j0 + (b < 4 ? 4 * tx + b : 64 + 4 * tx + b - 4);
      if (gj < n) rowp[gj] = cur[b] - acc[a][b];
    }
  }
}

// ---- cluster triangular solve ------------------------------------------------

constexpr int kTrsvCluster = 8, kTrsvThreads = 512;

// tmp = Xb sb (or Xb^T sb) for one 64 x 4 block, then sb = tmp; Xb staged in
// shared memory first.  All threads of the CTA call it.
__device__ __forceinline__ void trsv_block_solve(const float* __restrict__ Xb, float (*Xs)[65],
                                                 float (*sb)[4], float (*tmp)[4], bool transpose) {
  const int tid = threadIdx.x;
  {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = Xb[tid + kTrsvThreads * u];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + kTrsvThreads * u;
      Xs[e >> 6][e & 63] = v[u];
    }
  }
  __syncthreads();
  if (tid < 256) {
    const int r = tid >> 2, qq = tid & 3;
    float v = 0.f;
    if (!transpose) {
      for (int l = 0; l <= r; ++l) v = fmaf(Xs[r][l], sb[l][qq], v);
    } else {
      for (int l = r; l < 64; ++l) v = fmaf(Xs[l][r], sb[l][qq], v);
    }
    tmp[r][qq] = v;
  }
  __syncthreads();
  if (tid < 256) sb[tid >> 2][tid & 3] = tmp[tid >> 2][tid & 3];
}

// One float solve of (D K D) z = D r with the factor L (lower triangle of Lf)
// and its 64 x 64 diagonal-block inverses by a cluster of kTrsvCluster CTAs.
// Block b of 64 rows belongs to CTA b mod kTrsvCluster, which keeps the four
// right-hand sides of its rows in shared memory.  Forward: the owner of block
// b forms y_b = Linv_b b_b; after a cluster barrier every CTA reads y_b from
// the owner's shared memory and subtracts L[i][block b] y_b from its rows
// below the block.  Backward with L^T the same way from the last block.
// X += D z in double.  Rres: the double residual R - K X.  Every CTA passes
// the same sequence of cluster barriers.
__global__ void __cluster_dims__(kTrsvCluster, 1, 1) __launch_bounds__(kTrsvThreads)
    k_trsv_cluster(const float* __restrict__ Lf, const float* __restrict__ Linv64, int n,
                   const double* __restrict__ d, const double* __restrict__ Rres,
                   double* __restrict__ X) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) float sbuf[];   // [owned blocks][64][4]
  __shared__ float yk[64][4], tmp[64][4];
  __shared__ float Xs[64][65];
  float (*sb)[4] = reinterpret_cast<float (*)[4]>(sbuf);
  const int q = (int)cl.block_rank(), tid = threadIdx.x;
  const int B = (n + 63) / 64;
  const int nown = B > q ? (B - q + kTrsvCluster - 1) / kTrsvCluster : 0;
  // local row lr = 64 lb + r of owned block lb is global row 64 (lb C + q) + r
  for (int e = tid; e < nown * 256; e += blockDim.x) {
    const int lr = e >> 2, qq = e & 3;
    const int gi = 64 * ((lr >> 6) * kTrsvCluster + q) + (lr & 63);
    sb[lr][qq] = gi < n ? float(d[gi] * Rres[4 * gi + qq]) : 0.f;
  }
  __syncthreads();
  // ---- forward: L y = b
  for (int b = 0; b < B; ++b) {
    const int own = b % kTrsvCluster, lb = b / kTrsvCluster;
    if (own == q) trsv_block_solve(Linv64 + (size_t)b * 4096, Xs, sb + 64 * lb, tmp, false);
    cl.sync();
    const float* ys = cl.map_shared_rank(&sb[64 * lb][0], own);
    if (tid < 256) yk[tid >> 2][tid & 3] = ys[tid];
    __syncthreads();
    // owned blocks after b: from the first local block lb' with lb' C + q > b
    const int lb0 = (b + 1 - q + kTrsvCluster - 1) / kTrsvCluster;
    for (int lr = 64 * lb0 + tid; lr < 64 * nown; lr += blockDim.x) {
      const int gi = 64 * ((lr >> 6) * kTrsvCluster + q) + (lr & 63);
      if (gi >= n) continue;
      // block b is whole here: row gi lies below it
      const float* row = Lf + (size_t)gi * n + 64 * b;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
      for (int h = 0; h < 64; h += 16) {
        float m[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) m[u] = row[h + u];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          s0 = fmaf(m[u], yk[h + u][0], s0); s1 = fmaf(m[u], yk[h + u][1], s1);
          s2 = fmaf(m[u], yk[h + u][2], s2); s3 = fmaf(m[u], yk[h + u][3], s3);
        }
      }
      sb[lr][0] -= s0; sb[lr][1] -= s1; sb[lr][2] -= s2; sb[lr][3] -= s3;
    }
    __syncthreads();
  }
  // ---- backward: L^T z = y
  for (int b = B - 1; b >= 0; --b) {
    const int own = b % kTrsvCluster, lb = b / kTrsvCluster;
    if (own == q) trsv_block_solve(Linv64 + (size_t)b * 4096, Xs, sb + 64 * lb, tmp, true);
    cl.sync();
    const float* zs = cl.map_shared_rank(&sb[64 * lb][0], own);
    if (tid < 256) yk[tid >> 2][tid & 3] = zs[tid];
    __syncthreads();
    const int nb = min(64, n - 64 * b);
    const int lb1 = b > q ? (b - q + kTrsvCluster - 1) / kTrsvCluster : 0;   // owned blocks < b
    for (int lr = tid; lr < 64 * lb1; lr += blockDim.x) {
      const int gi = 64 * ((lr >> 6) * kTrsvCluster + q) + (lr & 63);
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      for (int h = 0; h < nb; h += 16) {
        float m[16];
#pragma unroll
        for (int u = 0; u < 16; ++u)
          m[u] = h + u < nb ? Lf[(size_t)(64 * b + h + u) * n + gi] : 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          s0 = fmaf(m[u], yk[h + u][0], s0); s1 = fmaf(m[u], yk[h + u][1], s1);
          s2 = fmaf(m[u], yk[h + u][2], s2); s3 = fmaf(m[u], yk[h + u][3], s3);
        }
      }
      sb[lr][0] -= s0; sb[lr][1] -= s1; sb[lr][2] -= s2; sb[lr][3] -= s3;
    }
    __syncthreads();
  }
  for (int e = tid; e < nown * 256; e += blockDim.x) {
    const int lr = e >> 2, qq = e & 3;
    const int gi = 64 * ((lr >> 6) * kTrsvCluster + q) + (lr & 63);
    if (gi < n) X[4 * gi + qq] += d[gi] * double(sb[lr][qq]);
  }
  // no CTA leaves while another may still read its shared memory
  cl.sync();
}

size_t trsv_smem(int n) {
  const int B = (n + 63) / 64;
  return sizeof(float) * 256 * (size_t)((B + kTrsvCluster - 1) / kTrsvCluster);
}

}  // namespace

void chol_blocked_f32(bem_ctx* c, float* Kf, float* Lf, int n, float* Linv64, int* status,
                      float* bad_pivot) {
  for (int k0 = 0; k0 < n; k0 += 64) {
    k_chol_diag64<<<1, 256, 0, S(c)>>>(Kf, Lf, n, k0, Linv64, status, bad_pivot);
    BEM_LAUNCHED(c);
    const int rest = n - std::min(n, k0 + 64);
    if (rest == 0) break;
    k_chol_panel64<<<(rest + 63) / 64, 64, 0, S(c)>>>(Kf, Lf, n, k0);
    BEM_LAUNCHED(c);
    const int tiles = (rest + 127) / 128;
    k_chol_syrk128<<<tiles * (tiles + 1) / 2, 256, 0, S(c)>>>(Kf, Lf, n, k0);
    BEM_LAUNCHED(c);
  }
}

int trsv_cluster_prepare(bem_ctx* c, int n) {
  const size_t smem = trsv_smem(n);
  if (smem > 48 * 1024)
    return cuda_check(c, cudaFuncSetAttribute(k_trsv_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem), "smem attribute");
  return BEM_OK;
}

void trsv_cluster_f32(bem_ctx* c, const float* Lf, const float* Linv64, int n, const double* d,
                      const double* Rres, double* X) {
  k_trsv_cluster<<<kTrsvCluster, kTrsvThreads, trsv_smem(n), S(c)>>>(Lf, Linv64, n, d, Rres, X);
  BEM_LAUNCHED(c);
}

}  // namespace bem
