// Dense linear algebra of the hot path, all in double unless noted.
//
//  * Boundary system (Sec. 3.1.3).  The Neumann Galerkin matrix A has the
//    constants as right null vector.  The bordered matrix
//        B = [[A, 1], [1^T, 0]]
//    is non-singular; Gauss-Jordan elimination with partial pivoting gives
//    B^-1 once.  Its last row (first Nb entries) is the left null vector v of
//    A scaled so that 1.v = 1 (B^T [v; 0] = e_last).  With T the leading
//    Nb x Nb block of B^-1 and P = I - v v^T/|v|^2,
//        A^+ = T P
//    is the pseudo-inverse that drops the null space (equal to the SVD
//    solution with the smallest singular value discarded): A (T P f) = P f
//    and 1.(T P f) = 0.  Every later solve is a product with A^+ or (A^+)^T.
//  * Mixed precision: the float copy of A^+ is applied and corrected once
//    with the double residual P f - A u (one step of iterative refinement).
//  * LM system (Eq. (optimstep), Sec. 4.3): blocked Cholesky of H + lambda D,
//    triangular solves, and a 3 x 3 Schur complement for the compatibility
//    constraints (one per colour channel).
#include <cmath>

#include "ctx.h"

namespace bem {

// ---------------------------------------------------------------------------
// Gauss-Jordan on the augmented matrix G = [B | I], N rows, 2N columns.

__global__ void k_gj_init(const double* __restrict__ A, int Nb, double* __restrict__ G) {
  int N = Nb + 1, W = 2 * N;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)N * W) return;
  int i = idx / W, j = idx % W;
  double v;
  if (j < N) {
    if (i < Nb && j < Nb) v = A[(size_t)i * Nb + j];
    else if (i == Nb && j == Nb) v = 0.0;
    else v = 1.0;
  } else {
    v = (j - N == i) ? 1.0 : 0.0;
  }
  G[idx] = v;
}

// Pivot search in column k (rows >= k), row swap, scaling of the pivot row;
// saves the column for the elimination.  One block.
__global__ void k_gj_pivot(double* __restrict__ G, int N, int k, double* __restrict__ col,
                           int* __restrict__ status) {
  int W = 2 * N;
  __shared__ double bv[32];
  __shared__ int bi[32];
  double best = -1.0;
  int arg = k;
  for (int i = k + threadIdx.x; i < N; i += blockDim.x) {
    double v = fabs(G[(size_t)i * W + k]);
    if (v > best) { best = v; arg = i; }
  }
  for (int o = 16; o; o >>= 1) {
    double ov = __shfl_down_sync(0xffffffffu, best, o);
    int oi = __shfl_down_sync(0xffffffffu, arg, o);
    if (ov > best || (ov == best && oi < arg)) { best = ov; arg = oi; }
  }
  int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) { bv[w] = best; bi[w] = arg; }
  __syncthreads();
  __shared__ int piv;
  __shared__ double pval;
  if (threadIdx.x == 0) {
    double b = -1.0;
    int a = k;
    for (int q = 0; q < (int)(blockDim.x / 32); ++q)
      if (bv[q] > b || (bv[q] == b && bi[q] < a)) { b = bv[q]; a = bi[q]; }
    piv = a;
    if (!(b > 1e-300)) *status = 1;
  }
  __syncthreads();
  int r = piv;
  if (r != k)
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
      double t = G[(size_t)k * W + j];
      G[(size_t)k * W + j] = G[(size_t)r * W + j];
      G[(size_t)r * W + j] = t;
    }
  __syncthreads();
  if (threadIdx.x == 0) pval = G[(size_t)k * W + k];
  __syncthreads();
  double inv = 1.0 / pval;
  for (int j = threadIdx.x; j < W; j += blockDim.x) G[(size_t)k * W + j] *= inv;
  for (int i = threadIdx.x; i < N; i += blockDim.x) col[i] = G[(size_t)i * W + k];
}

__global__ void k_gj_elim(double* __restrict__ G, int N, int k, const double* __restrict__ col) {
  int W = 2 * N;
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (j >= W || i == k || j < k) return;    // columns < k of rows != k are already zero
  double f = col[i];
  if (f != 0.0) G[(size_t)i * W + j] -= f * G[(size_t)k * W + j];
}

// W = T - (T v) v^T / |v|^2 from the inverse, plus W^T and float copies.
__global__ void k_pinv_tv(const double* __restrict__ G, int Nb, double* __restrict__ tv,
                          double* __restrict__ vv) {
  int N = Nb + 1, W = 2 * N;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Nb) {
    const double* Ti = G + (size_t)i * W + N;   // row i of T
    const double* v = G + (size_t)Nb * W + N;   // last row of B^-1
    double s = 0;
    for (int j = 0; j < Nb; ++j) s += Ti[j] * v[j];
    tv[i] = s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double* v = G + (size_t)Nb * W + N;
    double s = 0;
    for (int j = 0; j < Nb; ++j) s += v[j] * v[j];
    *vv = s;
  }
}

__global__ void k_pinv_form(const double* __restrict__ G, int Nb, const double* __restrict__ tv,
                            const double* __restrict__ vv, double* __restrict__ Wm,
                            double* __restrict__ WT, float* __restrict__ W32,
                            float* __restrict__ WT32) {
  int N = Nb + 1, Wd = 2 * N;
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (j >= Nb) return;
  const double* v = G + (size_t)Nb * Wd + N;
  double w = G[(size_t)i * Wd + N + j] - tv[i] * v[j] / (*vv);
  Wm[(size_t)i * Nb + j] = w;
  WT[(size_t)j * Nb + i] = w;
  W32[(size_t)i * Nb + j] = float(w);
  WT32[(size_t)j * Nb + i] = float(w);
}

int la_pinv(bem_ctx* c) {
  int Nb = c->bd.Nb, N = Nb + 1;
  size_t gsz = (size_t)N * 2 * N * sizeof(double);
  int rc;
  if ((rc = grow(c, c->lmW, gsz + (N + Nb + 1) * sizeof(double)))) return rc;
  double* G = (double*)c->lmW.p;
  double* col = G + (size_t)N * 2 * N;
  double* tv = col + N;
  double* vv = tv + Nb;
  if ((rc = cuda_check(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), S(c)), "memset"))) return rc;
  size_t tot = (size_t)N * 2 * N;
  k_gj_init<<<(tot + 255) / 256, 256, 0, S(c)>>>(c->bd.d_A, Nb, G);
  BEM_LAUNCHED(c);
  for (int k = 0; k < N; ++k) {
    k_gj_pivot<<<1, 1024, 0, S(c)>>>(G, N, k, col, c->d_status);
    dim3 grid((2 * N + 255) / 256, N);
    k_gj_elim<<<grid, 256, 0, S(c)>>>(G, N, k, col);
    c->launches += 2;
  }
  k_pinv_tv<<<(Nb + 127) / 128, 128, 0, S(c)>>>(G, Nb, tv, vv);
  dim3 g2((Nb + 127) / 128, Nb);
  k_pinv_form<<<g2, 128, 0, S(c)>>>(G, Nb, tv, vv, c->bd.d_W, c->bd.d_WT, c->bd.d_W32,
                                     c->bd.d_WT32);
  c->launches += 2;
  if ((rc = cuda_check(c, cudaGetLastError(), "pinv"))) return rc;
  int st = 0;
  if ((rc = cuda_check(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                                          S(c)), "status")))
    return rc;
  if ((rc = cuda_check(c, cudaStreamSynchronize(S(c)), "pinv sync"))) return rc;
  if (st) return fail(c, BEM_ESINGULAR, "boundary matrix: zero pivot in the bordered system");
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// y[Nb][3] = W x[Nb][3]: one warp per row.

__global__ void k_apply3(const double* __restrict__ Wm, int Nb, const double* __restrict__ x,
                         double* __restrict__ y) {
  int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int l = threadIdx.x % 32;
  if (row >= Nb) return;
  const double* w = Wm + (size_t)row * Nb;
  double s0 = 0, s1 = 0, s2 = 0;
  for (int j = l; j < Nb; j += 32) {
    double a = w[j];
    s0 += a * x[3 * j];
    s1 += a * x[3 * j + 1];
    s2 += a * x[3 * j + 2];
  }
  for (int o = 16; o; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if (l == 0) { y[3 * row] = s0; y[3 * row + 1] = s1; y[3 * row + 2] = s2; }
}

int la_apply3(bem_ctx* c, const double* Wm, const double* x, double* y) {
  int Nb = c->bd.Nb;
  k_apply3<<<(Nb + 7) / 8, 256, 0, S(c)>>>(Wm, Nb, x, y);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "k_apply3");
}

// float product u = W32 x (double accumulate of float products)
__global__ void k_apply3_f(const float* __restrict__ Wm, int Nb, const double* __restrict__ x,
                           double* __restrict__ y) {
  int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int l = threadIdx.x % 32;
  if (row >= Nb) return;
  const float* w = Wm + (size_t)row * Nb;
  float s0 = 0, s1 = 0, s2 = 0;
  for (int j = l; j < Nb; j += 32) {
    float a = w[j];
    s0 += a * float(x[3 * j]);
    s1 += a * float(x[3 * j + 1]);
    s2 += a * float(x[3 * j + 2]);
  }
  for (int o = 16; o; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if (l == 0) { y[3 * row] = s0; y[3 * row + 1] = s1; y[3 * row + 2] = s2; }
}

// residual r = x - A u (or x - A^T u) in double.  A^+ annihilates the part
// of r outside the range, so u + A^+ r is the refined A^+ x.
__global__ void k_resid3(const double* __restrict__ A, int Nb, const double* __restrict__ x,
                         const double* __restrict__ u, double* __restrict__ r, bool transpose) {
  int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int l = threadIdx.x % 32;
  if (row >= Nb) return;
  double s0 = 0, s1 = 0, s2 = 0;
  for (int j = l; j < Nb; j += 32) {
    double a = transpose ? A[(size_t)j * Nb + row] : A[(size_t)row * Nb + j];
    s0 += a * u[3 * j];
    s1 += a * u[3 * j + 1];
    s2 += a * u[3 * j + 2];
  }
  for (int o = 16; o; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if (l == 0) {
    r[3 * row] = x[3 * row] - s0;
    r[3 * row + 1] = x[3 * row + 1] - s1;
    r[3 * row + 2] = x[3 * row + 2] - s2;
  }
}

__global__ void k_add3(double* __restrict__ y, const double* __restrict__ d, int n3) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n3) y[i] += d[i];
}

int la_apply3_refined(bem_ctx* c, const float* W32, const double* A, const double* x, double* y,
                      bool transpose) {
  int Nb = c->bd.Nb, rc;
  if ((rc = grow(c, c->gpart, sizeof(double) * 6 * Nb))) return rc;
  double* r = (double*)c->gpart.p;
  double* d = r + 3 * Nb;
  k_apply3_f<<<(Nb + 7) / 8, 256, 0, S(c)>>>(W32, Nb, x, y);
  // A^+ (x - A u): for u = A^+ x exactly this is A^+ P x - A^+ A A^+ x = 0
  k_resid3<<<(Nb + 7) / 8, 256, 0, S(c)>>>(A, Nb, x, y, r, transpose);
  k_apply3_f<<<(Nb + 7) / 8, 256, 0, S(c)>>>(W32, Nb, r, d);
  k_add3<<<(3 * Nb + 255) / 256, 256, 0, S(c)>>>(y, d, 3 * Nb);
  c->launches += 4;
  return cuda_check(c, cudaGetLastError(), "refined apply");
}

// Same refined product as la_apply3_refined with the caller's scratch
// (6 Nb doubles) instead of a context buffer.
int la_apply3_refined_buf(bem_ctx* c, const float* W32, const double* A, const double* x,
                          double* y, bool transpose, double* scratch) {
  int Nb = c->bd.Nb;
  double* r = scratch;
  double* d = r + 3 * Nb;
  k_apply3_f<<<(Nb + 7) / 8, 256, 0, S(c)>>>(W32, Nb, x, y);
  k_resid3<<<(Nb + 7) / 8, 256, 0, S(c)>>>(A, Nb, x, y, r, transpose);
  k_apply3_f<<<(Nb + 7) / 8, 256, 0, S(c)>>>(W32, Nb, r, d);
  k_add3<<<(3 * Nb + 255) / 256, 256, 0, S(c)>>>(y, d, 3 * Nb);
  c->launches += 4;
  return cuda_check(c, cudaGetLastError(), "refined apply");
}

// ---------------------------------------------------------------------------
// C = alpha op(A) op(B) + beta C, row-major, double.  64 x 64 tiles, 4 x 4 per thread.

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, double alpha,
                                               const double* __restrict__ A, int lda,
                                               const double* __restrict__ B, int ldb,
                                               double beta, double* __restrict__ C, int ldc) {
  __shared__ double As[16][65];
  __shared__ double Bs[16][65];
  int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int kk, mm;
      if (TA) { mm = e % 64; kk = e / 64; } else { kk = e % 16; mm = e / 16; }
      int gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < K) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int kk, nn;
      if (TB) { kk = e % 16; nn = e / 16; } else { nn = e % 64; kk = e / 64; }
      int gn = n0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < N && gk < K) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      double* cp = C + (size_t)gm * ldc + gn;
      *cp = alpha * acc[i][j] + (beta == 0.0 ? 0.0 : beta * *cp);
    }
  }
}

void la_dgemm(bem_ctx* c, bool ta, bool tb, int M, int N, int K, double alpha, const double* A,
              int lda, const double* B, int ldb, double beta, double* C, int ldc) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  if (!ta && !tb) k_dgemm<false, false><<<grid, 256, 0, S(c)>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else if (ta && !tb) k_dgemm<true, false><<<grid, 256, 0, S(c)>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else if (!ta && tb) k_dgemm<false, true><<<grid, 256, 0, S(c)>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else k_dgemm<true, true><<<grid, 256, 0, S(c)>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  BEM_LAUNCHED(c);
}

// ---------------------------------------------------------------------------
// LM system.

// max of the diagonal over active parameters -> *mx
__global__ void k_diag_max(const double* __restrict__ H, int n, double* __restrict__ mx) {
  __shared__ double red[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, H[(size_t)i * n + i]);
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) r = fmax(r, red[q]);
    *mx = r;
  }
}

// K = H + lam diag(max(H_ii, 1e-12 max)) on active parameters; inactive
// rows/columns become identity rows.  rhs[n][4] = (-g, a-columns).
__global__ void k_lm_build(const double* __restrict__ H, const double* __restrict__ g, int n,
                           int C, const uint8_t* __restrict__ closed, const double* __restrict__ a,
                           const double* __restrict__ mx, double lam, double* __restrict__ Kmat,
                           double* __restrict__ rhs) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (j >= n) return;
  auto active = [&](int t) {
    int h = t / 8, comp = t % 8;
    return !(comp < 2 && (h % 4) == 3 && closed[h / 4]);
  };
  bool ai = active(i), aj = active(j);
  double v;
  if (!ai || !aj) v = (i == j) ? 1.0 : 0.0;
  else {
    v = H[(size_t)i * n + j];
    if (i == j) v += lam * fmax(v, 1e-12 * (*mx));
  }
  Kmat[(size_t)i * n + j] = v;
  if (j == 0) {
    int h = i / 8, comp = i % 8;
    rhs[4 * i] = ai ? -g[i] : 0.0;
    for (int c = 0; c < 3; ++c) rhs[4 * i + 1 + c] = (comp == 5 + c) ? a[h] : 0.0;
  }
}

// cons[n][4]: columns 1..3 = compatibility constraint of channel 0..2
// (a_h at the w_c entry of control handle h), column 0 unused.
__global__ void k_constraint_cols(int n, const double* __restrict__ a, double* __restrict__ cons) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int h = i / 8, comp = i % 8;
  cons[4 * i] = 0.0;
  for (int c = 0; c < 3; ++c) cons[4 * i + 1 + c] = (comp == 5 + c) ? a[h] : 0.0;
}

// Cholesky of the nb x nb (nb <= 32) diagonal block at (k0,k0): one warp,
// lane r owns row r of the block in shared memory; no block-wide barriers.
__global__ void k_potrf_diag(double* __restrict__ Km, int n, int k0, int nb,
                             int* __restrict__ status) {
  __shared__ double T[32][33];
  const int lane = threadIdx.x;
  for (int q = 0; q < nb; ++q) T[lane][q] = lane < nb ? Km[(size_t)(k0 + lane) * n + k0 + q] : 0.0;
  __syncwarp();
  for (int j = 0; j < nb; ++j) {
    double d = T[j][j];
    if (!(d > 0.0)) {
      if (lane == 0) *status = 1;
      d = 1.0;
    }
    const double ri = rsqrt(d);        // 1/sqrt(pivot)
    __syncwarp();
    if (lane == j) T[j][j] = d * ri;
    if (lane > j && lane < nb) T[lane][j] *= ri;
    __syncwarp();
    if (lane > j && lane < nb) {
      const double lrj = T[lane][j];
      for (int q = j + 1; q <= lane; ++q) T[lane][q] -= lrj * T[q][j];
    }
    __syncwarp();
  }
  if (lane < nb)
    for (int q = 0; q < nb; ++q) Km[(size_t)(k0 + lane) * n + k0 + q] = q <= lane ? T[lane][q] : 0.0;
}

// rows i >= k0+nb of the panel: L_i = A_i L_kk^-T (forward substitution per row)
__global__ void k_trsm_rows(double* __restrict__ Km, int n, int k0, int nb) {
  __shared__ double Lk[32][33];
  __shared__ double inv[32];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int r = e / nb, q = e % nb;
    Lk[r][q] = Km[(size_t)(k0 + r) * n + k0 + q];
  }
  __syncthreads();
  if (threadIdx.x < nb) inv[threadIdx.x] = 1.0 / Lk[threadIdx.x][threadIdx.x];
  __syncthreads();
  int i = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[32];
  double* row = Km + (size_t)i * n + k0;
  for (int j = 0; j < nb; ++j) {
    double s = row[j];
    for (int l = 0; l < j; ++l) s -= x[l] * Lk[j][l];
    x[j] = s * inv[j];
  }
  for (int j = 0; j < nb; ++j) row[j] = x[j];
}

// Lt = L^T (lower triangle of Km)
__global__ void k_transpose_lower(const double* __restrict__ Km, int n, double* __restrict__ Lt) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (j >= n) return;
  Lt[(size_t)j * n + i] = (j <= i) ? Km[(size_t)i * n + j] : 0.0;
}

// Triangular solves with four right-hand sides R[n][4], blocked by 32 rows,
// column oriented: a one-warp kernel solves the 32 x 32 diagonal block
// (lane = row), then a kernel over all CTAs subtracts that block's
// contribution from every remaining row.  Forward sweep with L (rows of L),
// back sweep with L^T (rows of Lt).

// forward: diagonal block [kb, kb+nb) of L y = R
__global__ void k_trsv_diag_fwd(const double* __restrict__ L, int n, int kb, int nb,
                                double* __restrict__ R) {
  const int lane = threadIdx.x, i = kb + lane;
  const bool in = lane < nb;
  double r[4];
  for (int q = 0; q < 4; ++q) r[q] = in ? R[4 * i + q] : 0.0;
  for (int k = 0; k < nb; ++k) {
    double y[4];
    if (lane == k) {
      const double inv = 1.0 / L[(size_t)i * n + i];
      for (int q = 0; q < 4; ++q) r[q] *= inv;
    }
    for (int q = 0; q < 4; ++q) y[q] = __shfl_sync(0xffffffffu, r[q], k);
    if (in && lane > k) {
      const double l = L[(size_t)i * n + kb + k];
      for (int q = 0; q < 4; ++q) r[q] -= l * y[q];
    }
  }
  if (in)
    for (int q = 0; q < 4; ++q) R[4 * i + q] = r[q];
}

// back: diagonal block [kb, kb+nb) of L^T x = R (upper triangular rows of Lt)
__global__ void k_trsv_diag_bwd(const double* __restrict__ Lt, int n, int kb, int nb,
                                double* __restrict__ R) {
  const int lane = threadIdx.x, i = kb + lane;
  const bool in = lane < nb;
  double r[4];
  for (int q = 0; q < 4; ++q) r[q] = in ? R[4 * i + q] : 0.0;
  for (int k = nb - 1; k >= 0; --k) {
    double y[4];
    if (lane == k) {
      const double inv = 1.0 / Lt[(size_t)i * n + i];
      for (int q = 0; q < 4; ++q) r[q] *= inv;
    }
    for (int q = 0; q < 4; ++q) y[q] = __shfl_sync(0xffffffffu, r[q], k);
    if (in && lane < k) {
      const double l = Lt[(size_t)i * n + kb + k];
      for (int q = 0; q < 4; ++q) r[q] -= l * y[q];
    }
  }
  if (in)
    for (int q = 0; q < 4; ++q) R[4 * i + q] = r[q];
}

// R[i] -= M[i][kb..kb+nb) . R[kb..kb+nb) for the rows i in [r0, r1)
// (M = L for the forward sweep, rows below the block; M = Lt for the back
// sweep, rows above it).  One warp per row.
__global__ void k_trsv_update(const double* __restrict__ M, int n, int kb, int nb, int r0, int r1,
                              double* __restrict__ R) {
  const int row = r0 + blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= r1) return;
  double s[4] = {0, 0, 0, 0};
  if (lane < nb) {
    const double m = M[(size_t)row * n + kb + lane];
    for (int q = 0; q < 4; ++q) s[q] = m * R[4 * (kb + lane) + q];
  }
  for (int o = 16; o; o >>= 1)
    for (int q = 0; q < 4; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
  if (lane == 0)
    for (int q = 0; q < 4; ++q) R[4 * row + q] -= s[q];
}

static void chol_solve4(bem_ctx* c, const double* L, const double* Lt, int n, double* R) {
  for (int kb = 0; kb < n; kb += 32) {
    const int nb = min(32, n - kb);
    k_trsv_diag_fwd<<<1, 32, 0, S(c)>>>(L, n, kb, nb, R);
    const int r0 = kb + nb;
    if (r0 < n) k_trsv_update<<<(n - r0 + 7) / 8, 256, 0, S(c)>>>(L, n, kb, nb, r0, n, R);
    c->launches += 2;
  }
  for (int kb = (n - 1) / 32 * 32; kb >= 0; kb -= 32) {
    const int nb = min(32, n - kb);
    k_trsv_diag_bwd<<<1, 32, 0, S(c)>>>(Lt, n, kb, nb, R);
    if (kb > 0) k_trsv_update<<<(kb + 7) / 8, 256, 0, S(c)>>>(Lt, n, kb, nb, 0, kb, R);
    c->launches += 2;
  }
}

// delta = y - Z mu, (A^T Z) mu = A^T y with A the three constraint columns.
// X[n][4] = (y, Z0, Z1, Z2); rhs[n][4] holds the constraint columns in 1..3.
__global__ void k_kkt_finish(const double* __restrict__ X, const double* __restrict__ rhs, int n,
                             double* __restrict__ delta, double* __restrict__ gnorm_out,
                             const double* __restrict__ g) {
  __shared__ double red[12 + 1][32];
  double s[13];
  for (int q = 0; q < 13; ++q) s[q] = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      double ac = rhs[4 * i + 1 + a];
      s[a] += ac * X[4 * i];                          // a_a . y
      for (int b = 0; b < 3; ++b) s[3 + 3 * a + b] += ac * X[4 * i + 1 + b];   // a_a . Z_b
    }
    s[12] += g[i] * g[i];
  }
  for (int q = 0; q < 13; ++q)
    for (int o = 16; o; o >>= 1) s[q] += __shfl_down_sync(0xffffffffu, s[q], o);
  if (threadIdx.x % 32 == 0)
    for (int q = 0; q < 13; ++q) red[q][threadIdx.x / 32] = s[q];
  __syncthreads();
  __shared__ double tot[13];
  __shared__ double mu[3];
  if (threadIdx.x < 13) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[threadIdx.x][w];
    tot[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // 3x3 solve by Gaussian elimination with partial pivoting
    double M[3][4];
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) M[a][b] = tot[3 + 3 * a + b];
      M[a][3] = tot[a];
    }
    for (int k = 0; k < 3; ++k) {
      int p = k;
      for (int r = k + 1; r < 3; ++r)
        if (fabs(M[r][k]) > fabs(M[p][k])) p = r;
      for (int q = 0; q < 4; ++q) { double t = M[k][q]; M[k][q] = M[p][q]; M[p][q] = t; }
      double d = M[k][k];
      if (d == 0.0) d = 1e-300;
      for (int r = k + 1; r < 3; ++r) {
        double f = M[r][k] / d;
        for (int q = k; q < 4; ++q) M[r][q] -= f * M[k][q];
      }
    }
    double m3[3];
    for (int k = 2; k >= 0; --k) {
      double t = M[k][3];
      for (int q = k + 1; q < 3; ++q) t -= M[k][q] * m3[q];
      m3[k] = t / (M[k][k] == 0.0 ? 1e-300 : M[k][k]);
    }
    for (int k = 0; k < 3; ++k) mu[k] = m3[k];
    *gnorm_out = sqrt(tot[12]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    delta[i] = X[4 * i] - (X[4 * i + 1] * mu[0] + X[4 * i + 2] * mu[1] + X[4 * i + 3] * mu[2]);
}

int la_lm_solve(bem_ctx* c, const double* H, const double* g, double lam, double* delta) {
  int n = c->sc.nth, rc;
  size_t nn = (size_t)n * n * sizeof(double);
  if ((rc = grow(c, c->lmK, nn))) return rc;
  if ((rc = grow(c, c->lmLt, nn))) return rc;
  if ((rc = grow(c, c->lmL, sizeof(double) * (8 * (size_t)n + 8)))) return rc;
  double* Km = (double*)c->lmK.p;
  double* Lt = (double*)c->lmLt.p;
  double* R = (double*)c->lmL.p;          // [n][4] right-hand sides, then solutions
  double* cons = R + 4 * (size_t)n;       // [n][4] constraint columns
  double* mx = cons + 4 * (size_t)n;
  double* gn = mx + 1;
  if ((rc = cuda_check(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), S(c)), "memset"))) return rc;
  ProfScope _ps(c, "lm_solve");
  dim3 grid((n + 127) / 128, n);
  {
    ProfScope _pb(c, "lm_build");
    k_diag_max<<<1, 1024, 0, S(c)>>>(H, n, mx);
    k_lm_build<<<grid, 128, 0, S(c)>>>(H, g, n, c->sc.C, c->sc.d_closed, c->d_compat, mx, lam, Km, R);
    c->launches += 2;
  }
  const int NB = 32;
  {
  ProfScope _pc(c, "lm_cholesky");
  for (int k0 = 0; k0 < n; k0 += NB) {
    int nb = n - k0 < NB ? n - k0 : NB;
    k_potrf_diag<<<1, 32, 0, S(c)>>>(Km, n, k0, nb, c->d_status);
    BEM_LAUNCHED(c);
    int rest = n - k0 - nb;
    if (rest > 0) {
      k_trsm_rows<<<(rest + 127) / 128, 128, 0, S(c)>>>(Km, n, k0, nb);
      BEM_LAUNCHED(c);
      double* Lp = Km + (size_t)(k0 + nb) * n + k0;
      double* Ct = Km + (size_t)(k0 + nb) * n + k0 + nb;
      la_dgemm(c, false, true, rest, rest, nb, -1.0, Lp, n, Lp, n, 1.0, Ct, n);
    }
  }
  }
  {
    ProfScope _pt(c, "lm_trisolve");
    k_transpose_lower<<<grid, 128, 0, S(c)>>>(Km, n, Lt);
    BEM_LAUNCHED(c);
    chol_solve4(c, Km, Lt, n, R);
  }
  // the constraint columns are needed again for the Schur complement
  k_constraint_cols<<<(n + 255) / 256, 256, 0, S(c)>>>(n, c->d_compat, cons);
  BEM_LAUNCHED(c);
  k_kkt_finish<<<1, 1024, 0, S(c)>>>(R, cons, n, delta, gn, g);
  BEM_LAUNCHED(c);
  if ((rc = cuda_check(c, cudaGetLastError(), "lm solve"))) return rc;
  int st = 0;
  if ((rc = cuda_check(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                                          S(c)), "status")))
    return rc;
  if ((rc = cuda_check(c, cudaStreamSynchronize(S(c)), "lm sync"))) return rc;
  if (st) return fail(c, BEM_ENOTSPD, "LM matrix is not positive definite");
  return BEM_OK;
}

}  // namespace bem
