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
#include <cstring>

#include <algorithm>
#include <vector>

#include "ctx.h"

namespace bem {

// ---------------------------------------------------------------------------
// Gauss-Jordan on the augmented matrix G = [B | I], N rows, 2N columns.

// G = [B | I] with B = A (bordered = 0, N = Nb) or B = [[A, c],[r^T, 0]]
// (bordered = 1, N = Nb + 1; c, r default to the constants).
__global__ void k_gj_init(const double* __restrict__ A, int Nb, int bordered,
                          const double* __restrict__ bcol, const double* __restrict__ brow,
                          double* __restrict__ G) {
  int N = Nb + bordered, W = 2 * N;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)N * W) return;
  int i = idx / W, j = idx % W;
  double v;
  if (j < N) {
    if (i < Nb && j < Nb) v = A[(size_t)i * Nb + j];
    else if (i == Nb && j == Nb) v = 0.0;
    else if (j == Nb) v = bcol ? bcol[i] : 1.0;
    else v = brow ? brow[j] : 1.0;
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

// y = M x (trans = 0, one warp per row) or M^T x (trans = 1, one thread per
// entry); M is n x n with row stride ld.
__global__ void k_mv(const double* __restrict__ M, int ld, int n, int trans,
                     const double* __restrict__ x, double* __restrict__ y) {
  if (trans) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0;
    for (int j = 0; j < n; ++j) s += M[(size_t)j * ld + i] * x[j];
    y[i] = s;
    return;
  }
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, l = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0;
  for (int j = l; j < n; j += 32) s += M[(size_t)row * ld + j] * x[j];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (l == 0) y[row] = s;
}

// x /= |x| (one block)
__global__ void k_normalize(double* __restrict__ x, int n) {
  __shared__ double red[32];
  __shared__ double nrm;
  double s = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i] * x[i];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    nrm = sqrt(t);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] /= nrm;
}

// W = leading Nb x Nb block of the bordered inverse, plus W^T and float copies
__global__ void k_pinv_copy(const double* __restrict__ G, int Nb, double* __restrict__ Wm,
                            double* __restrict__ WT, float* __restrict__ W32,
                            float* __restrict__ WT32) {
  int N = Nb + 1, Wd = 2 * N;
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (j >= Nb) return;
  double w = G[(size_t)i * Wd + N + j];
  Wm[(size_t)i * Nb + j] = w;
  WT[(size_t)j * Nb + i] = w;
  W32[(size_t)i * Nb + j] = float(w);
  WT32[(size_t)j * Nb + i] = float(w);
}

static void gj_run(bem_ctx* c, double* G, int N, double* col) {
  for (int k = 0; k < N; ++k) {
    k_gj_pivot<<<1, 1024, 0, S(c)>>>(G, N, k, col, c->d_status);
    dim3 grid((2 * N + 255) / 256, N);
    k_gj_elim<<<grid, 256, 0, S(c)>>>(G, N, k, col);
    c->launches += 2;
  }
}

// Pseudo-inverse that drops the smallest singular value (Sec. 3.1.3) of a
// matrix that is only nearly singular (galerkin_mode 1): with (s, u, v) the
// smallest singular triple of A, the bordered system [[A, u],[v^T, 0]] is
// well conditioned and [x; m] = its inverse times [f; 0] gives A x + m u = f,
// v.x = 0, i.e. x = sum over the other singular triples of v_k (u_k.f)/s_k.
// v comes from inverse iteration with A^-1 A^-T (Gauss-Jordan inverse of A;
// the gap to the next singular value makes two steps exact to rounding),
// u = A v / |A v|.
static int la_pinv_truncated(bem_ctx* c) {
  int Nb = c->bd.Nb, N = Nb + 1, rc;
  const size_t gsz = (size_t)N * 2 * N;
  if ((rc = grow(c, c->lmW, sizeof(double) * (gsz + N + 3 * (size_t)Nb)))) return rc;
  double* G = (double*)c->lmW.p;
  double* col = G + gsz;
  double* v = col + N;
  double* u = v + Nb;
  double* t = u + Nb;
  if ((rc = cuda_check(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), S(c)), "memset"))) return rc;
  // A^-1
  size_t tot = (size_t)Nb * 2 * Nb;
  k_gj_init<<<(tot + 255) / 256, 256, 0, S(c)>>>(c->bd.d_A, Nb, 0, nullptr, nullptr, G);
  BEM_LAUNCHED(c);
  gj_run(c, G, Nb, col);
  const double* Ainv = G + Nb;   // right half, row stride 2 Nb
  std::vector<double> ones(Nb, 1.0);
  if ((rc = cuda_check(c, cudaMemcpyAsync(v, ones.data(), sizeof(double) * Nb,
                                          cudaMemcpyHostToDevice, S(c)), "copy")))
    return rc;
  for (int it = 0; it < 3; ++it) {
    k_mv<<<(Nb + 255) / 256, 256, 0, S(c)>>>(Ainv, 2 * Nb, Nb, 1, v, t);   // t = A^-T v
    k_mv<<<(Nb + 7) / 8, 256, 0, S(c)>>>(Ainv, 2 * Nb, Nb, 0, t, v);       // v = A^-1 t
    k_normalize<<<1, 1024, 0, S(c)>>>(v, Nb);
    c->launches += 3;
  }
  k_mv<<<(Nb + 7) / 8, 256, 0, S(c)>>>(c->bd.d_A, Nb, Nb, 0, v, u);
  k_normalize<<<1, 1024, 0, S(c)>>>(u, Nb);
  c->launches += 2;
  // bordered inverse with (u, v)
  tot = (size_t)N * 2 * N;
  k_gj_init<<<(tot + 255) / 256, 256, 0, S(c)>>>(c->bd.d_A, Nb, 1, u, v, G);
  BEM_LAUNCHED(c);
  gj_run(c, G, N, col);
  dim3 g2((Nb + 127) / 128, Nb);
  k_pinv_copy<<<g2, 128, 0, S(c)>>>(G, Nb, c->bd.d_W, c->bd.d_WT, c->bd.d_W32, c->bd.d_WT32);
  BEM_LAUNCHED(c);
  if ((rc = cuda_check(c, cudaGetLastError(), "pinv"))) return rc;
  int st = 0;
  if ((rc = cuda_check(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                                          S(c)), "status")) ||
      (rc = cuda_check(c, cudaStreamSynchronize(S(c)), "pinv sync")))
    return rc;
  if (st) return fail(c, BEM_ESINGULAR, "boundary matrix: zero pivot in Gauss-Jordan");
  return BEM_OK;
}

int la_pinv(bem_ctx* c) {
  if (c->opts.galerkin_mode == 1) return la_pinv_truncated(c);
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
  k_gj_init<<<(tot + 255) / 256, 256, 0, S(c)>>>(c->bd.d_A, Nb, 1, nullptr, nullptr, G);
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

// Refined product with the caller's scratch (6 Nb doubles): y = A^+ x by the
// float A^+, then one correction A^+ (x - A y) with the residual in double.
int la_apply3_refined_buf(bem_ctx* c, const float* W32, const double* A, const double* x,
                          double* y, bool transpose, double* scratch) {
  int Nb = c->bd.Nb;
  double* r = scratch;
  double* d = r + 3 * Nb;
  k_apply3_f<<<(Nb + 7) / 8, 256, 0, S(c)>>>(W32, Nb, x, y);
  // A^+ (x - A u): for u = A^+ x exactly this is A^+ P x - A^+ A A^+ x = 0
  k_resid3<<<(Nb + 7) / 8, 256, 0, S(c)>>>(A, Nb, x, y, r, transpose);
  k_apply3_f<<<(Nb + 7) / 8, 256, 0, S(c)>>>(W32, Nb, r, d);
  k_add3<<<(3 * Nb + 255) / 256, 256, 0, S(c)>>>(y, d, 3 * Nb);
  c->launches += 4;
  return cuda_check(c, cudaGetLastError(), "refined apply");
}

// The same with the context's scratch buffer.
int la_apply3_refined(bem_ctx* c, const float* W32, const double* A, const double* x, double* y,
                      bool transpose) {
  int rc;
  if ((rc = grow(c, c->gpart, sizeof(double) * 6 * c->bd.Nb))) return rc;
  return la_apply3_refined_buf(c, W32, A, x, y, transpose, (double*)c->gpart.p);
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
// Parameter t of colour owner h = t / (pp + 6), component t % (pp + 6):
// pp position entries, then w_d (RGB), then w_c (RGB).  Inactive: the
// duplicated end point of a closed Bezier curve (pp = 2).
__device__ __forceinline__ bool param_active(int t, int pp, const uint8_t* closed) {
  if (pp != 2) return true;
  const int h = t / 8, comp = t % 8;
  return !(comp < 2 && (h % 4) == 3 && closed[h / 4]);
}

__global__ void k_lm_build(const double* __restrict__ H, const double* __restrict__ g, int n,
                           int pp, const uint8_t* __restrict__ closed, const double* __restrict__ a,
                           const double* __restrict__ mx, double lam, double* __restrict__ Kmat,
                           double* __restrict__ rhs) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (j >= n) return;
  bool ai = param_active(i, pp, closed), aj = param_active(j, pp, closed);
  double v;
  if (!ai || !aj) v = (i == j) ? 1.0 : 0.0;
  else {
    v = H[(size_t)i * n + j];
    if (i == j) v += lam * fmax(v, 1e-12 * (*mx));
  }
  Kmat[(size_t)i * n + j] = v;
  if (j == 0) {
    const int stride = pp + 6, h = i / stride, comp = i % stride;
    rhs[4 * i] = ai ? -g[i] : 0.0;
    for (int c = 0; c < 3; ++c) rhs[4 * i + 1 + c] = (comp == pp + 3 + c) ? a[h] : 0.0;
  }
}

// cons[n][4]: columns 1..3 = compatibility constraint of channel 0..2
// (a_h at the w_c entry of colour owner h), column 0 unused.
__global__ void k_constraint_cols(int n, int pp, const double* __restrict__ a,
                                  double* __restrict__ cons) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int stride = pp + 6, h = i / stride, comp = i % stride;
  cons[4 * i] = 0.0;
  for (int c = 0; c < 3; ++c) cons[4 * i + 1 + c] = (comp == pp + 3 + c) ? a[h] : 0.0;
}

// Blocked right-looking Cholesky K = L L^T in double, 32-column panels.
// FP64 throughput is low on this GPU, so the sequential parts are kept short:
// the diagonal block is factored by a 32 x 32 thread block and inverted at
// once (recursive doubling), the panel below it is the product with that
// inverse, the trailing update touches the lower triangle only, and the
// triangular solves use the stored diagonal inverses (one launch per block).

// Cholesky of the nb x nb (nb <= 32) diagonal block at (k0, k0) and the
// inverse of its factor into Linv[k0/32] (32 x 32, zero-padded).  Thread
// (r, q) owns entry (r, q).  A pivot that is not positive sets *status.
template <typename T_>
__global__ void __launch_bounds__(1024) k_potrf_inv(T_* __restrict__ Km, int n, int k0, int nb,
                                                    T_* __restrict__ Linv,
                                                    int* __restrict__ status) {
  __shared__ T_ T[32][33];
  __shared__ T_ X[32][33];
  __shared__ T_ Y[32][33];
  __shared__ T_ piv;
  const int q = threadIdx.x & 31, r = threadIdx.x >> 5;
  const bool in = r < nb && q < nb;
  T[r][q] = (in && q <= r) ? Km[(size_t)(k0 + r) * n + k0 + q] : T_(0);
  X[r][q] = T_(0);
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (r == j && q == j) {
      T_ d = T[j][j];
      if (!(d > T_(0))) {
        atomicExch(status, 1);
        d = T_(1);
      }
      const T_ sd = sqrt(d);
      T[j][j] = sd;
      piv = T_(1) / sd;
    }
    __syncthreads();
    if (q == j && r > j && r < nb) T[r][j] *= piv;
    __syncthreads();
    if (q > j && q <= r && r < nb) T[r][q] -= T[r][j] * T[q][j];
    __syncthreads();
  }
  // inverse of the lower-triangular T: diagonal reciprocals, then for block
  // sizes s = 1, 2, 4, 8, 16 the off-diagonal block of every 2s x 2s diagonal
  // block, X_BA = -X_BB T_BA X_AA
  if (r == q && r < nb) X[r][r] = T_(1) / T[r][r];
  __syncthreads();
  for (int sz = 1; sz < 32; sz *= 2) {
    const int base = r / (2 * sz) * (2 * sz);         // start of r's 2s block
    const bool off = (r - base) >= sz && (q - base) >= 0 && (q - base) < sz && r < nb && q < nb;
    if (off) {            // Y = T_BA X_AA  (k over the A block, X_AA lower)
      T_ y = T_(0);
      for (int k = q; k < base + sz; ++k) y += T[r][k] * X[k][q];
      Y[r][q] = y;
    }
    __syncthreads();
    if (off) {            // X_BA = -X_BB Y  (k over the B block, X_BB lower)
      T_ x = T_(0);
      for (int k = base + sz; k <= r; ++k) x -= X[r][k] * Y[k][q];
      X[r][q] = x;
    }
    __syncthreads();
  }
  if (in) Km[(size_t)(k0 + r) * n + k0 + q] = q <= r ? T[r][q] : T_(0);
  Linv[(size_t)(k0 / 32) * 1024 + r * 32 + q] = (in && q <= r) ? X[r][q] : T_(0);
}

// Panel below the diagonal block: L[i][k0 + q] = sum_{l <= q} K[i][k0 + l] Linv[q][l]
// for the rows i >= k0 + nb; one warp per row, lane q computes column q.
template <typename T>
__global__ void __launch_bounds__(256) k_trsm_panel(T* __restrict__ Km, int n, int k0, int nb,
                                                    const T* __restrict__ Linv) {
  __shared__ T Li[32][33];
  for (int e = threadIdx.x; e < 1024; e += blockDim.x)
    Li[e >> 5][e & 31] = Linv[(size_t)(k0 / 32) * 1024 + e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = k0 + nb + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  T* row = Km + (size_t)i * n + k0;
  const T a = lane < nb ? row[lane] : T(0);
  T x = T(0);
  for (int l = 0; l < nb; ++l) {
    const T al = __shfl_sync(0xffffffffu, a, l);
    if (l <= lane) x += al * Li[lane][l];
  }
  if (lane < nb) row[lane] = x;
}

// Trailing update on the lower triangle: K[i][j] -= sum_l P[i][l] P[j][l]
// over 64 x 64 tiles (bi, bj), bj <= bi, of the rows/columns >= r0, with the
// panel P = K[:, k0 .. k0+nb).  Diagonal tiles are computed whole; the strict
// upper triangle of K is never read.
template <typename T>
__global__ void __launch_bounds__(256) k_syrk_lower(T* __restrict__ Km, int n, int k0, int nb,
                                                    int r0) {
  __shared__ T Pa[32][65];
  __shared__ T Pb[32][65];
  int t = blockIdx.x, bi = 0;
  while (t > bi) { t -= bi + 1; ++bi; }
  const int bj = t;
  const int i0 = r0 + bi * 64, j0 = r0 + bj * 64;
  for (int e = threadIdx.x; e < 64 * 32; e += 256) {
    const int rr = e >> 5, l = e & 31;
    const int gi = i0 + rr, gj = j0 + rr;
    Pa[l][rr] = (gi < n && l < nb) ? Km[(size_t)gi * n + k0 + l] : T(0);
    Pb[l][rr] = (gj < n && l < nb) ? Km[(size_t)gj * n + k0 + l] : T(0);
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int l = 0; l < nb; ++l) {
    T pa[4], pb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) pa[a] = Pa[l][ty + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) pb[b] = Pb[l][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += pa[a] * pb[b];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int gi = i0 + ty + 16 * a;
    if (gi >= n) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gj = j0 + tx + 16 * b;
      if (gj < n) Km[(size_t)gi * n + gj] -= acc[a][b];
    }
  }
}

// One block step of the forward solve L y = b with four right-hand sides
// R[n][4]: every CTA forms y_k = Linv_k b_k for block k (CTA 0 stores it in
// Y), then subtracts L[i][block k] y_k from the rows i below the block that
// it owns (one warp per row).  b_k is final when step k starts.
__global__ void __launch_bounds__(256) k_trsv_fwd_step(const double* __restrict__ L, int n, int kb,
                                                       int nb, const double* __restrict__ Linv,
                                                       double* __restrict__ R, double* __restrict__ Y) {
  __shared__ double bk[32][4];
  __shared__ double yk[32][4];
  const int tid = threadIdx.x;
  if (tid < 128) bk[tid >> 2][tid & 3] = (tid >> 2) < nb ? R[4 * (kb + (tid >> 2)) + (tid & 3)] : 0.0;
  __syncthreads();
  if (tid < 128) {
    const int rr = tid >> 2, qq = tid & 3;
    const double* li = Linv + (size_t)(kb / 32) * 1024 + rr * 32;
    double y = 0.0;
    for (int l = 0; l <= rr; ++l) y += li[l] * bk[l][qq];
    yk[rr][qq] = y;
    if (blockIdx.x == 0 && rr < nb) Y[4 * (kb + rr) + qq] = y;
  }
  __syncthreads();
  const int lane = tid & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int row = kb + nb + (int)((blockIdx.x * blockDim.x + tid) >> 5); row < n; row += nw) {
    const double m = lane < nb ? L[(size_t)row * n + kb + lane] : 0.0;
    double s[4];
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) s[qq] = m * yk[lane][qq];
    for (int o = 16; o; o >>= 1)
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) s[qq] += __shfl_xor_sync(0xffffffffu, s[qq], o);
    if (lane == 0)
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) R[4 * row + qq] -= s[qq];
  }
}

// One block step of the back solve L^T x = y: every CTA forms
// x_k = Linv_k^T y_k (CTA 0 stores it in X), then subtracts
// sum_r L[kb + r][i] x_r from the rows i < kb that it owns (one thread per row).
__global__ void __launch_bounds__(256) k_trsv_bwd_step(const double* __restrict__ L, int n, int kb,
                                                       int nb, const double* __restrict__ Linv,
                                                       double* __restrict__ Yv, double* __restrict__ X) {
  __shared__ double yk[32][4];
  __shared__ double xk[32][4];
  const int tid = threadIdx.x;
  if (tid < 128) yk[tid >> 2][tid & 3] = (tid >> 2) < nb ? Yv[4 * (kb + (tid >> 2)) + (tid & 3)] : 0.0;
  __syncthreads();
  if (tid < 128) {
    const int rr = tid >> 2, qq = tid & 3;
    const double* li = Linv + (size_t)(kb / 32) * 1024;
    double x = 0.0;
    for (int l = rr; l < 32; ++l) x += li[l * 32 + rr] * yk[l][qq];
    xk[rr][qq] = x;
    if (blockIdx.x == 0 && rr < nb) X[4 * (kb + rr) + qq] = x;
  }
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + tid; i < kb; i += gridDim.x * blockDim.x) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int rr = 0; rr < nb; ++rr) {
      const double m = L[(size_t)(kb + rr) * n + i];
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) s[qq] += m * xk[rr][qq];
    }
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) Yv[4 * i + qq] -= s[qq];
  }
}

// Blocked Cholesky of the n x n matrix in the lower triangle of Km (in place)
// with the diagonal-block inverses in Linv.
template <typename T>
static void chol_factor(bem_ctx* c, T* Km, int n, T* Linv, int* status) {
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int nb = std::min(32, n - k0);
    k_potrf_inv<T><<<1, 1024, 0, S(c)>>>(Km, n, k0, nb, Linv, status);
    BEM_LAUNCHED(c);
    const int r0 = k0 + nb, rest = n - r0;
    if (rest > 0) {
      k_trsm_panel<T><<<(rest + 7) / 8, 256, 0, S(c)>>>(Km, n, k0, nb, Linv);
      const int tiles = (rest + 63) / 64;
      k_syrk_lower<T><<<tiles * (tiles + 1) / 2, 256, 0, S(c)>>>(Km, n, k0, nb, r0);
      c->launches += 2;
    }
  }
}

// One 32-column step of the float Cholesky in a single launch.  Every CTA
// factors the 32 x 32 diagonal block of the working matrix Kf in one warp
// (the same arithmetic in every CTA, so the same bits).  The last CTA also
// inverts the factor and stores L_kk and its inverse; CTA (bi, bj), bj <= bi, forms the
// panel rows of its two 64-row blocks by forward substitution,
// P = A_panel L_kk^-T, and subtracts P_I P_J^T from its tile of the trailing
// matrix.  The factor goes to Lf (the panel rows of block bi by CTA (bi, 0))
// so that no CTA writes what another reads; Kf keeps the trailing updates.
__global__ void __launch_bounds__(256) k_chol_step_f32(float* __restrict__ Kf, float* __restrict__ Lf,
                                                       int n, int k0, float* __restrict__ Linv,
                                                       int* __restrict__ status,
                                                       float* __restrict__ bad_pivot) {
  __shared__ float T[32][33], X[32][33];
  __shared__ float Araw[2][64][33];
  __shared__ float P[2][32][65];
  __shared__ float rdg[32];
  const int tid = threadIdx.x;
  const int nb = min(32, n - k0), r0 = k0 + nb;
  const bool diag_cta = blockIdx.x == gridDim.x - 1;
  int bi = 0, bj = 0, i0 = 0, j0 = 0, nsides = 0;
  if (!diag_cta) {
    int t = blockIdx.x;
    while (t > bi) { t -= bi + 1; ++bi; }
    bj = t;
    i0 = r0 + 64 * bi;
    j0 = r0 + 64 * bj;
    nsides = bi == bj ? 1 : 2;
  }
  // loads, all issued before the first use so that one round trip covers
  // them: the diagonal block, (tile CTAs) the raw panel rows of I and J and
  // the CTA's tile of the trailing matrix (no other CTA of the launch writes
  // the panel columns or this tile)
  const int tx = tid & 15, ty = tid >> 4;
  float old[4][4];
  {
    float tv[4], av[16];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u, r = e >> 5, q = e & 31;
      tv[u] = (r < nb && q <= r) ? Kf[(size_t)(k0 + r) * n + k0 + q] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * u, sd = e >> 11, rr = (e >> 5) & 63, l = e & 31;
      const int g = (sd == 0 ? i0 : j0) + rr;
      av[u] = (!diag_cta && sd < nsides && g < n && l < nb) ? Kf[(size_t)g * n + k0 + l] : 0.f;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * b;
        old[a][b] = (!diag_cta && gi < n && gj < n) ? Kf[(size_t)gi * n + gj] : 0.f;
      }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u;
      T[e >> 5][e & 31] = tv[u];
    }
    if (!diag_cta)
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = tid + 256 * u;
        Araw[e >> 11][(e >> 5) & 63][e & 31] = av[u];
      }
  }
  __syncthreads();
  // ---- factor the diagonal block in warp 0: lane r holds row r in
  // registers; column j: pivot from lane j, l_rj = a_rj / sqrt(pivot) for
  // r > j, then a_rq -= l_rj l_qj with l_qj shuffled from lane q (entries
  // above the diagonal are left as garbage and never used)
  if (tid < 32) {
    const int r = tid;
    float a[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) a[q] = T[r][q];
    float rd = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j < nb) {
        float d = __shfl_sync(0xffffffffu, a[j], j);
        if (!(d > 0.f)) {
          // the first failing pivot (all CTAs compute the same one)
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
    for (int q = 0; q < 32; ++q) T[r][q] = (q <= r && r < nb) ? a[q] : 0.f;
    rdg[r] = r < nb ? rd : 0.f;
    if (diag_cta) {
      // inverse, lane c computes column c: X_rc = (delta_rc - sum_{k=c}^{r-1} L_rk X_kc) / L_rr
      // with L_rk shuffled from lane r (row r of the factor)
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
  }
  __syncthreads();
  if (diag_cta) {
    for (int e = tid; e < 1024; e += 256) {
      const int r = e >> 5, q = e & 31;
      if (r < nb && q < nb) Lf[(size_t)(k0 + r) * n + k0 + q] = q <= r ? T[r][q] : 0.f;
      Linv[(size_t)(k0 / 32) * 1024 + e] = (r < nb && q <= r) ? X[r][q] : 0.f;
    }
    return;
  }
  // ---- panel rows by forward substitution: x_q = (a_q - sum_{l<q} x_l L_ql) / L_qq
  if (tid < 128) {
    const int sd = tid >> 6, rr = tid & 63;
    if (sd < nsides) {
      float x[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        float v = Araw[sd][rr][q];
#pragma unroll
        for (int l = 0; l < q; ++l) v = fmaf(-x[l], T[q][l], v);
        x[q] = q < nb ? v * rdg[q] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 32; ++q) P[sd][q][rr] = x[q];
    }
  }
  __syncthreads();
  if (bj == 0) {
    for (int e = tid; e < 64 * 32; e += 256) {
      const int rr = e >> 5, q = e & 31;
      const int g = i0 + rr;
      if (g < n && q < nb) Lf[(size_t)g * n + k0 + q] = P[0][q][rr];
    }
  }
  const float (*PJ)[65] = P[nsides - 1];
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int l = 0; l < nb; ++l) {
    float pa[4], pb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) pa[a] = P[0][l][ty + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) pb[b] = PJ[l][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(pa[a], pb[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int gi = i0 + ty + 16 * a;
    if (gi >= n) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gj = j0 + tx + 16 * b;
      if (gj < n) Kf[(size_t)gi * n + gj] = old[a][b] - acc[a][b];
    }
  }
}

// Mixed-precision solve of the LM system (iterative refinement, e.g. Carson
// and Higham 2018): the equilibrated matrix d_i K_ij d_j (d_i = K_ii^-1/2) is
// factored in float; each refinement step solves with that factor and
// updates X in double against the double residual R - K X.

// Kf[i][j] = float(d_i K[i][j] d_j) on the lower triangle, d_i = 1/sqrt(K_ii)
__global__ void k_equilibrate(const double* __restrict__ K, int n, float* __restrict__ Kf,
                              double* __restrict__ d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j > i || j >= n) return;
  const double di = rsqrt(K[(size_t)i * n + i]), dj = rsqrt(K[(size_t)j * n + j]);
  Kf[(size_t)i * n + j] = float(di * K[(size_t)i * n + j] * dj);
  if (j == 0) d[i] = di;
}

// ---- explicit inverse of the float factor (systems below the blocked size)
//
// W = L^-1 by recursive doubling over the 32-row blocks: on a pair of s-row
// ranges, L = [[A, 0], [B, C]] has the inverse [[A^-1, 0], [-C^-1 B A^-1,
// C^-1]].  Level s takes every pair (a0 = 2 p s, c0 = a0 + s) at once:
// first T = B W_A, then W_CA = -W_C T; the 32 x 32 diagonal blocks are the
// factor's block inverses.  W lives in the lower triangle of an n x n float
// matrix.  T is kept transposed in the strictly upper triangle (rows
// [a0, c0), columns [c0, c0 + s)), which no later level reads; a last pass
// mirrors the lower triangle into the upper one, so that row k holds column
// k of W from the diagonal on.  Each refinement solve is then two parallel
// matrix-vector products, z = W^T (W b), where a substitution would take
// 2 n / 32 block steps one after another.

// W's diagonal blocks from the factor's block inverses (zeros above the
// diagonal included)
__global__ void __launch_bounds__(1024) k_inv_init(const float* __restrict__ Linv, int n,
                                                   float* __restrict__ W) {
  const int b = blockIdx.x, i = 32 * b + (threadIdx.x >> 5), j = 32 * b + (threadIdx.x & 31);
  if (i < n && j < n) W[(size_t)i * n + j] = Linv[(size_t)b * 1024 + threadIdx.x];
}

// T = B W_A for every pair of level s (blockIdx.z = pair), one 32 x 32 tile
// per CTA: T[i][j] = sum_k L[c0+i][a0+k] W[a0+k][a0+j], k from the tile's
// first column on (W_A is lower triangular), stored at W[a0+j][c0+i].  The
// next 32-column chunk is loaded into registers while the current one is used.
__global__ void __launch_bounds__(256) k_inv_level_t(const float* __restrict__ Lf,
                                                     float* __restrict__ W, int n, int s) {
  __shared__ float As[32][33], Bs[32][33];
  const int a0 = 2 * s * blockIdx.z, c0 = a0 + s, sC = min(s, n - c0);
  const int i0 = 32 * blockIdx.y, j0 = 32 * blockIdx.x;
  if (i0 >= sC) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float av[4], bv[4], acc[4] = {0.f, 0.f, 0.f, 0.f};
  auto load = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = ty + 8 * u;
      av[u] = i0 + r < sC ? Lf[(size_t)(c0 + i0 + r) * n + a0 + k0 + tx] : 0.f;
      bv[u] = W[(size_t)(a0 + k0 + r) * n + a0 + j0 + tx];
    }
  };
  load(j0);
  for (int k0 = j0; k0 < s; k0 += 32) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) { As[ty + 8 * u][tx] = av[u]; Bs[ty + 8 * u][tx] = bv[u]; }
    __syncthreads();
    if (k0 + 32 < s) load(k0 + 32);
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const float b = Bs[kk][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmaf(As[ty + 8 * u][kk], b, acc[u]);
    }
  }
  // transposed store through shared memory: As[j][i] = T[i][j]
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) As[tx][ty + 8 * u] = acc[u];
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int jj = ty + 8 * u;
    if (i0 + tx < sC) W[(size_t)(a0 + j0 + jj) * n + c0 + i0 + tx] = As[jj][tx];
  }
}

// W_CA = -W_C T for every pair of level s: W[c0+i][a0+j] = -sum_k
// W[c0+i][c0+k] T[k][j] with T[k][j] read from W[a0+j][c0+k]; k ends with
// the tile's last row (W_C is lower triangular).
__global__ void __launch_bounds__(256) k_inv_level_w(float* __restrict__ W, int n, int s) {
  __shared__ float As[32][33], Bt[32][33];
  const int a0 = 2 * s * blockIdx.z, c0 = a0 + s, sC = min(s, n - c0);
  const int i0 = 32 * blockIdx.y, j0 = 32 * blockIdx.x;
  if (i0 >= sC) return;
  const int kend = min(i0 + 32, sC);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float av[4], bv[4], acc[4] = {0.f, 0.f, 0.f, 0.f};
  auto load = [&](int k0) {
    const bool kin = k0 + tx < sC;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = ty + 8 * u;
      av[u] = (i0 + r < sC && kin) ? W[(size_t)(c0 + i0 + r) * n + c0 + k0 + tx] : 0.f;
      bv[u] = kin ? W[(size_t)(a0 + j0 + r) * n + c0 + k0 + tx] : 0.f;
    }
  };
  load(0);
  for (int k0 = 0; k0 < kend; k0 += 32) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) { As[ty + 8 * u][tx] = av[u]; Bt[ty + 8 * u][tx] = bv[u]; }
    __syncthreads();
    if (k0 + 32 < kend) load(k0 + 32);
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const float b = Bt[tx][kk];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmaf(As[ty + 8 * u][kk], b, acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = ty + 8 * u;
    if (i0 + r < sC) W[(size_t)(c0 + i0 + r) * n + a0 + j0 + tx] = -acc[u];
  }
}

// W[j][i] = W[i][j] for i > j, one 32 x 32 tile pair (ib >= jb) per CTA.
// Reads touch only the strictly lower triangle, writes only the strictly
// upper one.
__global__ void __launch_bounds__(256) k_inv_mirror(float* __restrict__ W, int n) {
  __shared__ float t[32][33];
  int tt = blockIdx.x, ib = 0;
  while (tt > ib) { tt -= ib + 1; ++ib; }
  const int jb = tt, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = ty + 8 * u, i = 32 * ib + r, j = 32 * jb + tx;
    t[r][tx] = (i < n && i > j) ? W[(size_t)i * n + j] : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = ty + 8 * u, orow = 32 * jb + r, ocol = 32 * ib + tx;
    if (ocol < n && ocol > orow) W[(size_t)orow * n + ocol] = t[tx][r];
  }
}

// One float solve of (D K D) z = D r with the explicit inverse: FWD forms
// y = W (D r); !FWD adds D W^T y to X (double).  One warp per row, the
// n x 4 vector staged in shared memory.  Rres: the double residual R - K X.
template <bool FWD>
__global__ void __launch_bounds__(256) k_inv_apply(const float* __restrict__ W, int n,
                                                   const double* __restrict__ d,
                                                   const double* __restrict__ Rres,
                                                   float* __restrict__ y, double* __restrict__ X) {
  extern __shared__ float4 v4[];   // [n]
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    if constexpr (FWD) {
      const double dk = d[k];
      v4[k] = make_float4(float(dk * Rres[4 * k]), float(dk * Rres[4 * k + 1]),
                          float(dk * Rres[4 * k + 2]), float(dk * Rres[4 * k + 3]));
    } else {
      v4[k] = reinterpret_cast<const float4*>(y)[k];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= n) return;
  const float* row = W + (size_t)i * n;
  const int ke = FWD ? i + 1 : n;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 4
  for (int k = (FWD ? 0 : i) + lane; k < ke; k += 32) {
    const float m = row[k];
    const float4 v = v4[k];
    s0 = fmaf(m, v.x, s0); s1 = fmaf(m, v.y, s1); s2 = fmaf(m, v.z, s2); s3 = fmaf(m, v.w, s3);
  }
  for (int o = 16; o; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s3 += __shfl_xor_sync(0xffffffffu, s3, o);
  }
  if (lane != 0) return;
  if constexpr (FWD) {
    reinterpret_cast<float4*>(y)[i] = make_float4(s0, s1, s2, s3);
  } else {
    const double di = d[i];
    X[4 * i] += di * double(s0);
    X[4 * i + 1] += di * double(s1);
    X[4 * i + 2] += di * double(s2);
    X[4 * i + 3] += di * double(s3);
  }
}

// Rres = R - K X (double, one warp per row, K full) and per-block sums for
// the normwise backward error: part[block] = (max_q |Rres|, max |R|, max row
// sum |K|, max |X|) over the block's rows.
__global__ void __launch_bounds__(256) k_resid4(const double* __restrict__ K, int n,
                                                const double* __restrict__ R,
                                                const double* __restrict__ X,
                                                double* __restrict__ Rres, double* __restrict__ part) {
  __shared__ double red[8][4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 8 + w;
  double m[4] = {0.0, 0.0, 0.0, 0.0};
  if (i < n) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, a = 0.0;
    const double* row = K + (size_t)i * n;
    for (int j = lane; j < n; j += 32) {
      const double k = row[j];
      s0 += k * X[4 * j]; s1 += k * X[4 * j + 1]; s2 += k * X[4 * j + 2]; s3 += k * X[4 * j + 3];
      a += fabs(k);
    }
    for (int o = 16; o; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      s3 += __shfl_xor_sync(0xffffffffu, s3, o);
      a += __shfl_xor_sync(0xffffffffu, a, o);
    }
    const double r0 = R[4 * i] - s0, r1 = R[4 * i + 1] - s1, r2 = R[4 * i + 2] - s2,
                 r3 = R[4 * i + 3] - s3;
    if (lane == 0) {
      Rres[4 * i] = r0; Rres[4 * i + 1] = r1; Rres[4 * i + 2] = r2; Rres[4 * i + 3] = r3;
    }
    m[0] = fmax(fmax(fabs(r0), fabs(r1)), fmax(fabs(r2), fabs(r3)));
    m[1] = fmax(fmax(fabs(R[4 * i]), fabs(R[4 * i + 1])), fmax(fabs(R[4 * i + 2]), fabs(R[4 * i + 3])));
    m[2] = a;
    m[3] = fmax(fmax(fabs(X[4 * i]), fabs(X[4 * i + 1])), fmax(fabs(X[4 * i + 2]), fabs(X[4 * i + 3])));
  }
  if (lane == 0)
    for (int q = 0; q < 4; ++q) red[w][q] = m[q];
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int k = 0; k < 8; ++k) v = fmax(v, red[k][threadIdx.x]);
    part[4 * blockIdx.x + threadIdx.x] = v;
  }
}

// eta = |R - K X|_max / (|K|_inf |X|_max + |R|_max) from the block partials
__global__ void k_backward_error(const double* __restrict__ part, int nblk,
                                 double* __restrict__ eta) {
  __shared__ double red[4][32];
  double m[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
    for (int q = 0; q < 4; ++q) m[q] = fmax(m[q], part[4 * b + q]);
  for (int o = 16; o; o >>= 1)
    for (int q = 0; q < 4; ++q) m[q] = fmax(m[q], __shfl_xor_sync(0xffffffffu, m[q], o));
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x >> 5] = m[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < 4; ++q)
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) red[q][0] = fmax(red[q][0], red[q][w]);
    const double den = red[2][0] * red[3][0] + red[1][0];
    *eta = den > 0.0 ? red[0][0] / den : 0.0;
  }
}

// Solve K X = R (four right-hand sides) with the factor in the lower
// triangle of L and the diagonal inverses in Linv; the solution replaces R.
// Y: scratch [n][4].
static void chol_solve4(bem_ctx* c, const double* L, const double* Linv, int n, double* R,
                        double* Y) {
  const int grid = std::max(1, std::min(c->sms, (n + 255) / 256));
  for (int kb = 0; kb < n; kb += 32) {
    k_trsv_fwd_step<<<std::max(1, std::min(c->sms, (n - kb + 7) / 8)), 256, 0, S(c)>>>(
        L, n, kb, std::min(32, n - kb), Linv, R, Y);
    BEM_LAUNCHED(c);
  }
  for (int kb = (n - 1) / 32 * 32; kb >= 0; kb -= 32) {
    k_trsv_bwd_step<<<grid, 256, 0, S(c)>>>(L, n, kb, std::min(32, n - kb), Linv, Y, R);
    BEM_LAUNCHED(c);
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

// Refinement: checked from step kRefineCheck on, at most kRefineMax steps,
// converged when the normwise backward error is below kRefineTol.
constexpr int kRefineCheck = 2, kRefineMax = 10;
constexpr double kRefineTol = 1e-14;
constexpr int kBlockedMinN = 2048, kMaxBlockedSolve = 32768;
constexpr float kIndefinitePivot = -1e-2f;

int la_lm_solve(bem_ctx* c, const double* H, const double* g, double lam, double* delta) {
  int n = c->sc.nth, rc;
  size_t nn = (size_t)n * n * sizeof(double);
  const size_t nblk = ((size_t)n + 31) / 32;
  const size_t rblk = ((size_t)n + 7) / 8;
  if ((rc = grow(c, c->lmK, nn))) return rc;
  if ((rc = grow(c, c->lmLt, sizeof(double) * 1024 * nblk))) return rc;
  const size_t nb64 = ((size_t)n + 63) / 64;
  if ((rc = grow(c, c->lmW, nn + sizeof(float) * std::max<size_t>(1024 * nblk, 4096 * nb64) + 256)))
    return rc;
  if ((rc = grow(c, c->lmL, sizeof(double) * (25 * (size_t)n + 4 * rblk + 16)))) return rc;
  double* Km = (double*)c->lmK.p;
  double* Linv = (double*)c->lmLt.p;      // [n/32][32][32] inverses of the diagonal blocks
  float* Kf = (float*)c->lmW.p;           // equilibrated matrix in float (trailing updates)
  float* Lf = Kf + (size_t)n * n;         // its float Cholesky factor (lower triangle)
  float* Linvf = Lf + (size_t)n * n;      // the factor's diagonal-block inverses
                                          // (32 x 32 blocks; 64 x 64 when blocked)
  double* R = (double*)c->lmL.p;          // [n][4] right-hand sides, then solutions
  double* cons = R + 4 * (size_t)n;       // [n][4] constraint columns
  double* Ytmp = cons + 4 * (size_t)n;    // [n][4] forward-solve result (double path;
                                          // float y of the inverse solves)
  double* Rres = Ytmp + 4 * (size_t)n;    // [n][4] refinement residual
  double* Xs = Rres + 4 * (size_t)n;      // [n][4] refined solution
  double* dsc = Xs + 4 * (size_t)n;       // [n] equilibration
  double* epart = dsc + (size_t)n;        // [rblk][4] backward-error partials
  double* eta_d = epart + 4 * rblk;
  int* fstat = (int*)(eta_d + 1);
  float* fpiv = (float*)(eta_d + 1) + 1;
  double* mx = eta_d + 2;
  double* gn = mx + 1;
  if ((rc = cuda_check(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), S(c)), "memset"))) return rc;
  ProfScope _ps(c, "lm_solve");
  dim3 grid((n + 127) / 128, n);
  {
    ProfScope _pb(c, "lm_build");
    k_diag_max<<<1, 1024, 0, S(c)>>>(H, n, mx);
    k_lm_build<<<grid, 128, 0, S(c)>>>(H, g, n, c->sc.pp, c->sc.d_closed, c->d_compat, mx, lam, Km, R);
    c->launches += 2;
  }
  // float factor of the equilibrated matrix, refined in double; the double
  // factorization is the fallback when the float one fails or stalls
  bool done = false;
  // large systems: 64-column blocked factor and the cluster solve; below
  // kBlockedMinN the 32-column step kernel, the explicit inverse of the
  // factor (written over Kf, which the factor no longer needs) and two
  // matrix-vector products per solve
  const bool blocked = n >= kBlockedMinN;
  if (c->opts.lm_solver == BEM_LM_AUTO && (blocked ? n <= kMaxBlockedSolve : true)) {
    int fst = 0;
    {
      ProfScope _pc(c, "lm_cholesky");
      k_equilibrate<<<dim3((n + 127) / 128, n), 128, 0, S(c)>>>(Km, n, Kf, dsc);
      BEM_LAUNCHED(c);
      if ((rc = cuda_check(c, cudaMemsetAsync(fstat, 0, 2 * sizeof(int), S(c)), "memset"))) return rc;
      if (blocked) {
        chol_blocked_f32(c, Kf, Lf, n, Linvf, fstat, fpiv);
      } else {
        for (int k0 = 0; k0 < n; k0 += 32) {
          const int tiles = (n - std::min(n, k0 + 32) + 63) / 64;
          k_chol_step_f32<<<tiles * (tiles + 1) / 2 + 1, 256, 0, S(c)>>>(Kf, Lf, n, k0, Linvf,
                                                                           fstat, fpiv);
          BEM_LAUNCHED(c);
        }
      }
    }
    // a failed float factor is known before any solve with it (the pivot
    // status and value sit in the word after eta_d)
    bool factored = true;
    {
      double h1 = 0;
      if ((rc = cuda_check(c, cudaMemcpyAsync(&h1, eta_d + 1, sizeof(double), cudaMemcpyDeviceToHost, S(c)), "pivot")) ||
          (rc = cuda_check(c, cudaStreamSynchronize(S(c)), "factor sync")))
        return rc;
      std::memcpy(&fst, &h1, sizeof(int));
      if (fst) {
        float pv;
        std::memcpy(&pv, reinterpret_cast<const char*>(&h1) + sizeof(int), sizeof(float));
        if (pv < kIndefinitePivot || c->opts.precision == BEM_MIXED)
          return fail(c, BEM_ENOTSPD, "LM matrix is not positive definite");
        factored = false;     // the double factor decides
      }
    }
    if (factored && !blocked) {
      ProfScope _pi(c, "lm_inverse");
      const int nblk32 = (n + 31) / 32;
      k_inv_init<<<nblk32, 1024, 0, S(c)>>>(Linvf, n, Kf);
      BEM_LAUNCHED(c);
      for (int s = 32; s < n; s *= 2) {
        const dim3 g(s / 32, s / 32, (n - s + 2 * s - 1) / (2 * s));   // pairs with c0 < n
        k_inv_level_t<<<g, 256, 0, S(c)>>>(Lf, Kf, n, s);
        k_inv_level_w<<<g, 256, 0, S(c)>>>(Kf, n, s);
        c->launches += 2;
      }
      k_inv_mirror<<<nblk32 * (nblk32 + 1) / 2, 256, 0, S(c)>>>(Kf, n);
      BEM_LAUNCHED(c);
    }
    ProfScope _pt(c, "lm_trisolve");
    if (factored &&
        ((rc = cuda_check(c, cudaMemcpyAsync(Rres, R, sizeof(double) * 4 * n, cudaMemcpyDeviceToDevice, S(c)), "copy")) ||
         (rc = cuda_check(c, cudaMemsetAsync(Xs, 0, sizeof(double) * 4 * n, S(c)), "memset"))))
      return rc;
    const int rblk = (n + 7) / 8;
    const size_t vsmem = sizeof(float) * 4 * (size_t)n;   // below 48 KB for n < kBlockedMinN
    float* yf = reinterpret_cast<float*>(Ytmp);
    if (blocked && (rc = trsv_cluster_prepare(c, n))) return rc;
    // X += float solve of the residual Rres
    auto correct = [&]() {
      if (blocked) {
        trsv_cluster_f32(c, Lf, Linvf, n, dsc, Rres, Xs);
      } else {
        k_inv_apply<true><<<rblk, 256, vsmem, S(c)>>>(Kf, n, dsc, Rres, yf, nullptr);
        k_inv_apply<false><<<rblk, 256, vsmem, S(c)>>>(Kf, n, dsc, nullptr, yf, Xs);
        c->launches += 2;
      }
    };
    double eta = 1.0, eta_prev = 2.0;
    for (int it = 0; factored && it < kRefineMax; ++it) {
      correct();
      k_resid4<<<rblk, 256, 0, S(c)>>>(Km, n, R, Xs, Rres, epart);
      k_backward_error<<<1, 256, 0, S(c)>>>(epart, rblk, eta_d);
      c->launches += 2;
      if (it + 1 < kRefineCheck) continue;
      double h[2];
      if ((rc = cuda_check(c, cudaMemcpyAsync(h, eta_d, 2 * sizeof(double), cudaMemcpyDeviceToHost, S(c)), "eta")) ||
          (rc = cuda_check(c, cudaStreamSynchronize(S(c)), "refine sync")))
        return rc;
      std::memcpy(&fst, &h[1], sizeof(int));
      if (fst) {
        // the float factor hit a non-positive pivot.  The equilibrated
        // matrix has a unit diagonal, so float rounding moves a pivot by
        // about n * 6e-8; a pivot far below zero means the matrix itself is
        // not positive definite, which the double factor would only confirm.
        // In a mixed context H is a bf16 Gram matrix, accurate to about 1e-2
        // of its largest entries: a damped matrix that float cannot factor
        // counts as not positive definite there, and the step raises the
        // damping instead of factoring it in double.
        float pv;
        std::memcpy(&pv, reinterpret_cast<const char*>(&h[1]) + sizeof(int), sizeof(float));
        if (pv < kIndefinitePivot || c->opts.precision == BEM_MIXED)
          return fail(c, BEM_ENOTSPD, "LM matrix is not positive definite");
        break;
      }
      eta_prev = it + 1 == kRefineCheck ? 2.0 : eta;
      eta = h[0];
      if (eta < kRefineTol) {
        // one more correction with the residual just formed: the test
        // bounds the residual normwise, which on a badly scaled K still
        // leaves an error of up to cond(K) times it in X, and each
        // correction shrinks the error by about cond(D K D) times the float
        // rounding unit
        correct();
        done = true;
        break;
      }
      if (!(eta < 0.5 * eta_prev)) break;  // stalled
    }
    if (done &&
        (rc = cuda_check(c, cudaMemcpyAsync(R, Xs, sizeof(double) * 4 * n, cudaMemcpyDeviceToDevice, S(c)), "copy")))
      return rc;
  }
  if (!done) {
    ProfScope _pc(c, "lm_cholesky_fp64");
    chol_factor<double>(c, Km, n, Linv, c->d_status);
    chol_solve4(c, Km, Linv, n, R, Ytmp);
  }
  // the constraint columns are needed again for the Schur complement
  k_constraint_cols<<<(n + 255) / 256, 256, 0, S(c)>>>(n, c->sc.pp, c->d_compat, cons);
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
