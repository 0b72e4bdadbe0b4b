// Tensor-core contractions of the Gauss-Newton matrix (tcgen05, TMEM, TMA).
//
// Every product here has the form D[M][N] = sum_k A[m][k] B[n][k] with both
// operands K-major in global memory (row-major, k contiguous).  One CTA of 4
// warps computes one 128 x 128 tile: lane 0 of warp 0 streams 64-wide K slabs
// of A and B into a 3-stage shared-memory ring with TMA (128-byte swizzle),
// lane 0 of warp 1 issues tcgen05.mma (M = N = 128, K = 16 per instruction)
// into a 128-column fp32 accumulator in TMEM and releases ring slots with
// tcgen05.commit, and all four warps drain the accumulator (warp w owns TMEM
// lanes 32w..32w+31) through the epilogue of the launch mode:
//   EPI_STORE  D -> fp32 [M][N]
//   EPI_JROWS  J^T = M_c^T Phi^T + F^T: D + F (fp32) -> bf16 [M][N]
//   EPI_SYRK   one upper-triangular 128 x 128 block of J_c^T J_c over a K
//              slice of samples, added to that slice's fp32 partial sum
// Every wait is bounded (about one second); a timeout sets *err and the CTA
// drains and frees its TMEM before returning.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "ctx.h"
#include "umma.cuh"

namespace bem {

namespace {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int STAGES = 3;
constexpr int TILE_BYTES = BM * BK * 2;     // 16 KB per operand per stage
constexpr int SMEM_BYTES = 1024 + STAGES * 2 * TILE_BYTES + 256;

enum { EPI_STORE = 0, EPI_JROWS = 1, EPI_SYRK = 2 };

struct TcArgs {
  int M, N, K;
  int mode;
  float* D;                 // EPI_STORE
  int ldd;
  const float* F;           // EPI_JROWS
  int ldf;
  __nv_bfloat16* J;
  int ldj;
  int nc, tiles, npairs;    // EPI_SYRK
  int k_per_split;
  float* part;              // [splits][3][nc][nc]
  int* err;
};

__global__ void __launch_bounds__(128, 2)
    k_tc_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
              TcArgs g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * TILE_BYTES;
  uint64_t* full = (uint64_t*)(sB + STAGES * TILE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // ---- tile coordinates
  int arow, brow, kb, ke, ch = 0, ti = 0, tj = 0;
  if (g.mode == EPI_SYRK) {
    ch = blockIdx.x / g.npairs;
    int p = blockIdx.x % g.npairs;
    // p -> (ti, tj), ti <= tj, row-major over the upper triangle
    ti = 0;
    while (p >= g.tiles - ti) { p -= g.tiles - ti; ++ti; }
    tj = ti + p;
    arow = ch * g.nc + ti * BM;
    brow = ch * g.nc + tj * BN;
    kb = blockIdx.y * g.k_per_split;
    ke = min(g.K, kb + g.k_per_split);
  } else {
    arow = blockIdx.x * BM;
    brow = blockIdx.y * BN;
    kb = 0;
    ke = g.K;
  }
  const int nk = ke > kb ? (ke - kb + BK - 1) / BK : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    umma::mbar_init(done, 1);
    umma::fence_barrier_init();
  }
  if (warp == 0) umma::tmem_alloc(tmem_slot, 128);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (it / STAGES) & 1;
      if (!umma::mbar_wait(&empty[s], ph ^ 1, g.err)) break;
      umma::mbar_expect_tx(&full[s], 2 * TILE_BYTES);
      const int kc = kb + it * BK;
      umma::tma_load_2d(sA + s * TILE_BYTES, &tA, &full[s], kc, arow);
      umma::tma_load_2d(sB + s * TILE_BYTES, &tB, &full[s], kc, brow);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t id = umma::idesc(1, BM, BN);
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (it / STAGES) & 1;
      if (!umma::mbar_wait(&full[s], ph, g.err)) break;
      umma::fence_after();
      const uint32_t a0 = umma::smem_u32(sA + s * TILE_BYTES);
      const uint32_t b0 = umma::smem_u32(sB + s * TILE_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)
        umma::mma_bf16(tmem, umma::sdesc_sw128(a0 + kk * 32), umma::sdesc_sw128(b0 + kk * 32), id,
                       (it | kk) != 0);
      umma::mma_commit(&empty[s]);
    }
    umma::mma_commit(done);
  }
  __syncwarp();
  // ---- epilogue: all four warps
  const bool ok = umma::mbar_wait(done, 0, g.err);
  umma::fence_after();
  const int r = warp * 32 + lane;     // row of the tile owned by this thread
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
  for (int cb = 0; cb < BN; cb += 32) {
    float v[32];
    umma::tmem_ld32(trow + cb, v);
    if (!ok || nk == 0) {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = 0.f;
    }
    if (g.mode == EPI_STORE) {
      const int row = arow + r;
      if (row < g.M) {
        float* d = g.D + (size_t)row * g.ldd + brow + cb;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (brow + cb + j < g.N) d[j] = v[j];
      }
    } else if (g.mode == EPI_JROWS) {
      const int row = arow + r;
      if (row < g.M) {
        const float* f = g.F + (size_t)row * g.ldf + brow + cb;
        __nv_bfloat16* o = g.J + (size_t)row * g.ldj + brow + cb;
        if (brow + cb + 32 <= g.N) {
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            float4 fv = *reinterpret_cast<const float4*>(f + j);
            __nv_bfloat162 p0 = __floats2bfloat162_rn(v[j] + fv.x, v[j + 1] + fv.y);
            __nv_bfloat162 p1 = __floats2bfloat162_rn(v[j + 2] + fv.z, v[j + 3] + fv.w);
            uint2 w;
            w.x = *reinterpret_cast<uint32_t*>(&p0);
            w.y = *reinterpret_cast<uint32_t*>(&p1);
            *reinterpret_cast<uint2*>(o + j) = w;
          }
        } else {
          for (int j = 0; j < 32; ++j)
            if (brow + cb + j < g.N) o[j] = __float2bfloat16_rn(v[j] + f[j]);
        }
      }
    } else {
      const int i = ti * BM + r;
      if (i < g.nc) {
        float* d = g.part + (((size_t)blockIdx.y * 3 + ch) * g.nc + i) * g.nc;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = tj * BN + cb + j;
          if (col < g.nc) d[col] += v[j];
        }
      }
    }
  }
  umma::fence_before();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, 128);
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// bf16 K-major operand [rows][ld], inner extent k, boxes of 64 x 128
int make_map(bem_ctx* c, CUtensorMap* m, const void* base, uint64_t k, uint64_t rows,
             uint64_t ld) {
  auto enc = encoder();
  if (!enc) return fail(c, BEM_ECUDA, "cuTensorMapEncodeTiled is not available");
  if (((uintptr_t)base & 15) || (ld * 2) % 16)
    return fail(c, BEM_EINVAL, "tensor-core operand not 16-byte aligned");
  cuuint64_t dims[2] = {k, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {BK, BM};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, BEM_ECUDA, "cuTensorMapEncodeTiled failed");
  return BEM_OK;
}

int launch(bem_ctx* c, const CUtensorMap& a, const CUtensorMap& b, const TcArgs& g, dim3 grid) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return cuda_check(c, e, "tc gemm smem attribute");
    attr = true;
  }
  k_tc_gemm<<<grid, 128, SMEM_BYTES, S(c)>>>(a, b, g);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "k_tc_gemm");
}

}  // namespace

// D[M][N] = A[M][K] B[N][K]^T, bf16 in, fp32 out (all device, row-major).
int tc_gemm_store(bem_ctx* c, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                  float* D, int ldd) {
  int rc;
  CUtensorMap ta, tb;
  if ((rc = make_map(c, &ta, A, K, M, lda)) || (rc = make_map(c, &tb, B, K, N, ldb))) return rc;
  TcArgs g{};
  g.M = M; g.N = N; g.K = K; g.mode = EPI_STORE; g.D = D; g.ldd = ldd; g.err = c->d_status;
  return launch(c, ta, tb, g, dim3((M + BM - 1) / BM, (N + BN - 1) / BN));
}

// J[rows][m] = bf16(Mt[rows][Nb] Phi[m][Nb]^T + F[rows][m])
int tc_jrows(bem_ctx* c, int rows, int m, int Nb, const void* Mt, int ldm, const void* Phi,
             int ldp, const float* F, int ldf, void* J, int ldj) {
  int rc;
  CUtensorMap ta, tb;
  if ((rc = make_map(c, &ta, Mt, Nb, rows, ldm)) || (rc = make_map(c, &tb, Phi, Nb, m, ldp)))
    return rc;
  if ((ldf % 4) || ((uintptr_t)F & 15)) return fail(c, BEM_EINVAL, "F rows not 16-byte aligned");
  TcArgs g{};
  g.M = rows; g.N = m; g.K = Nb; g.mode = EPI_JROWS; g.F = F; g.ldf = ldf;
  g.J = (__nv_bfloat16*)J; g.ldj = ldj; g.err = c->d_status;
  ProfScope _ps(c, "tc_jrows");
  return launch(c, ta, tb, g, dim3((rows + BM - 1) / BM, (m + BN - 1) / BN));
}

// part[split][ch][nc][nc] += upper blocks of J_ch^T J_ch over the m samples of J
// (J rows ch*nc .. ch*nc+nc-1 hold channel ch), K split into `splits` slices.
int tc_syrk(bem_ctx* c, int nc, int m, const void* J, int ldj, float* part, int splits) {
  int rc;
  CUtensorMap tj;
  if ((rc = make_map(c, &tj, J, m, 3 * nc, ldj))) return rc;
  TcArgs g{};
  g.M = g.N = nc; g.K = m; g.mode = EPI_SYRK; g.nc = nc;
  g.tiles = (nc + BM - 1) / BM;
  g.npairs = g.tiles * (g.tiles + 1) / 2;
  g.k_per_split = ((m + splits - 1) / splits + BK - 1) / BK * BK;
  g.part = part; g.err = c->d_status;
  int sp = (m + g.k_per_split - 1) / g.k_per_split;
  ProfScope _ps(c, "tc_syrk");
  return launch(c, tj, tj, g, dim3(3 * g.npairs, sp));
}

int tc_syrk_splits(int nc) {
  int tiles = (nc + BM - 1) / BM;
  int ctas = 3 * tiles * (tiles + 1) / 2;
  return std::max(1, std::min(64, (2 * 152 + ctas - 1) / ctas));
}

}  // namespace bem
