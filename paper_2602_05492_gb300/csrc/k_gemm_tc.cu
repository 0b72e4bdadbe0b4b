// Tensor-core contractions of the Gauss-Newton matrix (tcgen05, TMEM, TMA).
//
// Every product here has the form D[M][N] = sum_k A[m][k] B[n][k] with both
// operands K-major in global memory (row-major, k contiguous).  One CTA of 4
// warps computes one 128 x 128 tile: lane 0 of warp 0 streams 128-byte-wide
// K slabs of A and B into a 3-stage shared-memory ring with TMA (128-byte
// swizzle), lane 0 of warp 1 issues tcgen05.mma (M = N = 128) into a
// 128-column fp32 accumulator in TMEM and releases ring slots with
// tcgen05.commit, and all four warps drain the accumulator (warp w owns TMEM
// lanes 32w..32w+31) through the epilogue of the launch mode.
// Three operand schemes:
//   bf16    one kind::f16 product, 64-element slabs, K = 16 per instruction
//   bf16x3  (compensated bf16) bf16 hi + lo parts of every operand (x = hi +
//           lo, lo the rounded rest); three kind::f16 products lo.hi + hi.lo
//           + hi.hi accumulate into the same TMEM tile
//   3xtf32  fp32 operands stored as tf32 hi + lo parts; three kind::tf32
//           products (32-element slabs, K = 8)
// Epilogues of the per-tile kernel k_tc_gemm:
//   EPI_STORE  D -> fp32 [M][N] (bem_gemm_bf16)
//   EPI_JROWS  J^T = M_c^T Phi^T + F^T: the tf32 hi/lo pair of D + F (3xtf32)
//   EPI_SYRK   one 128 x 128 block of J_c^T J_c over a K slice of samples,
//              added to that slice's fp32 partial sums by TMA reductions
//              (bf16x3 and 3xtf32; the bf16 Gram blocks run in
//              k_tc_syrk_pair, two blocks per CTA that share an operand slab)
// The bf16 and bf16x3 J rows run in a persistent, warp-specialised kernel
// (k_tc_jrows_pers): one CTA per SM, a producer warp, an MMA warp and eight
// epilogue warps, with two TMEM accumulators so that a tile's epilogue
// overlaps the next tile's MMAs, and TMA loads and stores in the epilogue.
// Every wait is bounded.  The pipeline waits (a ring slot, a TMEM buffer)
// give up after the context's limit (bem_set_wait_limit, one second by
// default); the waits that guard work already in flight (copies landing in
// shared memory, MMAs writing TMEM) after one second whatever that limit.  A
// timeout sets *err, and the CTA lets its copies and MMAs finish and frees
// its TMEM before returning.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "ctx.h"
#include "umma.cuh"

namespace bem {

namespace {

constexpr int BM = 128, BN = 128;
constexpr int STAGES = 3;
constexpr int TILE_BYTES = BM * 128;        // 16 KB: 128 rows x 128 bytes per operand part
template <int SCH> struct Scheme {
  static constexpr bool X3 = SCH != SCH_BF16;
  static constexpr bool TF32 = SCH == SCH_TF32X3;
  static constexpr int BK = TF32 ? 32 : 64;           // elements per 128-byte row
  static constexpr int PARTS = X3 ? 4 : 2;            // A(hi, lo), B(hi, lo) / A, B
  static constexpr int SMEM = 1024 + STAGES * PARTS * TILE_BYTES + 256;
};

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

enum { EPI_STORE = 0, EPI_JROWS = 1, EPI_SYRK = 2 };

struct TcArgs {
  int M, N, K;
  int mode;
  float* D;                 // EPI_STORE
  int ldd;
  const float* F;           // EPI_JROWS
  int ldf;
  __nv_bfloat16* J;          // bf16 scheme
  void* Jhi;                  // split schemes: tf32 parts as fp32, or bf16 parts
  void* Jlo;
  int ldj;
  int nc, tiles, npairs;    // EPI_SYRK
  int k_per_split;
  float* part;              // [splits][3][nc][nc]
  int* err;
  uint64_t wait_ns;         // limit of the pipeline waits (ring slots, TMEM buffers)
  JLayout L;                // J^T row layout (EPI_JROWS gradient, EPI_SYRK tiles)
  // bf16 J rows (k_tc_jrows_pers) with residuals: for each J^T row and each
  // channel c whose column col it holds (JLayout), gpart[(c gnc + col) *
  // gstride + 64-sample block] = sum over the block's samples s of F[row][s]
  // resid[s][c]
  const float* resid;
  int gnc;
  float* gpart;
  int64_t gstride;
};

template <int SCH>
__global__ void __launch_bounds__(128, Scheme<SCH>::X3 ? 1 : 2)
    k_tc_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
              const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tB2,
              const __grid_constant__ CUtensorMap tP, TcArgs g) {
  constexpr int BK = Scheme<SCH>::BK, PARTS = Scheme<SCH>::PARTS;
  constexpr bool X3 = Scheme<SCH>::X3, TF = Scheme<SCH>::TF32;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // stage s holds parts p = 0..PARTS-1 at smem + (s * PARTS + p) * TILE_BYTES:
  // bf16: A, B;  3xtf32: A hi, B hi, A lo, B lo
  uint64_t* full = (uint64_t*)(smem + STAGES * PARTS * TILE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  int* gave_up = (int*)(tmem_slot + 1);   // set when the MMA warp stopped early

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // ---- tile coordinates
  int arow, brow, kb, ke, ch = 0, ti = 0, tj = 0;
  if (g.mode == EPI_SYRK) {
    // channel 0 takes every upper block of its channel-order tiles (npairs
    // of them), channels 1 and 2 the npairs1 blocks whose row tile lies in
    // the position range; the jump-jump blocks are channel 0's for all three
    const int npairs1 = g.tiles * g.L.ptiles() - g.L.ptiles() * (g.L.ptiles() - 1) / 2;
    int p = blockIdx.x;
    ch = 0;
    if (p >= g.npairs) {
      p -= g.npairs;
      ch = 1 + p / npairs1;
      p %= npairs1;
    }
    // p -> (ti, tj), ti <= tj, row-major over the upper triangle
    ti = 0;
    while (p >= g.tiles - ti) { p -= g.tiles - ti; ++ti; }
    tj = ti + p;
    arow = g.L.tile_row(ch, ti);
    brow = g.L.tile_row(ch, tj);
    kb = blockIdx.y * g.k_per_split;
    ke = min(g.K, kb + g.k_per_split);
  } else {
    arow = blockIdx.x * BM;
    brow = blockIdx.y * BN;
    kb = 0;
    ke = g.K;
  }
  const int nk = ke > kb ? (ke - kb + BK - 1) / BK : 0;   // BK of the scheme

  if (threadIdx.x == 0) {
    *gave_up = 0;
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

  // a diagonal Gram tile multiplies a tile of J^T by itself: one load serves
  // as both operands
  const bool same_ab = g.mode == EPI_SYRK && ti == tj;
  if (warp == 0 && lane == 0) {
    // TMA producer
    int issued = 0;
    for (int it = 0; it < nk; ++it, issued = it) {
      const int s = it % STAGES;
      const uint32_t ph = (it / STAGES) & 1;
      if (!umma::mbar_wait(&empty[s], ph ^ 1, g.err, g.wait_ns)) break;
      umma::mbar_expect_tx(&full[s], (same_ab ? PARTS / 2 : PARTS) * TILE_BYTES);
      const int kc = kb + it * BK;
      uint8_t* st = smem + (size_t)s * PARTS * TILE_BYTES;
      umma::tma_load_2d(st, &tA, &full[s], kc, arow);
      if (!same_ab) umma::tma_load_2d(st + TILE_BYTES, &tB, &full[s], kc, brow);
      if (X3) {
        umma::tma_load_2d(st + 2 * TILE_BYTES, &tA2, &full[s], kc, arow);
        if (!same_ab) umma::tma_load_2d(st + 3 * TILE_BYTES, &tB2, &full[s], kc, brow);
      }
    }
    // the loads still in flight (after a timeout) land before the CTA can leave
    for (int j = issued > STAGES ? issued - STAGES : 0; j < issued; ++j)
      umma::mbar_wait(&full[j % STAGES], (j / STAGES) & 1, g.err);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t id = umma::idesc(TF ? 2 : 1, BM, BN);
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (it / STAGES) & 1;
      if (!umma::mbar_wait(&full[s], ph, g.err, g.wait_ns)) {
        *(volatile int*)gave_up = 1;
        break;
      }
      umma::fence_after();
      const uint32_t a0 = umma::smem_u32(smem + (size_t)s * PARTS * TILE_BYTES);
      const uint32_t b0 = same_ab ? a0 : a0 + TILE_BYTES;
      // each instruction consumes 32 bytes of every row (16 bf16 or 8 tf32)
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t da = umma::sdesc_sw128(a0 + kk * 32);
        const uint64_t db = umma::sdesc_sw128(b0 + kk * 32);
        if (X3) {
          const uint64_t dal = umma::sdesc_sw128(a0 + 2 * TILE_BYTES + kk * 32);
          const uint64_t dbl = umma::sdesc_sw128(b0 + 2 * TILE_BYTES + kk * 32);
          if (TF) {
            umma::mma_tf32(tmem, dal, db, id, (it | kk) != 0);   // lo . hi
            umma::mma_tf32(tmem, da, dbl, id, 1);                 // hi . lo
            umma::mma_tf32(tmem, da, db, id, 1);                  // hi . hi
          } else {
            umma::mma_bf16(tmem, dal, db, id, (it | kk) != 0);
            umma::mma_bf16(tmem, da, dbl, id, 1);
            umma::mma_bf16(tmem, da, db, id, 1);
          }
        } else {
          umma::mma_bf16(tmem, da, db, id, (it | kk) != 0);
        }
      }
      umma::mma_commit(&empty[s]);
    }
    umma::mma_commit(done);
  }
  __syncwarp();
  // ---- epilogue: all four warps (the guard limit: MMAs may be in flight)
  const bool ok = umma::mbar_wait(done, 0, g.err) && *(volatile int*)gave_up == 0;
  umma::fence_after();
  const int r = warp * 32 + lane;     // row of the tile owned by this thread
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  // the stage ring is free once the accumulator is complete (EPI_SYRK stages
  // its boxes there)
  float* fs = reinterpret_cast<float*>(smem);
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
    } else if (g.mode == EPI_JROWS && X3) {
      const int row = arow + r;
      if (row < g.M) {
        const float* f = g.F + (size_t)row * g.ldf + brow + cb;
        const size_t o = (size_t)row * g.ldj + brow + cb;
        for (int j = 0; j < 32; ++j)
          if (brow + cb + j < g.N) {
            const float x = v[j] + f[j];
            if (TF) {
              const float hi = tf32_rna(x);
              ((float*)g.Jhi)[o + j] = hi;
              ((float*)g.Jlo)[o + j] = tf32_rna(x - hi);
            } else {
              const __nv_bfloat16 hi = __float2bfloat16_rn(x);
              ((__nv_bfloat16*)g.Jhi)[o + j] = hi;
              ((__nv_bfloat16*)g.Jlo)[o + j] = __float2bfloat16_rn(x - __bfloat162float(hi));
            }
          }
      }
    } else {
      // EPI_SYRK: stage the row in box cb / 32 (128 rows x 32 fp32 columns,
      // 128-byte swizzle) of the idle ring, for the TMA reduction below
      uint8_t* row = reinterpret_cast<uint8_t*>(fs + (cb >> 5) * (BM * 32)) + r * 128;
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8)
        *reinterpret_cast<float4*>(row + ((c8 ^ (r & 7)) << 4)) =
            make_float4(v[4 * c8], v[4 * c8 + 1], v[4 * c8 + 2], v[4 * c8 + 3]);
    }
  }
  if (g.mode == EPI_SYRK) {
    // the block += into this K slice's partial sums (rows of part[slice][ch])
    umma::fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0 && ok && nk > 0) {
      const int y = ((int)blockIdx.y * 3 + ch) * g.L.cdim() + ti * BM;
      for (int k4 = 0; k4 < 4; ++k4)
        umma::tma_reduce_add_2d(&tP, fs + k4 * (BM * 32), tj * BN + 32 * k4, y);
      umma::bulk_commit();
      umma::bulk_wait0();
    }
  }
  umma::fence_before();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, 128);
}

// ---- bf16 J rows, persistent ----------------------------------------------
// One CTA per SM walks the tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// of 128 rows x 256 samples (t = row tile + col tile * row tiles, so
// consecutive tiles share their Phi tile).  Warp 0 lane 0 streams A/B slabs
// (A 128 rows, B 256 rows as two 128-row boxes) through a ring of stages (TMA),
// warp 1 lane 0 issues M = 128, N = 256 MMAs into one of two 256-column TMEM
// accumulators, and warps 2..9 drain the other in two passes of 128 columns:
// warp w owns TMEM lanes 32 (w % 4) .. +31 and the columns 64 ((w - 2) / 4)
// .. +63 of the pass.  The epilogue of a tile (F rows added, bf16 packing,
// the handle part of the gradient) overlaps the MMAs of the next.  One
// 256-sample tile per MMA halves the operand bytes per output of the A slabs
// against 128-sample tiles, the share of the L2 traffic that bounds this
// contraction.  The epilogue runs as two independent halves of four warps,
// half h owning the columns 64 h .. 64 h + 63 of every pass, with their own
// load barrier, named barrier and leader thread, and it moves its data with
// TMA as well: the leader loads the half's F rows of a pass as two 128-row x
// 32-column boxes (128-byte swizzle: row r at 128 r bytes, 16-byte chunk c at
// position c ^ (r & 7)) and its residuals by one bulk copy, and stores the
// half's J^T rows as a 64-column bf16 box in the same swizzle.  The bf16 rows
// of half h are packed in place over F box 2 h, which only that half's warps
// read, and each thread reads its row of the box before it writes there.
// Compensated bf16 (BF16X3) runs the same kernel on 128-sample tiles: a
// stage holds the hi and lo parts of the A and B slabs (64 KB, two stages),
// each K step issues the three products lo.hi, hi.lo, hi.hi into one
// 128-column accumulator, and the epilogue writes the hi and lo parts of
// J^T, hi over F box 2 h and lo over F box 2 h + 1 after the thread has read
// its row of both.
template <bool X3>
struct Pers {
  static constexpr int BNT = X3 ? 128 : 256;               // samples per tile
  static constexpr int PASSES = BNT / BN;                  // epilogue passes of BN columns
  static constexpr int STAGES = X3 ? 2 : 3;
  static constexpr int STAGE = X3 ? 4 * TILE_BYTES : TILE_BYTES * (1 + PASSES);
  static constexpr int SMEM = 1024 + STAGES * STAGE + BM * BN * 4 + 3 * BN * 4 + 256;
  static_assert(SMEM <= 227 * 1024, "persistent J-row kernel exceeds shared memory");
};
constexpr int kPersThreads = 320;           // 2 control warps + 8 epilogue warps

// the named barrier of epilogue half h (its four warps)
__device__ __forceinline__ void bar_half(int h) {
  if (h) asm volatile("bar.sync 3, 128;" ::: "memory");
  else asm volatile("bar.sync 2, 128;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_u32(bar)) : "memory");
}

// bf16 of x and of its rounding remainder
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// tA, tB: the hi (or only) parts of M^T and Phi; tA2, tB2: their lo parts
// (X3); tF: F^T; tJ, tJ2: J^T (hi and lo parts for X3)
template <bool X3>
__global__ void __launch_bounds__(kPersThreads, 1)
    k_tc_jrows_pers(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
                    const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tB2,
                    const __grid_constant__ CUtensorMap tF, const __grid_constant__ CUtensorMap tJ,
                    const __grid_constant__ CUtensorMap tJ2, TcArgs g) {
  using P = Pers<X3>;
  constexpr int BK = Scheme<SCH_BF16>::BK;
  constexpr int BNT = P::BNT, PASSES = P::PASSES, STAGES = P::STAGES, STAGE = P::STAGE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* fs = reinterpret_cast<float*>(smem + STAGES * STAGE);         // 4 boxes [BM][32] F rows
  float* rs = fs + BM * BN;                                            // [2][64][3] residuals
  uint64_t* full = reinterpret_cast<uint64_t*>(rs + 3 * BN);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* fbar = tempty + 2;                              // [2] a half's F rows landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fbar + 2);
  int* fail_flag = reinterpret_cast<int*>(tmem_slot + 1);   // set when an epilogue wait gave up
  int* stop_flag = fail_flag + 1;                           // set when the MMA warp gave up
  int* half_ok = stop_flag + 1;                             // [2] a half's view of fail_flag

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rtiles = (g.M + BM - 1) / BM, ctiles = (g.N + BNT - 1) / BNT;
  const int ntiles = rtiles * ctiles;
  const int nk = (g.K + BK - 1) / BK;
  if (threadIdx.x == 0) {
    *fail_flag = 0;
    *stop_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      umma::mbar_init(&tfull[b], 1);
      umma::mbar_init(&tempty[b], 8);
    }
    umma::mbar_init(&fbar[0], 1);
    umma::mbar_init(&fbar[1], 1);
    umma::fence_barrier_init();
  }
  if (warp == 0) umma::tmem_alloc(tmem_slot, 2 * BNT);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer over all of this CTA's tiles
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int arow = (t % rtiles) * BM, brow = (t / rtiles) * BNT;
        for (int kk = 0; kk < nk; ++kk, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          if (!umma::mbar_wait(&empty[s], ph ^ 1, g.err, g.wait_ns)) { ok = false; break; }
          umma::mbar_expect_tx(&full[s], STAGE);
          uint8_t* st = smem + (size_t)s * STAGE;
          umma::tma_load_2d(st, &tA, &full[s], kk * BK, arow);
          if constexpr (X3) {
            // A hi, B hi, A lo, B lo
            umma::tma_load_2d(st + TILE_BYTES, &tB, &full[s], kk * BK, brow);
            umma::tma_load_2d(st + 2 * TILE_BYTES, &tA2, &full[s], kk * BK, arow);
            umma::tma_load_2d(st + 3 * TILE_BYTES, &tB2, &full[s], kk * BK, brow);
          } else {
#pragma unroll
            for (int p = 0; p < PASSES; ++p)
              umma::tma_load_2d(st + (1 + p) * TILE_BYTES, &tB, &full[s], kk * BK, brow + p * BN);
          }
        }
      }
      // the last loads of every slot have landed before the CTA can leave
      for (int j = it > STAGES ? it - STAGES : 0; j < it; ++j)
        umma::mbar_wait(&full[j % STAGES], (j / STAGES) & 1, g.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: tile i of this CTA accumulates into TMEM buffer i & 1
      const uint32_t id = umma::idesc(1, BM, BNT);
      int it = 0, i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        const int b = i & 1;
        if (!umma::mbar_wait(&tempty[b], ((i >> 1) & 1) ^ 1, g.err, g.wait_ns)) {
          *(volatile int*)stop_flag = 1;
          break;
        }
        umma::fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * BNT);
        for (int kk = 0; kk < nk; ++kk, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          if (!umma::mbar_wait(&full[s], ph, g.err, g.wait_ns)) {
            // the epilogue learns from stop_flag, after this tile's commit,
            // that no further tile follows
            *(volatile int*)stop_flag = 1;
            ok = false;
            break;
          }
          umma::fence_after();
          const uint32_t a0 = umma::smem_u32(smem + (size_t)s * STAGE);
          const uint32_t b0 = a0 + TILE_BYTES;   // bf16: 256 rows, two 128-row boxes back to back
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4) {
            const uint64_t da = umma::sdesc_sw128(a0 + k4 * 32), db = umma::sdesc_sw128(b0 + k4 * 32);
            if constexpr (X3) {
              const uint64_t dal = umma::sdesc_sw128(a0 + 2 * TILE_BYTES + k4 * 32);
              const uint64_t dbl = umma::sdesc_sw128(b0 + 2 * TILE_BYTES + k4 * 32);
              umma::mma_bf16(acc, dal, db, id, (kk | k4) != 0);   // lo . hi
              umma::mma_bf16(acc, da, dbl, id, 1);                // hi . lo
              umma::mma_bf16(acc, da, db, id, 1);                 // hi . hi
            } else {
              umma::mma_bf16(acc, da, db, id, (kk | k4) != 0);
            }
          }
          umma::mma_commit(&empty[s]);
        }
        umma::mma_commit(&tfull[b]);
      }
    }
  } else {
    // epilogue, 256 threads in two halves of four warps; half h owns the
    // columns 64 h .. 64 h + 63 of every pass (F boxes 2 h and 2 h + 1, the
    // J^T box or boxes over them) and runs its own pipeline: its leader
    // thread loads and stores its boxes, its warps sync on their own named
    // barrier, and each thread writes the gradient partial of its row and 64
    // columns
    const int et = threadIdx.x - 64;                 // 0 .. 255
    const int q = warp & 3, half = (warp - 2) >> 2;  // TMEM lane quarter, column half
    const int r = 32 * q + lane;                     // tile row of this thread
    const int sw = r & 7;
    const bool leader = (et & 127) == 0;
    float* rh = rs + half * (3 * 64);                // residuals of the half's 64 columns
    float* fb = fs + 2 * half * (BM * 32);           // the half's two F boxes
    uint64_t* fh = fbar + half;
    // leader: the half's F rows (two TMA boxes) and residuals of pass p of tile t
    auto load_half = [&](int t, int p) {
      const int arow = (t % rtiles) * BM, c0 = (t / rtiles) * BNT + p * BN + 64 * half;
      const bool rbulk = g.gpart && c0 + 64 <= g.N;
      if (g.gpart && !rbulk)   // the chunk's ragged end: zeros past it
        for (int e = 0; e < 3 * 64; ++e) {
          const int col = c0 + e / 3;
          rh[e] = col < g.N ? g.resid[3 * (size_t)col + e % 3] : 0.f;
        }
      umma::mbar_expect_tx(fh, 2 * BM * 32 * 4 + (rbulk ? 3 * 64 * 4 : 0));
      if (rbulk) umma::bulk_load(rh, g.resid + 3 * (size_t)c0, 3 * 64 * 4, fh);
      umma::tma_load_2d(fb, &tF, fh, c0, arow);
      umma::tma_load_2d(fb + BM * 32, &tF, fh, c0 + 32, arow);
    };
    // pass k of this CTA: tile blockIdx.x + (k / passes) gridDim.x, pass k % passes
    const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int npass = my_tiles * PASSES;
    if (leader && npass > 0) load_half(blockIdx.x, 0);
    int issued = npass > 0 ? 1 : 0;   // loads issued (leader)
    bool ok = true;
    int k = 0;
    for (; k < npass && ok; ++k) {
      const int t = (int)blockIdx.x + (k / PASSES) * (int)gridDim.x, p = k % PASSES;
      const int i = k / PASSES, b = i & 1;
      const int arow = (t % rtiles) * BM, ct = t / rtiles;
      const int c0 = ct * BNT + p * BN + 64 * half;
      if (p == 0) {
        // (the guard limit: MMAs of this buffer may still be in flight)
        if (!umma::mbar_wait(&tfull[b], (i >> 1) & 1, g.err)) atomicOr(fail_flag, 1);
        umma::fence_after();
        if (*(volatile int*)stop_flag) atomicOr(fail_flag, 1);
      }
      // (guard limit: the copies of this pass are in flight)
      if (!umma::mbar_wait(fh, k & 1, g.err)) atomicOr(fail_flag, 1);
      if (leader) half_ok[half] = *(volatile int*)fail_flag == 0;
      bar_half(half);
      ok = half_ok[half] != 0;   // one value for the whole half
      // gradient rows: a position row sums against its channel's
      // residual; a jump row (the whole tile, since the jump range starts
      // on a tile) against all three
      const bool jump = arow >= 3 * g.L.Pp;
      int gch = 0;
      if (g.gpart && !jump) gch = (arow + r) / g.L.Pp;
      float gacc = 0.f, gacc1 = 0.f, gacc2 = 0.f;
      // bf16: the half's rows go over its F box 2 h, after this thread has
      // read its row of that box; X3: hi over box 2 h and lo over box 2 h + 1,
      // after it has read its row of both
      uint8_t* ob = reinterpret_cast<uint8_t*>(fb) + r * 128;
      uint8_t* ob2 = reinterpret_cast<uint8_t*>(fb + BM * 32) + r * 128;
      float fx[X3 ? 32 : 1];   // X3: the row of box 2 h + 1, read up front
      if constexpr (X3) {
        const uint8_t* fr1 = reinterpret_cast<const uint8_t*>(fb + BM * 32) + r * 128;
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
          const float4 w4 = *reinterpret_cast<const float4*>(fr1 + ((c8 ^ sw) << 4));
          fx[4 * c8] = w4.x; fx[4 * c8 + 1] = w4.y; fx[4 * c8 + 2] = w4.z; fx[4 * c8 + 3] = w4.w;
        }
      }
#pragma unroll 1
      for (int s2 = 0; s2 < 2; ++s2) {
        float v[32];
        umma::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) +
                            (uint32_t)(b * BNT + p * BN + 64 * half + 32 * s2),
                        v);
        if (!ok) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0.f;
        }
        float f[32];
        if (X3 && s2 == 1) {
#pragma unroll
          for (int j = 0; j < 32; ++j) f[j] = fx[X3 ? j : 0];
        } else {
          const uint8_t* fr = reinterpret_cast<const uint8_t*>(fb + s2 * (BM * 32)) + r * 128;
#pragma unroll
          for (int c8 = 0; c8 < 8; ++c8) {
            const float4 w4 = *reinterpret_cast<const float4*>(fr + ((c8 ^ sw) << 4));
            f[4 * c8] = w4.x; f[4 * c8 + 1] = w4.y; f[4 * c8 + 2] = w4.z; f[4 * c8 + 3] = w4.w;
          }
        }
        const float* rr = rh + 3 * 32 * s2;
        if (g.gpart && !jump) {
#pragma unroll
          for (int j = 0; j < 32; ++j) gacc = fmaf(f[j], rr[3 * j + gch], gacc);
        } else if (g.gpart) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            gacc = fmaf(f[j], rr[3 * j], gacc);
            gacc1 = fmaf(f[j], rr[3 * j + 1], gacc1);
            gacc2 = fmaf(f[j], rr[3 * j + 2], gacc2);
          }
        }
        // output chunks 4 s2 .. 4 s2 + 3 of the row (8 bf16 each)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          uint4 w, w2;
          uint32_t* wp = &w.x;
          uint32_t* wp2 = &w2.x;
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float x0 = v[8 * kk + 2 * h] + f[8 * kk + 2 * h];
            const float x1 = v[8 * kk + 2 * h + 1] + f[8 * kk + 2 * h + 1];
            if constexpr (X3) {
              __nv_bfloat16 h0, l0, h1, l1;
              split_bf16(x0, h0, l0);
              split_bf16(x1, h1, l1);
              const __nv_bfloat162 bh(h0, h1), bl(l0, l1);
              wp[h] = *reinterpret_cast<const uint32_t*>(&bh);
              wp2[h] = *reinterpret_cast<const uint32_t*>(&bl);
            } else {
              const __nv_bfloat162 b2 = __floats2bfloat162_rn(x0, x1);
              wp[h] = *reinterpret_cast<const uint32_t*>(&b2);
            }
          }
          *reinterpret_cast<uint4*>(ob + (((4 * s2 + kk) ^ sw) << 4)) = w;
          if constexpr (X3) *reinterpret_cast<uint4*>(ob2 + (((4 * s2 + kk) ^ sw) << 4)) = w2;
        }
      }
      if (p == PASSES - 1 || !ok) {
        // this warp's TMEM reads of the tile are complete (or given up, and
        // the loop ends after this pass): release the buffer
        umma::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
      // the gradient partial of the row over the half's 64 samples, 64-sample
      // block 2 (128-sample block) + half (a block past the chunk's end holds
      // nothing and is not written)
      if (g.gpart && ok && arow + r < g.M && c0 < g.N) {
        const int row = arow + r;
        const int64_t blk = 2 * (PASSES * ct + p) + half;
        if (!jump) {
          const int ch = row / g.L.Pp, col = row - ch * g.L.Pp;
          if (col < g.L.npos) g.gpart[((size_t)ch * g.gnc + col) * g.gstride + blk] = gacc;
        } else {
          const int w = row - 3 * g.L.Pp;
          if (w < 2 * g.L.nh) {
            const size_t o = (size_t)(g.L.npos + w) * g.gstride + blk;
            g.gpart[o] = gacc;
            g.gpart[(size_t)g.gnc * g.gstride + o] = gacc1;
            g.gpart[2 * (size_t)g.gnc * g.gstride + o] = gacc2;
          }
        }
      }
      umma::fence_proxy_async();   // the bf16 rows, for the TMA store
      bar_half(half);
      if (leader) {
        // the half's J^T rows (rows and columns past the matrix are not
        // written), then its next F rows once the stores have read fb
        umma::tma_store_2d(&tJ, fb, c0, arow);
        if constexpr (X3) umma::tma_store_2d(&tJ2, fb + BM * 32, c0, arow);
        umma::bulk_commit();
        umma::bulk_wait_read0();
        if (ok && k + 1 < npass) {
          const int k1 = k + 1;
          load_half((int)blockIdx.x + (k1 / PASSES) * (int)gridDim.x, k1 % PASSES);
          ++issued;
        }
      }
    }
    if (leader) {
      // a load issued for a pass the loop did not reach lands before the CTA
      // leaves (guard limit), and the stores complete
      if (issued > k) umma::mbar_wait(fh, (issued - 1) & 1, g.err);
      umma::bulk_wait0();
    }
  }
  __syncwarp();
  umma::fence_before();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, 2 * BNT);
}

// ---- bf16 Gram blocks on paired tiles ----------------------------------------
// The upper 128 x 128 blocks (ti <= tj) of each channel's J_c^T J_c are
// grouped into units of two blocks that share an operand slab:
//   kind 1  (ti, tj), (ti, tj + 1): one M = 128, N = 256 MMA on B rows of
//           tiles tj, tj + 1 (the pairs along each block row, from the
//           diagonal on)
//   kind 2  (ti, T - 1), (ti + 2, T - 1): two M = 128, N = 128 MMAs on the
//           same B slab (the last blocks of the rows with an odd count)
//   kind 0  (T - 1, T - 1) when one such block is left over
// A unit streams two or three 16 KB slabs per K step (one fewer where an A
// tile is also the B tile) for two blocks, against two slabs per block
// for single blocks: about a quarter fewer L2 bytes per MMA.
struct SyrkUnit {
  int kind, a0, a1, b;
};

// Odd-count block rows r0, r0 + 2, .. below R of a T x T triangle: their number.
__host__ __device__ __forceinline__ int syrk_odd_rows(int T, int R) {
  const int r0 = (T - 1) & 1;
  return R > r0 ? (R - r0 + 1) / 2 : 0;
}

// unit u of the block rows 0 .. R-1 of the T x T upper block triangle, in the
// order above (also compiled for the host, where bem_gram_unit exposes it to
// the tests for R = T)
__host__ __device__ __forceinline__ SyrkUnit syrk_unit(int T, int R, int u) {
  int np = 0;
  for (int r = 0; r < R; ++r) np += (T - r) / 2;
  SyrkUnit un;
  if (u < np) {
    int r = 0;
    while (u >= (T - r) / 2) { u -= (T - r) / 2; ++r; }
    un.kind = 1; un.a0 = r; un.a1 = r; un.b = r + 2 * u;
  } else {
    u -= np;
    const int r0 = (T - 1) & 1, L = syrk_odd_rows(T, R);   // rows with an odd block count
    if (2 * u + 1 < L) {
      un.kind = 2; un.a0 = r0 + 4 * u; un.a1 = un.a0 + 2; un.b = T - 1;
    } else {
      un.kind = 0; un.a0 = r0 + 4 * u; un.a1 = un.a0; un.b = T - 1;
    }
  }
  return un;
}

__host__ __device__ __forceinline__ int syrk_units(int T, int R) {
  int np = 0;
  for (int r = 0; r < R; ++r) np += (T - r) / 2;
  return np + (syrk_odd_rows(T, R) + 1) / 2;
}

constexpr int SY_STAGES = 4;
constexpr int kSyStage = 3 * TILE_BYTES;     // up to three 128-row slabs (48 KB)
constexpr int kSySmem = 1024 + SY_STAGES * kSyStage + 256;

// part[split][ch][i][j] += the unit's two blocks over its K slice (channel-
// order indices i, j); blockIdx.x = channel 0's units (its whole triangle,
// g.npairs of them), then those of channels 1 and 2 (the rows of their
// position range only: the jump-jump blocks are channel 0's), blockIdx.y =
// K slice.  g.tiles = T channel-order tiles.
__global__ void __launch_bounds__(128, 1)
    k_tc_syrk_pair(const __grid_constant__ CUtensorMap tJ, const __grid_constant__ CUtensorMap tP,
                   TcArgs g) {
  constexpr int BK = Scheme<SCH_BF16>::BK;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + SY_STAGES * kSyStage);
  uint64_t* empty = full + SY_STAGES;
  uint64_t* done = empty + SY_STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  int* gave_up = (int*)(tmem_slot + 1);   // set when the MMA warp stopped early
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ch = 0, u = blockIdx.x;
  const int Tp = g.L.ptiles();
  if (u >= g.npairs) {
    const int n1 = syrk_units(g.tiles, Tp);
    u -= g.npairs;
    ch = 1 + u / n1;
    u %= n1;
  }
  const SyrkUnit un = syrk_unit(g.tiles, ch == 0 ? g.tiles : Tp, u);
  const int kb = blockIdx.y * g.k_per_split, ke = min(g.K, kb + g.k_per_split);
  const int nk = ke > kb ? (ke - kb + BK - 1) / BK : 0;
  // slab 0: A (a0), slab 1: A (a1, kind 2) or B, slab 2: B (kind 2) or B's second tile (kind 1)
  const bool loadA0 = un.kind == 2 || un.a0 != un.b;
  const bool loadA1 = un.kind == 2 && un.a1 != un.b;
  const int nslab = (loadA0 ? 1 : 0) + (loadA1 ? 1 : 0) + (un.kind == 0 ? 1 : 2) - (un.kind == 2 ? 1 : 0);
  if (threadIdx.x == 0) {
    *gave_up = 0;
    for (int s = 0; s < SY_STAGES; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    umma::mbar_init(done, 1);
    umma::fence_barrier_init();
  }
  if (warp == 0) umma::tmem_alloc(tmem_slot, 256);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tmem_slot;
  if (warp == 0 && lane == 0) {
    // TMA producer
    int issued = 0;
    for (int it = 0; it < nk; ++it, issued = it) {
      const int s = it % SY_STAGES;
      const uint32_t ph = (it / SY_STAGES) & 1;
      if (!umma::mbar_wait(&empty[s], ph ^ 1, g.err, g.wait_ns)) break;
      umma::mbar_expect_tx(&full[s], nslab * TILE_BYTES);
      const int kc = kb + it * BK;
      uint8_t* st = smem + (size_t)s * kSyStage;
      if (loadA0) umma::tma_load_2d(st, &tJ, &full[s], kc, g.L.tile_row(ch, un.a0));
      if (un.kind == 2) {
        if (loadA1) umma::tma_load_2d(st + TILE_BYTES, &tJ, &full[s], kc, g.L.tile_row(ch, un.a1));
        umma::tma_load_2d(st + 2 * TILE_BYTES, &tJ, &full[s], kc, g.L.tile_row(ch, un.b));
      } else {
        umma::tma_load_2d(st + TILE_BYTES, &tJ, &full[s], kc, g.L.tile_row(ch, un.b));
        if (un.kind == 1)
          umma::tma_load_2d(st + 2 * TILE_BYTES, &tJ, &full[s], kc, g.L.tile_row(ch, un.b + 1));
      }
    }
    // the loads still in flight (after a timeout) land before the CTA can leave
    for (int j = issued > SY_STAGES ? issued - SY_STAGES : 0; j < issued; ++j)
      umma::mbar_wait(&full[j % SY_STAGES], (j / SY_STAGES) & 1, g.err);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t id128 = umma::idesc(1, BM, BN), id256 = umma::idesc(1, BM, 2 * BN);
    for (int it = 0; it < nk; ++it) {
      const int s = it % SY_STAGES;
      const uint32_t ph = (it / SY_STAGES) & 1;
      if (!umma::mbar_wait(&full[s], ph, g.err, g.wait_ns)) {
        *(volatile int*)gave_up = 1;
        break;
      }
      umma::fence_after();
      const uint32_t s0 = umma::smem_u32(smem + (size_t)s * kSyStage);
      const uint32_t s1 = s0 + TILE_BYTES, s2 = s0 + 2 * TILE_BYTES;
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4) {
        const uint32_t acc = (it | k4) != 0;
        if (un.kind == 2) {
          const uint64_t db = umma::sdesc_sw128(s2 + k4 * 32);
          umma::mma_bf16(tmem, umma::sdesc_sw128(s0 + k4 * 32), db, id128, acc);
          umma::mma_bf16(tmem + BN, umma::sdesc_sw128((loadA1 ? s1 : s2) + k4 * 32), db, id128,
                         acc);
        } else {
          const uint64_t da = umma::sdesc_sw128((loadA0 ? s0 : s1) + k4 * 32);
          umma::mma_bf16(tmem, da, umma::sdesc_sw128(s1 + k4 * 32), un.kind == 1 ? id256 : id128,
                         acc);
        }
      }
      umma::mma_commit(&empty[s]);
    }
    umma::mma_commit(done);
  }
  __syncwarp();
  // ---- epilogue: the unit's blocks are added into this K slice's partial
  // sums by TMA reductions.  Thread r (row r of the unit's row tiles) moves
  // its accumulator row through shared memory (the ring, idle once the MMAs
  // are done) into 128-row x 32-column fp32 boxes in the 128-byte swizzle
  // (row r at 128 r bytes, 16-byte chunk c at position c ^ (r & 7)), and one
  // thread issues the reductions.
  // (the guard limit: MMAs may be in flight)
  const bool ok = umma::mbar_wait(done, 0, g.err) && *(volatile int*)gave_up == 0;
  umma::fence_after();
  const int r = warp * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  const int nout = un.kind == 0 ? 1 : 2;
  float* stage = reinterpret_cast<float*>(smem);   // box (o, c4) at stage + (4 o + c4) BM 32
  if (ok) {
    for (int o = 0; o < nout; ++o) {
#pragma unroll 1
      for (int c4 = 0; c4 < 4; ++c4) {
        float v[32];
        umma::tmem_ld32(trow + o * BN + 32 * c4, v);
        uint8_t* row = reinterpret_cast<uint8_t*>(stage + (4 * o + c4) * (BM * 32)) + r * 128;
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8)
          *reinterpret_cast<float4*>(row + ((c8 ^ (r & 7)) << 4)) =
              make_float4(v[4 * c8], v[4 * c8 + 1], v[4 * c8 + 2], v[4 * c8 + 3]);
      }
    }
  }
  umma::fence_proxy_async();   // the staged rows, for the TMA
  umma::fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && ok && nk > 0) {
    const int D = g.L.cdim();
    for (int o = 0; o < nout; ++o) {
      const int ti = (un.kind == 2 && o == 1) ? un.a1 : un.a0;
      const int tj = un.kind == 1 ? un.b + o : un.b;
      const int y = ((int)blockIdx.y * 3 + ch) * D + ti * BM;   // row of part[slice][ch][ti BM]
      for (int c4 = 0; c4 < 4; ++c4)
        umma::tma_reduce_add_2d(&tP, stage + (4 * o + c4) * (BM * 32), tj * BN + 32 * c4, y);
    }
    umma::bulk_commit();
    umma::bulk_wait0();
  }
  if (warp == 0) umma::tmem_dealloc(tmem, 256);
}

// looked up once (a function-local static: initialised once even when several
// host threads call it first at the same time)
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000)p;
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}

// K-major operand [rows][ld] (elements), inner extent k, 128-byte x 128-row boxes
int make_map(bem_ctx* c, CUtensorMap* m, const void* base, uint64_t k, uint64_t rows,
             uint64_t ld, bool f32) {
  auto enc = encoder();
  if (!enc) return fail(c, BEM_ECUDA, "cuTensorMapEncodeTiled is not available");
  const uint64_t es = f32 ? 4 : 2;
  if (((uintptr_t)base & 15) || (ld * es) % 16)
    return fail(c, BEM_EINVAL, "tensor-core operand not 16-byte aligned");
  cuuint64_t dims[2] = {k, rows};
  cuuint64_t strides[1] = {ld * es};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es), BM};
  cuuint32_t est[2] = {1, 1};
  CUresult r = enc(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, est, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, BEM_ECUDA, "cuTensorMapEncodeTiled failed");
  return BEM_OK;
}

// tp: the Gram partial sums (EPI_SYRK); any valid map otherwise (not read)
template <int SCH>
int launch(bem_ctx* c, const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& a2,
           const CUtensorMap& b2, const CUtensorMap& tp, const TcArgs& g, dim3 grid) {
  // set once per process (a function-local static; safe when several host
  // threads launch at the same time)
  static const cudaError_t attr = cudaFuncSetAttribute(
      k_tc_gemm<SCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, Scheme<SCH>::SMEM);
  if (attr != cudaSuccess) return cuda_check(c, attr, "tc gemm smem attribute");
  k_tc_gemm<SCH><<<grid, 128, Scheme<SCH>::SMEM, S(c)>>>(a, b, a2, b2, tp, g);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "k_tc_gemm");
}

}  // namespace

// D[M][N] = A[M][K] B[N][K]^T, bf16 in, fp32 out (all device, row-major).
int tc_gemm_store(bem_ctx* c, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                  float* D, int ldd) {
  int rc;
  CUtensorMap ta, tb;
  if ((rc = make_map(c, &ta, A, K, M, lda, false)) || (rc = make_map(c, &tb, B, K, N, ldb, false)))
    return rc;
  TcArgs g{};
  g.M = M; g.N = N; g.K = K; g.mode = EPI_STORE; g.D = D; g.ldd = ldd; g.err = c->d_status;
  g.wait_ns = c->wait_ns;
  return launch<SCH_BF16>(c, ta, tb, ta, tb, ta, g, dim3((M + BM - 1) / BM, (N + BN - 1) / BN));
}

// J^T rows: J[rows][m] = Mt[rows][Nb] Phi[m][Nb]^T + F[rows][m].
//   bf16:   Mt, Phi bf16; J bf16 (Jout[0]); with gpart, also the handle part
//           of the gradient per 128-sample tile (see TcArgs)
//   3xtf32: Mt = (Mt[0] hi, Mt[1] lo), Phi likewise, fp32; J hi/lo fp32 (Jout[0], Jout[1])
int tc_jrows(bem_ctx* c, int sch, const JLayout& L, int m, int Nb, const void* const* Mt, int ldm,
             const void* const* Phi, int ldp, const float* F, int ldf, void* const* Jout, int ldj,
             const float* resid, int nc, float* gpart, int64_t gstride) {
  const int rows = L.rows();
  const bool x3 = sch != SCH_BF16, f32 = sch == SCH_TF32X3;
  int rc;
  CUtensorMap ta, tb, ta2, tb2;
  if ((rc = make_map(c, &ta, Mt[0], Nb, rows, ldm, f32)) ||
      (rc = make_map(c, &tb, Phi[0], Nb, m, ldp, f32)))
    return rc;
  if (x3 && ((rc = make_map(c, &ta2, Mt[1], Nb, rows, ldm, f32)) ||
             (rc = make_map(c, &tb2, Phi[1], Nb, m, ldp, f32))))
    return rc;
  if ((ldf % 4) || ((uintptr_t)F & 15)) return fail(c, BEM_EINVAL, "F rows not 16-byte aligned");
  TcArgs g{};
  g.M = rows; g.N = m; g.K = Nb; g.mode = EPI_JROWS; g.F = F; g.ldf = ldf; g.ldj = ldj;
  g.err = c->d_status;
  g.wait_ns = c->wait_ns;
  g.L = L;
  if (x3) { g.Jhi = Jout[0]; g.Jlo = Jout[1]; }
  else g.J = (__nv_bfloat16*)Jout[0];
  // bf16 and compensated bf16 run the persistent kernel, whose epilogue
  // forms the handle part of the gradient; 3xtf32 the per-tile kernel
  const bool pers = sch != SCH_TF32X3;
  if (pers && gpart) {
    g.resid = resid;
    g.gnc = nc;
    g.gpart = gpart;
    g.gstride = gstride;
  }
  ProfScope _ps(c, "tc_jrows");
  if (pers) {
    // the epilogue's TMA views: F^T (fp32) and J^T (bf16; hi and lo parts
    // for the compensated scheme), m columns x rows
    CUtensorMap tf, tj, tj2;
    if ((rc = make_map(c, &tf, F, m, rows, ldf, true)) ||
        (rc = make_map(c, &tj, Jout[0], m, rows, ldj, false)) ||
        (rc = make_map(c, &tj2, x3 ? Jout[1] : Jout[0], m, rows, ldj, false)))
      return rc;
    if (!x3) { ta2 = ta; tb2 = tb; }   // not read by the bf16 kernel
    auto run = [&](auto kern, int smem, int bnt) -> int {
      const int ntiles = ((rows + BM - 1) / BM) * ((m + bnt - 1) / bnt);
      const int grid = std::max(1, std::min(ntiles, c->sms));
      kern<<<grid, kPersThreads, smem, S(c)>>>(ta, tb, ta2, tb2, tf, tj, tj2, g);
      BEM_LAUNCHED(c);
      return cuda_check(c, cudaGetLastError(), "k_tc_jrows_pers");
    };
    if (x3) {
      // set once per process (a function-local static; safe when several host
      // threads launch at the same time)
      static const cudaError_t attr = cudaFuncSetAttribute(
          k_tc_jrows_pers<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, Pers<true>::SMEM);
      if (attr != cudaSuccess) return cuda_check(c, attr, "persistent J rows smem attribute");
      return run(k_tc_jrows_pers<true>, Pers<true>::SMEM, Pers<true>::BNT);
    }
    // set once per process (a function-local static; safe when several host
    // threads launch at the same time)
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_tc_jrows_pers<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, Pers<false>::SMEM);
    if (attr != cudaSuccess) return cuda_check(c, attr, "persistent J rows smem attribute");
    return run(k_tc_jrows_pers<false>, Pers<false>::SMEM, Pers<false>::BNT);
  }
  dim3 grid((rows + BM - 1) / BM, (m + BN - 1) / BN);
  return launch<SCH_TF32X3>(c, ta, tb, ta2, tb2, ta, g, grid);
}

// CTAs of one K slice of the Gram kernels: bf16 paired units, 3xtf32 single
// blocks; channel 0 over its whole channel-order triangle, channels 1 and 2
// without the jump-jump blocks
static int gram_ctas(const JLayout& L, bool x3) {
  const int T = L.tiles(), Tp = L.ptiles();
  if (x3) return T * (T + 1) / 2 + 2 * (T * Tp - Tp * (Tp - 1) / 2);
  return syrk_units(T, T) + 2 * syrk_units(T, Tp);
}

// part[split][ch][cdim][cdim] += upper blocks of J_ch^T J_ch (channel order,
// JLayout) over the m samples of J, K split into `splits` slices.
// bf16: J[0] bf16.  3xtf32: J[0] hi, J[1] lo, fp32.
int tc_syrk(bem_ctx* c, int sch, const JLayout& L, int m, const void* const* J, int ldj,
            float* part, int splits) {
  int rc;
  const bool x3 = sch != SCH_BF16, f32 = sch == SCH_TF32X3;
  CUtensorMap tj, tj2;
  if ((rc = make_map(c, &tj, J[0], m, L.rows(), ldj, f32))) return rc;
  if (x3 && (rc = make_map(c, &tj2, J[1], m, L.rows(), ldj, f32))) return rc;
  TcArgs g{};
  g.M = g.N = L.cdim(); g.K = m; g.mode = EPI_SYRK; g.nc = L.cdim(); g.L = L;
  g.tiles = L.tiles();
  g.npairs = g.tiles * (g.tiles + 1) / 2;
  const int bk = f32 ? Scheme<SCH_TF32X3>::BK : Scheme<SCH_BF16>::BK;
  g.k_per_split = ((m + splits - 1) / splits + bk - 1) / bk * bk;
  g.part = part; g.err = c->d_status;
  g.wait_ns = c->wait_ns;
  int sp = (m + g.k_per_split - 1) / g.k_per_split;
  ProfScope _ps(c, "tc_syrk");
  if (!x3) {
    // set once per process (a function-local static; safe when several host
    // threads launch at the same time)
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_tc_syrk_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, kSySmem);
    if (attr != cudaSuccess) return cuda_check(c, attr, "paired Gram smem attribute");
    g.npairs = syrk_units(g.tiles, g.tiles);
    // the partial sums as one fp32 matrix of splits x 3 x cdim rows, for the
    // epilogue's TMA reductions
    CUtensorMap tp;
    if ((rc = make_map(c, &tp, part, L.cdim(), (uint64_t)splits * 3 * L.cdim(), L.cdim(), true)))
      return rc;
    k_tc_syrk_pair<<<dim3(gram_ctas(L, false), sp), 128, kSySmem, S(c)>>>(tj, tp, g);
    BEM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "k_tc_syrk_pair");
  }
  dim3 grid(gram_ctas(L, true), sp);
  CUtensorMap tp;
  if ((rc = make_map(c, &tp, part, L.cdim(), (uint64_t)splits * 3 * L.cdim(), L.cdim(), true)))
    return rc;
  if (f32) return launch<SCH_TF32X3>(c, tj, tj, tj2, tj2, tp, g, grid);
  return launch<SCH_BF16X3>(c, tj, tj, tj2, tj2, tp, g, grid);
}

// K slices per block pair: as many as fill the resident CTA slots in one
// wave without starting a second, nearly empty one (rounding up would leave
// a short tail wave that costs as long as the first)
// out = {kind, a0, a1, b} of Gram unit u of a T x T block triangle
int tc_gram_unit(int T, int R, int u, int* out) {
  if (T < 1 || R < 1 || R > T || u < 0 || u >= syrk_units(T, R)) return BEM_EINVAL;
  const SyrkUnit un = syrk_unit(T, R, u);
  out[0] = un.kind;
  out[1] = un.a0;
  out[2] = un.a1;
  out[3] = un.b;
  return BEM_OK;
}

int tc_syrk_splits(const JLayout& L, bool x3, int sms) {
  // bf16: one CTA per SM on paired blocks; 3xtf32: one CTA per SM per block
  const int ctas = gram_ctas(L, x3);
  const int slots = std::max(1, sms);
  // the fewest slices whose CTAs fill their waves to 95 %, else the best fill up to 8 slices
  // (204 units at n_c = 2,048: one slice leaves the second wave a third full, three fill four)
  int best = 1;
  double best_fill = 0.0;
  for (int sp = 1; sp <= 64; ++sp) {
    const int n = ctas * sp;
    const double fill = double(n) / (double((n + slots - 1) / slots) * slots);
    if (fill >= 0.95) return sp;
    if (sp <= 8 && fill > best_fill) { best_fill = fill; best = sp; }
  }
  return best;
}

}  // namespace bem
