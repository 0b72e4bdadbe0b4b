// Internal state of a bem_ctx and the host-side launchers of every kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "bemgb.h"
#include "common.cuh"
#include "field_args.cuh"

namespace bem {

// Device buffer that grows on demand (never shrinks until the context dies).
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct Scene {
  int C = 0;          // curves
  int P = 0;          // panels
  int nth = 0;        // parameters, 32 C
  int nc = 0;         // parameters per colour channel: pp NH + 2 NH
  // colour owners: the 4 control handles of each Bezier curve (pp = 2
  // position parameters each, 8 parameters) or the paper's segment handles
  // (pp = 4: endpoints a and b, 10 parameters, one panel each)
  int pp = 2;
  int NH = 0;
  std::vector<int> K, off;        // panels per curve, panel offset of each curve
  std::vector<uint8_t> closed;
  // device metadata
  int* d_pcurve = nullptr;   // [P] curve of each panel
  int* d_pk = nullptr;       // [P] index within its curve
  int* d_off = nullptr;      // [C+1] panel offsets
  int* d_K = nullptr;        // [C]
  uint8_t* d_closed = nullptr;  // [C]
};

struct Boundary {
  int M = 0;      // segments per side (per polygon edge)
  int Nb = 0;     // M times the number of edges
  std::vector<double> poly;    // counter-clockwise polygon [V][2]; empty = the unit square
  double* d_vert = nullptr;    // [(Nb+1)][2] CCW vertices, vert[Nb] = vert[0]
  float* d_vert32 = nullptr;
  double* d_gp = nullptr;      // [3 Nb][2] Gauss points
  float* d_gp32 = nullptr;
  double* d_A = nullptr;       // [Nb][Nb] Galerkin matrix
  double* d_W = nullptr;       // [Nb][Nb] pseudo-inverse A^+
  double* d_WT = nullptr;      // [Nb][Nb] (A^+)^T
  float* d_W32 = nullptr;      // float copy of A^+ (mixed solves)
  float* d_WT32 = nullptr;
  bool factored = false;
};

}  // namespace bem

struct bem_ctx {
  int device = 0;
  bem_opts opts{};
  std::string err;
  cudaStream_t cur = nullptr;
  int64_t launches = 0;
  int64_t allocs = 0;              // device allocations made by the context (cudaMalloc calls)
  int sms = 0;                     // multiprocessors of the device
  // limit of the tensor-core kernels' pipeline waits (bem_set_wait_limit)
  uint64_t wait_ns = 1000000000ull;

  bem::Scene sc;
  bem::Boundary bd;
  double mean[3] = {0, 0, 0};
  bool have_scene = false;

  // parameters and panels
  double* d_theta = nullptr;       // [nth]
  double* d_trial = nullptr;       // [nth] trial parameters of the LM step
  double* d_delta = nullptr;       // [nth]
  bem::Panel<double>* d_pan64 = nullptr;   // [P]
  bem::Panel<float>* d_pan32 = nullptr;    // [P]
  double* d_compat = nullptr;      // [NH] compatibility weights a_h of the colour owners
  double* d_ub = nullptr;          // [Nb][3] boundary solution of the current panels
  double* d_fb = nullptr;          // [Nb][3] right-hand side
  double* d_q = nullptr;           // [Nb][3] adjoint boundary source
  double* d_lb = nullptr;          // [Nb][3] adjoint boundary solution
  double* d_scal = nullptr;        // small device scalars (loss, sums)
  int* d_status = nullptr;         // device error word (0 = fine)

  // per-kernel event timing (bem_profile_enable)
  bool prof = false;
  struct ProfRec { std::string name; cudaEvent_t a, b; };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  std::map<std::string, std::pair<double, int64_t>> prof_tot;

  // growable scratch
  bem::DevBuf part, part2, loss, gpart, jrow, phi, Hc, Mc, Dfc, Fg, lmK, lmL, lmLt, lmW, H, g,
      tcJ, tcPart, tcMt, nearP, nearS, nearF, gwork, rend, regw;
  bem_reg reg{};                   // Sec. 4.4 regularisers (segment handles)
  bool pbins_valid = false;        // panel -> cell bins match the current panels
  bool dmath_ready = false;        // the tables of the double logarithm and arctangent are on this device
  // When set, the Gauss-Newton chunk buffers (jrow, tcJ, tcPart, gwork) are
  // taken from this context: a batch of scenes processed one after another
  // on one stream shares them.
  bem_ctx* scratch = nullptr;
  // Host inputs of lm_step_host: their device copies, the copy stream, and
  // the events that mark the samples (all of them) and each Gauss-Newton
  // chunk's targets as arrived.  While hin_on is set, the Gauss-Newton pass
  // waits on those events before it first reads the samples and before each
  // chunk reads its targets.
  bem::DevBuf hin_xy, hin_t;
  cudaStream_t hin_stream = nullptr;
  cudaEvent_t hin_start = nullptr, hin_xy_ready = nullptr;
  std::vector<cudaEvent_t> hin_t_ready;
  bool hin_on = false;
};

namespace bem {

// Row layout of the J^T rows of the tensor-core Gauss-Newton pass.  Colour
// channel c's J_c has the position columns of every colour owner (pp per
// owner) and the two jump columns w_d,c and w_c,c of each owner.  The jump
// columns do not depend on the channel (the colour is linear in the jumps
// with the same layer values in every channel, and so are their boundary
// parts), so the rows hold them once:
//   rows [c Pp, c Pp + npos)     position columns of channel c (c = 0, 1, 2)
//   rows [3 Pp, 3 Pp + 2 NH)     jump columns: w_d of owner h at 3 Pp + h,
//                                w_c of owner h at 3 Pp + NH + h
// with npos = pp NH, Pp = npos and Pw = 2 NH rounded up to 128 rows (the
// padding rows are zero).  Channel c's rows, in "channel order", are its
// position range followed by the jump range: channel index i < Pp is
// position column i, i >= Pp is jump column i - Pp, which is column
// npos + i - Pp of the per-channel column order (w_d at npos + h, w_c at
// npos + NH + h).  The Gram blocks of the jump range with itself are the
// same for every channel and are formed once, for channel 0.
struct JLayout {
  int npos = 0, nh = 0, Pp = 0, Pw = 0;
  __host__ __device__ int rows() const { return 3 * Pp + Pw; }
  __host__ __device__ int cdim() const { return Pp + Pw; }
  __host__ __device__ int tiles() const { return (Pp + Pw) / 128; }    // channel-order 128-row tiles
  __host__ __device__ int ptiles() const { return Pp / 128; }          // of them in the position range
  // J^T row of the first row of channel-order tile t of channel ch
  __host__ __device__ int tile_row(int ch, int t) const {
    return 128 * t < Pp ? ch * Pp + 128 * t : 3 * Pp + (128 * t - Pp);
  }
};

inline JLayout jlayout(int pp, int NH) {
  JLayout L;
  L.npos = pp * NH;
  L.nh = NH;
  L.Pp = (L.npos + 127) / 128 * 128;
  L.Pw = (2 * NH + 127) / 128 * 128;
  return L;
}

// ---- error plumbing (api.cu) ------------------------------------------------
int fail(bem_ctx* c, int code, const std::string& msg);
int cuda_check(bem_ctx* c, cudaError_t e, const char* what);
int grow(bem_ctx* c, DevBuf& b, size_t bytes);
inline cudaStream_t S(bem_ctx* c) { return c->cur; }

// Samples per chunk of the tensor-core Gauss-Newton pass over n samples
inline int64_t gn_chunk_tc(const bem_ctx* c, int64_t n) {
  const int64_t ch = c->opts.gn_chunk > 0 ? c->opts.gn_chunk : 262144;
  return n < 1 ? 1 : (n < ch ? n : ch);
}

// ---- context helpers (api.cu) --------------------------------------------------
int ctx_set_device(bem_ctx* c);
int ctx_ready(bem_ctx* c);                              // set up and factored
int ctx_refresh(bem_ctx* c, const double* theta);       // panels, RHS, boundary solution
void ctx_axpy(bem_ctx* c, const double* a, const double* b, int n, double* out);
void ctx_scale_norm(bem_ctx* c, double* v, int n, double s, double* norm2);

// ---- geometry (k_geom.cu) -----------------------------------------------------
int geom_panelize(bem_ctx* c, const double* d_theta);
// compatibility weights a_h of the current panels into d_compat; with
// project, w_c of theta is instead projected onto the compatibility
// hyperplane of the current panels in place, and d_compat is left as it is
int geom_compat(bem_ctx* c, double* d_theta, bool project);
int geom_boundary_tables(bem_ctx* c);                  // vertices, Gauss points
int geom_assemble(bem_ctx* c);                         // d_A

// ---- regularisers and pruning of segment handles (k_reg.cu) ------------------
bool reg_active(const bem_ctx* c);
int reg_pairs(bem_ctx* c, const double* theta);                 // snapping pairs at theta
int reg_add(bem_ctx* c, const double* theta, double* H, double* g);
int reg_loss(bem_ctx* c, const double* theta, double* d_out);  // with the chosen pairs
int reg_prune(bem_ctx* c, double thr, std::vector<double>& kept_theta, std::vector<int>& kept_idx);

// ---- float Cholesky and cluster triangular solve for large LM systems (k_chol.cu)
// factor of the equilibrated matrix Kf (lower triangle, updated in place) into
// Lf, diagonal-block inverses into Linv64 [ceil(n/64)][64][64]
void chol_blocked_f32(bem_ctx* c, float* Kf, float* Lf, int n, float* Linv64, int* status,
                      float* bad_pivot);
int trsv_cluster_prepare(bem_ctx* c, int n);     // shared-memory size attribute
// X += D z with (D K D) z = D Rres solved with the factor (four right-hand sides)
void trsv_cluster_f32(bem_ctx* c, const float* Lf, const float* Linv64, int n, const double* d,
                      const double* Rres, double* X);

// ---- linear algebra (k_linalg.cu) -------------------------------------------
int la_pinv(bem_ctx* c);   // factor bordered system, W = A^+ (double, float copies)
// y[Nb][3] = W x[Nb][3] (transpose: W^T)
int la_apply3(bem_ctx* c, const double* W, const double* x, double* y);
// refined float solve: y = A^+ x via float W and a double residual
int la_apply3_refined(bem_ctx* c, const float* W32, const double* A, const double* x, double* y,
                      bool transpose);
int la_apply3_refined_buf(bem_ctx* c, const float* W32, const double* A, const double* x,
                          double* y, bool transpose, double* scratch);
void la_dgemm(bem_ctx* c, bool ta, bool tb, int M, int N, int K, double alpha, const double* A,
              int lda, const double* B, int ldb, double beta, double* C, int ldc);
// LM solve: delta for (H + lam D) delta = -g with the compatibility KKT;
// returns BEM_ENOTSPD if the Cholesky fails
int la_lm_solve(bem_ctx* c, const double* H, const double* g, double lam, double* delta);

// ---- forward field (k_field.cu) --------------------------------------------------
// u at n points into out (sample type), optional residual/loss; loss sum -> d_scal[0]
// residual and loss partials of m points whose handle term (with its near-field
// correction) is given in hand [m][3]: the boundary term, the mean colour and
// the clamp are added here.  loss_part receives field_blocks(m) block sums.
int field_finish_hand(bem_ctx* c, int64_t m, const float* xy, const double* hand,
                      const float* target, float* resid, double* loss_part);
int64_t field_blocks(int64_t m);
int field_sum_loss(bem_ctx* c, const double* loss_part, int64_t nblk);   // -> d_scal[0]
int field_eval(bem_ctx* c, int64_t n, const void* xy, void* out, const void* target,
               void* resid, bool want_loss);
int field_rhs(bem_ctx* c);           // d_fb from the current panels
int field_solve(bem_ctx* c);         // d_ub = A^+ d_fb
int field_sample_mean(bem_ctx* c, int64_t n, const void* target, double* host_mean);
// base float arguments of a mixed context (panels, boundary, eps, near field)
FieldArgs<float> field_args_f32(bem_ctx* c);
// one persistent launch over the tiles of all jobs (128 * spt points per
// tile, blocks_per_sm CTAs per SM); total_tiles and counter: device words
// (the counter is reset here), so that a captured graph can be replayed
// with new job contents
// nt > 1: every job evaluates its nt trials (BatchJob.tpan ..), sharing the
// boundary angles of its points
int field_batch_launch(bem_ctx* c, const BatchJob* jobs, int njobs, const int64_t* total_tiles,
                       unsigned long long* counter, int spt, int blocks_per_sm, int nt = 1);

// ---- near field of the mixed path (k_near.cu) ------------------------------------
// out[n][3] = double sum over the near panels of each point
int near_forward(bem_ctx* c, int64_t n, const float* xy, double* out);
// per point, sum over its near pairs of (double value - the F rows' float value)
int near_forward_minus_float(bem_ctx* c, int64_t n, const float* xy, double* out);
// out[P][11] = double adjoint sums of each panel over its near points
int near_adjoint(bem_ctx* c, int64_t n, const float* xy, const float* w, double* out);

// ---- adjoint (k_adjoint.cu) ------------------------------------------------------
int adj_vjp(bem_ctx* c, int64_t n, const void* xy, const void* resid, double* grad);

// ---- Gauss-Newton matrix (k_jtj.cu) ----------------------------------------------
// H = (1/n) J^T J; with resid (sample type [n][3]) and g also g = (1/n) J^T r
// when jtj_gives_gradient() (tensor-core modes of the mixed path)
// With target (tensor-core modes only), the residual at the current theta is
// formed inside the pass instead of read: resid is written, the loss sum
// sum |r|^2 lands in d_scal[0] (the handle term as F w, see jtj_tc).
int jtj_build(bem_ctx* c, int64_t n, const void* xy, double* H, const void* resid = nullptr,
              double* g = nullptr, const void* target = nullptr);
bool jtj_gives_gradient(const bem_ctx* c);
bool jtj_fuses_eval(const bem_ctx* c);   // jtj_build accepts a target

// ---- tensor-core contractions (k_gemm_tc.cu) ----------------------------------------
// Operand schemes of the J^T J contraction: one bf16 product, or each value
// split into a high and a low part (x = hi + lo) with the three products
// hi.hi + hi.lo + lo.hi accumulated in fp32, the parts tf32 (stored as fp32)
// or bf16.
enum { SCH_BF16 = 0, SCH_TF32X3 = 1, SCH_BF16X3 = 2 };
int tc_gemm_store(bem_ctx* c, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                  float* D, int ldd);
int tc_jrows(bem_ctx* c, int sch, const JLayout& L, int m, int Nb, const void* const* Mt, int ldm,
             const void* const* Phi, int ldp, const float* F, int ldf, void* const* Jout, int ldj,
             const float* resid = nullptr, int nc = 0, float* gpart = nullptr,
             int64_t gstride = 0);
int tc_syrk(bem_ctx* c, int sch, const JLayout& L, int m, const void* const* J, int ldj,
            float* part, int splits);
int tc_syrk_splits(const JLayout& L, bool x3, int sms);
// {kind, a0, a1, b} of the bf16 Gram kernel's unit u over the block rows
// 0 .. R-1 of T; BEM_EINVAL when T < 1, R outside [1, T] or u is not a unit
int tc_gram_unit(int T, int R, int u, int* out);

// Brackets the kernel launches of its lifetime with events when profiling.
struct ProfScope {
  bem_ctx* c;
  int idx = -1;
  ProfScope(bem_ctx* ctx, const char* name);
  ~ProfScope();
};

}  // namespace bem

#define BEM_LAUNCHED(c) ((c)->launches++)
