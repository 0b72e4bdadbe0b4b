/*
 * bemgb.h -- C ABI of the GB300 differential-BEM library.
 *
 * Per-iteration hot path of the Levenberg-Marquardt fit of diffusion-curve
 * handles to noisy Monte Carlo colour samples ("Monte Carlo Rendering to
 * Diffusion Curves with Differential BEM"):
 *   - evaluate the boundary-integral colour at every sample     (Sec. 3.1, Eq. (bie))
 *   - its adjoint with respect to handle positions and jumps   (Sec. 3.2, Eq. (diffbie))
 *   - the Gauss-Newton products J^T J, J^T r and the LM step   (Sec. 4.3, Eq. (optimstep))
 * against the dense BEM matrix of the image boundary, factored once (Sec. 3.1.3).
 *
 * Conventions shared by every entry point
 *   - Every call returns a bem_status (0 = BEM_OK); nothing aborts.  On
 *     failure bem_last_error() holds a one-line reason.
 *   - Pointers marked "device" are CUDA device pointers on the context's
 *     device; "host" pointers are ordinary host memory.  The caller owns
 *     every buffer it passes; the context owns all of its internal device
 *     buffers (panels, factors, Gram matrices, partial sums) and frees them
 *     in bem_destroy().
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Work is enqueued on it in order; entry points that return
 *     host-visible results (lm_step, bem_loss) synchronise that stream.
 *   - Per-sample arrays (xy, target, rgb, resid) are row-major
 *     [n][2] / [n][3] in the context's sample type: double for
 *     BEM_FP64 contexts, float for BEM_MIXED contexts.
 *   - Parameter vectors theta are double [n_theta], n_theta = 32 * n_curves,
 *     laid out [curve][control handle 0..3][x, y, wd_r, wd_g, wd_b, wc_r, wc_g, wc_b].
 *     wd is the colour jump (left side minus right side of the curve's
 *     direction of travel) and wc the jump of the normal derivative
 *     (Eq. (handleterm)).  A closed curve reuses control point 0 as its
 *     last point; the last point's x, y are then not free (their gradient is 0).
 *   - The image domain is the unit square; its boundary carries the zero
 *     Neumann condition of Eq. (neumann).
 */
#ifndef BEMGB_H
#define BEMGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BEM_OK = 0,
    BEM_EINVAL = -1,      /* bad argument (size, pointer, option) */
    BEM_ESTATE = -2,      /* call out of order, e.g. eval before factor */
    BEM_ESINGULAR = -3,   /* boundary matrix factorisation failed */
    BEM_ENOTSPD = -4,     /* LM matrix not positive definite at every trial lambda */
    BEM_ECUDA = -5,       /* a CUDA runtime call failed (message in bem_last_error) */
    BEM_ETIMEDOUT = -6,   /* a bounded device-side wait ran out */
    BEM_ENOMEM = -7       /* device allocation failed */
} bem_status;

enum { BEM_FP64 = 0, BEM_MIXED = 1 };                         /* bem_opts.precision */
/* bem_opts.jtj_mode, the arithmetic of H = J^T J in BEM_MIXED contexts:
 *   FP64     double products of the float J rows (SIMT)
 *   BF16     J rows rounded to bf16, one tensor-core product, fp32 accumulation
 *   3XTF32   every operand split into two tf32 parts (x = hi + lo), the three
 *            products hi.hi + hi.lo + lo.hi accumulated in fp32
 *   BF16X3   the same split with two bf16 parts (compensated bf16: about 16
 *            mantissa bits per operand, at half the operand bytes and twice
 *            the product rate of 3XTF32)
 * In every tensor-core mode the fp32 sums of slices of samples are added in
 * double. */
enum { BEM_JTJ_FP64 = 0, BEM_JTJ_BF16 = 1, BEM_JTJ_3XTF32 = 2, BEM_JTJ_BF16X3 = 3 };
/* bem_opts.lm_solver: how the damped KKT system of lm_step is solved.
 * AUTO: Cholesky of the equilibrated matrix in float, iterative refinement
 * against the double residual until the normwise backward error is below
 * 1e-14, double Cholesky if the float factor fails or the refinement stalls.
 * FP64: double Cholesky only. */
enum { BEM_LM_AUTO = 0, BEM_LM_FP64 = 1 };

typedef struct {
    int precision;        /* BEM_FP64: every step in double.  BEM_MIXED: float
                             sample/panel arithmetic, double near field and
                             refined double boundary solves */
    double eps_d;         /* regularisation of the w_d (double-layer) handle
                             term, Sec. 3.1.3 / 3.2.1; default 1e-2 */
    double eps_c;         /* regularisation of the w_c (single-layer) term; default 1e-2 */
    int segs_per_side;    /* boundary segments per side of the square, Sec. 3.1.3; default 256 */
    double near_factor;   /* BEM_MIXED: pairs closer than near_factor panel
                             lengths are evaluated in double; default 0.5; 0 = never */
    int jtj_mode;         /* arithmetic of the J^T J contraction (BEM_JTJ_*) */
    int lm_solver;        /* BEM_LM_AUTO (default) or BEM_LM_FP64 */
    int galerkin_mode;    /* boundary matrix, Sec. 3.1.3: 0 (default) inner integral of
                             each entry exact, outer by 3-point Gauss; 1 both by 3-point
                             Gauss (the paper's rule).  Mode 1 leaves the constants only
                             nearly in the null space; its pseudo-inverse drops the
                             smallest singular value exactly, as in mode 0 */
    int gn_chunk;         /* samples per chunk of the Gauss-Newton pass (Eq. (losshessian),
                             (lossjacobian)): J rows exist for one chunk at a time and the
                             chunks' sums are added in double.  0 (default): 262,144 in the
                             tensor-core J^T J modes, 32,768 otherwise; else a multiple of
                             128 in [128, 4,194,304].  The result does not depend on it
                             beyond the order of the chunk sums */
    int reserved[5];
} bem_opts;

typedef struct {
    double loss_before;   /* L(theta) = (1/2n) sum |u - min(t,1)|^2 at the current theta */
    double loss_after;    /* L at the best trial theta' (same samples, Sec. 4.3) */
    int accepted;         /* 1 if loss_after < loss_before (theta updated) */
    int best_trial;       /* index into lambdas of the trial that was taken (or -1) */
    double lambda_next;   /* damping proposal for the next step */
    double grad_norm;     /* |g|_2 of the gradient at theta */
} lm_result;

/* Regularisers of segment handles (Sec. 4.4); a zero weight turns a term
 * off, all off by default.  Each adds its loss to the LM objective and its
 * analytic gradient and Hessian to g and H of Eq. (optimstep):
 *   length    len_weight (|b - a| - len_max)^2 where |b - a| > len_max
 *   snapping  snap_weight |p - q|^2 for endpoints p, q of two handles closer
 *             than snap_radius that choose each other by the lowest score
 *             snap_alpha |p - q| / snap_radius + (1 - snap_alpha)(1 - |u_p.u_q|)
 *             (u = unit handle directions; ties to the lower endpoint index
 *             2h + s, s = 0 for a, 1 for b); pairs chosen once per LM step
 *   sparsity  lam t tanh(sqrt(w.w + eps^2) / t) per handle for w = w_d
 *             (lam = sparse_wd) and w = w_c (lam = sparse_wc), t = sparse_t,
 *             eps = sparse_eps; H receives its Hessian with the factor
 *             sech^2(rho/t) held fixed (positive semidefinite), without the
 *             negative curvature of the saturation. */
typedef struct {
    double len_weight, len_max;
    double snap_weight, snap_radius, snap_alpha;
    double sparse_wd, sparse_wc, sparse_eps, sparse_t;
} bem_reg;

typedef struct bem_ctx bem_ctx;

/* Fill *opts with the defaults above.  Never fails for a non-NULL opts. */
int bem_default_opts(bem_opts *opts);

/* Create a context on CUDA device `device`.  *out receives the handle (NULL
 * on failure).  opts may be NULL for the defaults.  Errors: BEM_EINVAL for
 * bad options, BEM_ECUDA if the device cannot be used. */
int bem_create(bem_ctx **out, const bem_opts *opts, int device);

/* Release every device buffer of the context.  ctx may be NULL. */
void bem_destroy(bem_ctx *ctx);

/* Last error message of this context (or of the last failed bem_create if
 * ctx is NULL); never NULL. */
const char *bem_last_error(const bem_ctx *ctx);

/* Describe the handle set (Sec. 4.1: handles with endpoints and constant
 * jumps; here cubic Bezier curves cut into straight panels, Sec. 6).
 *   n_curves >= 1; panels_per_curve[n_curves] >= 1 (host int32);
 *   closed[n_curves] (host uint8, 1 = loop);
 *   theta[32*n_curves] host double initial parameters;
 *   mean_color[3] host double: the per-domain constant colour added to the
 *   zero-mean BEM solution (Sec. 3.1.3, 4.3).
 * Allocates the per-scene buffers.  May be called again to replace the scene. */
int bem_setup(bem_ctx *ctx, int n_curves, const int32_t *panels_per_curve,
              const uint8_t *closed, const double *theta, const double *mean_color);

/* The paper's handle parametrisation (Sec. 4.2): n_handles independent
 * straight handles, each one panel, with 10 parameters
 *   theta[10 h ..] = (a_x, a_y, b_x, b_y, w_d RGB, w_c RGB)
 * (the jumps constant over the handle).  Every other call works as for
 * Bezier curves; n_theta = 10 n_handles, the compatibility condition uses
 * the handle lengths.  theta: host double [10 n_handles]; mean_color: host
 * double[3].  Errors: BEM_EINVAL. */
int bem_setup_segments(bem_ctx *ctx, int n_handles, const double *theta,
                       const double *mean_color);

/* Set (reg non-NULL) or clear (reg NULL) the Sec. 4.4 regularisers of a
 * segment-handle context; lm_step and lm_step_split then report the losses
 * with the regulariser values included.  Errors: BEM_EINVAL for negative or
 * non-finite weights, snap_radius <= 0, snap_alpha outside [0, 1],
 * sparse_eps or sparse_t <= 0 while their term is on, BEM_ESTATE unless the
 * scene was set up with bem_setup_segments. */
int bem_set_regularizers(bem_ctx *ctx, const bem_reg *reg);

/* Pruning (Sec. 4.4, Sparsity): remove every handle with |w_d| < threshold
 * and |w_c| < threshold (2-norms over RGB), keep the others in order, and
 * re-project w_c onto the compatibility hyperplane of the kept handles
 * (Sec. 4.3).  *n_kept receives their number and kept_index (host int32
 * [old n_handles], may be NULL) their former indices.  If no handle would
 * remain the scene is left as it is and *n_kept = 0.  The boundary
 * factorisation stays valid.  Synchronises `stream`.  Errors: BEM_EINVAL,
 * BEM_ESTATE unless the scene has segment handles and is factored. */
int bem_prune(bem_ctx *ctx, double threshold, int *n_kept, int32_t *kept_index, void *stream);

/* Initial segment handles (Sec. 4.2), host only (no context, no GPU): for
 * the sequence indices k = first_index .. first_index + n_points - 1, the
 * first endpoint a is point k of the two-dimensional Sobol sequence (Gray-
 * code order, unscrambled); handles are made only where a lies inside the
 * polygon (even-odd rule; vertices NULL = the unit square).  The second
 * endpoint is a + length (cos phi, sin phi) with phi = 2 pi times the base-3
 * radical inverse of k (a stand-in for a third Sobol coordinate), pulled
 * back along the handle to its first crossing with the polygon.  Jumps are
 * zero.  theta_out: host double [10 n_points] (the first 10 *n_handles
 * entries are written); vertices: host double [n_vertices][2].
 * Errors: BEM_EINVAL. */
int bem_init_segments(int n_points, double length, int64_t first_index, int n_vertices,
                      const double *vertices, double *theta_out, int *n_handles);

/* Replace the image boundary by a closed polygon, one subdomain of the
 * domain decomposition (Sec. 4.2): n_vertices >= 3 vertices, counter-
 * clockwise, inside the unit square; each edge is cut into segs_per_edge
 * equal segments (at most 8192 in all).  Invalidates the factorisation: call
 * bem_factor next.  Samples of this context must lie inside the polygon; a
 * multi-domain image is one context per subdomain (stepped together with
 * bem_batch_lm), each with its own mean colour.
 *   vertices: host double [n_vertices][2].  Errors: BEM_EINVAL. */
int bem_set_boundary(bem_ctx *ctx, int n_vertices, const double *vertices, int segs_per_edge);

/* Assemble the Galerkin matrix of the image boundary (Eq. (bie_galerkin),
 * 3-point Gauss outer rule, exact inner integral, zero coincident term) and
 * factor it once in double (Sec. 3.1.3): LU with partial pivoting of the
 * system bordered by the constant null vector, left null vector from the
 * transposed solve, then the pseudo-inverse that discards the null space.
 * Independent of theta (Sec. 3.1.3 last paragraph).  Synchronises `stream`.
 * Errors: BEM_ESINGULAR if a pivot vanishes. */
int bem_factor(bem_ctx *ctx, void *stream);

/* Replace theta (double [n_theta]); `theta_is_device` selects a device or
 * host pointer.  Stream-ordered. */
int bem_set_params(bem_ctx *ctx, const double *theta, int theta_is_device, void *stream);

/* Copy the current theta to host memory theta_out[n_theta] (synchronises). */
int bem_get_params(bem_ctx *ctx, double *theta_out, void *stream);

/* Set the per-domain mean colour (host double[3]). */
int bem_set_mean_color(bem_ctx *ctx, const double *mean_color);

/* Mean over n samples of min(target, 1) per channel (Sec. 4.3, last
 * paragraph) into host double[3].  target: device [n][3] sample type. */
int bem_sample_mean(bem_ctx *ctx, int64_t n, const void *target, double *mean_out, void *stream);

/* The image of the current theta on a width x height pixel grid: the colour
 * of Eq. (bie) at every pixel centre ((i + 1/2)/width, (j + 1/2)/height),
 * row-major with row j = y index; no rasterisation of the curves.
 *   rgb_out: device [height][width][3] (sample type).  Errors: BEM_EINVAL. */
int bem_render(bem_ctx *ctx, int width, int height, void *rgb_out, void *stream);

/* Two-sided colours of every panel (Sec. 3.1.3, recovering double-sided
 * colours): the colour u at the panel midpoint is the average c_avg across
 * the handle, and the two sides are c_avg +- w_d/2.
 *   out: host double [n_panels][2][3]: [p][0] = c_avg + w_d/2, the side to
 *   the left of a -> b (the one the right normal points away from);
 *   [p][1] = c_avg - w_d/2.  Synchronises `stream`. */
int bem_handle_colors(bem_ctx *ctx, double *out, void *stream);

/* Colours u(x) = mean + sum_j phi_j(x)/(2 pi) u_b,j + f(x; theta) at n
 * interior sample points (Eq. (bie) with alpha = 1, Sec. 3.1.3 last
 * paragraph; f from Eq. (handleterm) regularised as in Sec. 3.1.3).
 *   xy: device [n][2], rgb_out: device [n][3] (sample type).  n >= 0. */
int bem_eval(bem_ctx *ctx, int64_t n, const void *xy, void *rgb_out, void *stream);

/* Loss (1/2n) sum |u - min(t,1)|^2 (Eq. (squaredl2loss) as a Monte Carlo
 * mean with uniform density, clamp of Sec. 4.3) into host *loss_out; if
 * resid_out is not NULL it receives r = u - min(t,1), device [n][3].
 * Synchronises `stream`. */
int bem_loss(bem_ctx *ctx, int64_t n, const void *xy, const void *target,
             void *resid_out, double *loss_out, void *stream);

/* Vector-Jacobian product grad_out = J^T resid = sum_s sum_c resid[s][c]
 * du_c(x_s)/dtheta (no 1/n), computed in reverse mode through the handle
 * term and the boundary solve (Sec. 3.2, Eq. (diffbie)); kernel values are
 * recomputed, no n x P matrix is stored.
 *   xy: device [n][2]; resid: device [n][3] (sample type);
 *   grad_out: device double [n_theta]. */
int bem_vjp(bem_ctx *ctx, int64_t n, const void *xy, const void *resid,
            double *grad_out, void *stream);

/* Gauss-Newton matrix H = (1/n) sum_s J_s^T J_s (Eq. (losshessian), uniform
 * density, same samples as the gradient) into device double
 * H_out[n_theta][n_theta] (row-major, full symmetric).  The boundary part
 * of J uses the stacked right-hand sides of Sec. 3.2.3.  Arithmetic per
 * bem_opts.jtj_mode.  H_out may be NULL to only refresh the context's copy. */
int bem_jtj(bem_ctx *ctx, int64_t n, const void *xy, double *H_out, void *stream);

/* One Levenberg-Marquardt iteration (Eq. (optimstep)) on the n samples:
 * loss and gradient at theta, H (bem_jtj), then for each of the n_trials
 * damping values lambdas[] (host double): solve
 *   (H + lambda D) delta = -g,  D = diag(H) (floored at 1e-12 max),
 * restricted to steps that keep the compatibility condition with endpoints
 * fixed (Sec. 4.3), re-project w_c with the new lengths, and evaluate the
 * loss on the same samples.  H is positive semi-definite only up to
 * rounding: if H + lambda D does not factor, that trial's lambda is raised
 * tenfold until it does (at most 12 times).  The trial with the lowest loss
 * is taken if it lowers the loss (theta updated in the context).
 * lambda_next: the (raised) lambda / 3 after an accepted trial; after a
 * rejected single trial 2 lambda, after several rejected trials 10 times the
 * largest.
 *   xy, target: device (sample type); out: host.  Synchronises `stream`.
 * Errors: BEM_ENOTSPD if no trial matrix could be factored. */
int lm_step(bem_ctx *ctx, int64_t n, const void *xy, const void *target,
            int n_trials, const double *lambdas, lm_result *out, void *stream);

/* lm_step with a separate Hessian sample set (Sec. 4.3, Monte Carlo
 * integration: Eq. (losshessian) with M_H points, Eq. (lossjacobian) and the
 * trial losses with M_J points): H = (1/n_h) sum over xy_h of J^T J; g and
 * the losses from the n points (xy, target), g by the adjoint.  Passing
 * fewer Hessian points cuts the cost of J^T J.
 *   xy_h: device [n_h][2] (sample type), n_h > 0.  Otherwise as lm_step. */
int lm_step_split(bem_ctx *ctx, int64_t n, const void *xy, const void *target, int64_t n_h,
                  const void *xy_h, int n_trials, const double *lambdas, lm_result *out,
                  void *stream);

/* lm_step on samples and targets in host memory (Eq. (optimstep), as
 * lm_step): the call copies them into device buffers that the context owns
 * (kept for the next call), on a copy stream of its own, the samples first
 * and then the targets in the chunks of the Gauss-Newton pass, and the pass
 * starts on each chunk as soon as its targets have arrived, so that the
 * copies overlap the step's work.  Page-locked host memory lets the copies
 * run alongside; pageable memory gives the same results with the copies
 * taken before the step.
 *   xy: host [n][2], target: host [n][3] (sample type: float in BEM_MIXED,
 *   double in BEM_FP64); out: host.  The host buffers may be reused once the
 *   call returns.  Synchronises `stream`.  Errors: as lm_step. */
int lm_step_host(bem_ctx *ctx, int64_t n, const void *xy, const void *target, int n_trials,
                 const double *lambdas, lm_result *out, void *stream);

/* D[M][N] = A[M][K] B[N][K]^T on the tensor cores (tcgen05, fp32
 * accumulate): the contraction behind bem_jtj in BEM_MIXED contexts with
 * BEM_JTJ_BF16, exposed for validation.  A, B: device bf16, row-major, row
 * strides lda, ldb in elements (multiples of 8, 16-byte aligned bases);
 * D: device fp32 row-major, stride ldd.  M, N, K >= 1.  Errors: BEM_EINVAL
 * for bad sizes or alignment, BEM_ETIMEDOUT if a bounded device wait ran
 * out (synchronises `stream`). */
int bem_gemm_bf16(bem_ctx *ctx, int M, int N, int K, const void *A, int lda, const void *B,
                  int ldb, float *D, int ldd, void *stream);

/* The float approximations the mixed-precision kernels use, next to CUDA's
 * accurate float functions, for validation (no counterpart in the paper):
 * which = 0: atan2(a[i], b[i]); 1: log(a[i]); 2: log1p(a[i]);
 * 3: atan2(|a[i]|, b[i]) by the y >= 0 variant; 4: log1p(a[i])/2.  a, b,
 * out_fast, out_ref: device float [n] (b only for which = 0 and 3). */
int bem_fastmath_eval(bem_ctx *ctx, int which, int64_t n, const float *a, const float *b,
                      float *out_fast, float *out_ref, void *stream);

/* The double logarithm of the FP64 near field (a table-driven reduction,
 * Tang 1990), next to CUDA's log, for validation (no counterpart in the
 * paper): out_lib[i] = the library's log(x[i]), out_ref[i] = CUDA's log(x[i]).
 * x: device double [n], positive, normal and finite; out_lib, out_ref:
 * device double [n].  Errors: BEM_EINVAL for bad arguments. */
int bem_dlog_eval(bem_ctx *ctx, int64_t n, const double *x, double *out_lib, double *out_ref,
                  void *stream);

/* The double arctangent of the FP64 near field (octant reduction, a table of
 * 64 breakpoints and the addition theorem), next to CUDA's atan2, for
 * validation (no counterpart in the paper): out_lib[i] = the library's
 * atan2(y[i], x[i]), out_ref[i] = CUDA's.  y: device double [n], y >= 0;
 * x: device double [n]; both finite, of magnitude within [2^-1000, 2^1000]
 * or zero; out_lib, out_ref: device double [n].  Errors: BEM_EINVAL for bad
 * arguments. */
int bem_datan2_eval(bem_ctx *ctx, int64_t n, const double *y, const double *x, double *out_lib,
                    double *out_ref, void *stream);

/* The pairing of the bf16 Gram kernel, exposed for validation (host only, no
 * context, no GPU).  The upper 128 x 128 blocks (i <= j) of a channel's Gram
 * matrix in its J-row order, tiles block rows, are computed in units of two
 * blocks that share an operand slab; channel 0 takes the block rows
 * 0 .. tiles-1, channels 1 and 2 only the rows of their position range (the
 * blocks of the jump columns with each other are the same for all channels).
 * out[0..3] = {kind, a0, a1, b} of unit `unit` over the block rows
 * 0 .. rows-1:
 *   kind 1: blocks (a0, b) and (a0, b + 1), one N = 256 product;
 *   kind 2: blocks (a0, b) and (a1, b), two products on one B slab;
 *   kind 0: block (a0, b) alone.
 * Every upper block of those rows belongs to exactly one unit.  Errors:
 * BEM_EINVAL for tiles < 1, rows outside [1, tiles], unit outside
 * [0, number of units) or out == NULL. */
int bem_gram_unit(int tiles, int rows, int unit, int32_t *out);

/* bem_vjp without any device allocation (the paper has no counterpart; this
 * is for callers, not for the method).  Some callers may not allocate GPU
 * memory while they run the hot path: real-time loops that must never enter
 * the allocator (cudaMalloc and cudaFree can stall the whole device), and
 * host programs whose own memory pool owns the GPU and hands out no more
 * device memory once it is set up.  This entry point
 * computes the same vector-Jacobian product as bem_vjp on a context that
 * bem_setup and bem_factor have already prepared, taking every per-call
 * buffer from one static device array of 32 MiB that the library reserves
 * on each GPU that loads it (held until the process exits); it calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   - In BEM_MIXED contexts every pair is evaluated in float (no double near
 *     field), so the result agrees with bem_vjp to the mixed-path gradient
 *     accuracy; in BEM_FP64 contexts the arithmetic is the same as bem_vjp's.
 *   - Scenes whose panel sums do not fit the array (about 190,000 panels at
 *     1,024 boundary segments) are rejected with BEM_EINVAL and a message.
 *   - The first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *   - All calls on a device share the array and it keeps the last call's
 *     contents (each call writes what it reads).  Calls whose GPU work
 *     overlaps (other streams, other threads) race on it: serialise them.
 * Arguments and layouts as bem_vjp. */
int bem_vjp_noalloc(bem_ctx *ctx, int64_t n, const void *xy, const void *resid,
                    double *grad_out, void *stream);

/* ---- batches of scenes ------------------------------------------------
 * Many independent scenes of uneven size stepped together.  The paper fits
 * one scene at a time, so it has no counterpart; each scene's step is the
 * one lm_step computes (Sec. 4.3).  The bulk sample x panel work of all
 * scenes (the evaluation at theta and the evaluation of every damping
 * trial) runs in one persistent launch each, replayed from a captured CUDA
 * graph; its tile shape is chosen by timing the candidates on the first call. */
typedef struct bem_batch bem_batch;

/* Borrow n_scenes contexts (they must outlive the batch).  Each must be a
 * BEM_MIXED context that is set up and factored; all must share the device,
 * eps_c, eps_d and whether the near field is used.  The batch shares scene
 * 0's Gauss-Newton chunk buffers with the others until it is destroyed.
 * *out receives the batch.  Errors: BEM_EINVAL (message on scenes[0]). */
int bem_batch_create(bem_batch **out, bem_ctx *const *scenes, int n_scenes);
void bem_batch_destroy(bem_batch *b);

/* One LM iteration of every scene, each with the same n_trials (1..16)
 * damping values; out[s] is scene s's result as lm_step reports it, and
 * each scene's theta is updated when its best trial lowers its loss.
 *   n[s]: samples of scene s (> 0); xy[s], target[s]: device float
 *   pointers ([n][2], [n][3]); lambdas, out: host arrays.
 * The batch works on its own stream, ordered after `stream` and before any
 * later work on it; the call synchronises.  Errors: as lm_step, reported on
 * scenes[0] with the failing scene's index. */
int bem_batch_lm(bem_batch *b, const int64_t *n, const void *const *xy,
                 const void *const *target, int n_trials, const double *lambdas,
                 lm_result *out, void *stream);

/* The tile shape the batch uses: points per tile and CTAs per SM (0 before
 * the first bem_batch_lm). */
int bem_batch_tile_shape(const bem_batch *b, int *points_per_tile, int *ctas_per_sm);

/* Sizes of the current scene (host ints; any pointer may be NULL). */
int bem_sizes(const bem_ctx *ctx, int *n_theta, int *n_panels, int *n_boundary);

/* Copy the boundary solution u_b (double [n_boundary][3]) of the current
 * theta to host memory (diagnostics and tests; synchronises). */
int bem_boundary_values(bem_ctx *ctx, double *ub_out, void *stream);

/* Number of this library's kernels launched by the context so far. */
int64_t bem_launch_count(const bem_ctx *ctx);

/* Throughput of one SM pipe the float pair kernels issue to, measured on
 * the context's device: the denominators of those kernels' roofline (no
 * counterpart in the paper).  which = 0: FP32 fused multiply-add; 1: MUFU
 * base-2 logarithm; 2: MUFU reciprocal; 3: MUFU reciprocal square root.  One
 * warm-up launch, then `launches` (1..1000) timed launches of about 30 ms
 * each, every thread with eight independent chains of the operation;
 * *ops_per_s receives the median launch's operations per second (one fused
 * multiply-add counts as one operation).  Synchronises `stream`.  Errors:
 * BEM_EINVAL. */
int bem_pipe_peak(bem_ctx *ctx, int which, int launches, double *ops_per_s, void *stream);

/* Number of device allocations (cudaMalloc calls) the context has made so
 * far: its buffers grow on demand and never shrink, so a call that needs no
 * new buffer leaves the count as it is (no counterpart in the paper). */
int64_t bem_alloc_count(const bem_ctx *ctx);

/* Limit of the bounded waits inside the tensor-core kernels (bem_jtj,
 * lm_step and bem_gemm_bf16 in the tensor-core J^T J modes): a wait for a
 * pipeline slot that is not free after `seconds` of device time gives up,
 * the kernel records the failure in the context's device status word, lets
 * the copies and MMAs it has already issued finish (their own waits keep a
 * one-second limit), frees its tensor memory and returns; the call then
 * reports BEM_ETIMEDOUT and the context stays usable.  Default 1.0; 0 gives
 * up at the first wait that is not already complete (to exercise the
 * failure path).  No counterpart in the paper.  Errors: BEM_EINVAL for a
 * negative or non-finite value or more than 60 seconds. */
int bem_set_wait_limit(bem_ctx *ctx, double seconds);

/* The Gauss-Newton products of one LM iteration at the current theta, as
 * lm_step forms them before its solve (Eq. (losshessian), (lossjacobian),
 * uniform density, the same n samples for both):
 *   loss_out  host double: L = (1/2n) sum |u - min(t,1)|^2
 *   g_out     device double [n_theta]: g = (1/n) J^T r
 *   H_out     device double [n_theta][n_theta]: H = (1/n) J^T J
 * (any of the three may be NULL); the data term only, without the Sec. 4.4
 * regularisers lm_step adds.  xy, target: device (sample type).
 * Synchronises `stream`.  Errors: as lm_step. */
int bem_gn_products(bem_ctx *ctx, int64_t n, const void *xy, const void *target,
                    double *loss_out, double *g_out, double *H_out, void *stream);

/* Per-kernel timing (tracing support; no counterpart in the paper).  While
 * enabled, every hot kernel launch (field evaluation, adjoint, J rows, J^T J
 * products, LM solve) is bracketed by CUDA events recorded on the stream it
 * is launched on.  Enabling or disabling clears the totals. */
int bem_profile_enable(bem_ctx *ctx, int on);

/* Resolve the recorded events (synchronises them) and copy up to
 * max_entries totals: names (host char[max_entries][32], NUL-terminated),
 * total_ms (host double[]), counts (host int64[]; any of the three may be
 * NULL); *n_entries receives the number written. */
int bem_profile_read(bem_ctx *ctx, int max_entries, char *names, double *total_ms,
                     int64_t *counts, int *n_entries);

#ifdef __cplusplus
}
#endif
#endif /* BEMGB_H */
