// C ABI of libbemgb: context lifecycle and the hot-path entry points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "ctx.h"

namespace bem {

static std::string g_create_err = "no error";

int fail(bem_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_err = msg;
  return code;
}

int cuda_check(bem_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return BEM_OK;
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  return fail(c, e == cudaErrorMemoryAllocation ? BEM_ENOMEM : BEM_ECUDA, buf);
}

int grow(bem_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes <= b.cap) return BEM_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t want = bytes + bytes / 8;
  ++c->allocs;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return cuda_check(c, e, "device allocation");
  }
  b.cap = want;
  return BEM_OK;
}

template <typename T>
static int alloc(bem_ctx* c, T*& p, size_t count) {
  if (p) cudaFree(p);
  p = nullptr;
  if (count == 0) count = 1;
  ++c->allocs;
  return cuda_check(c, cudaMalloc((void**)&p, sizeof(T) * count), "device allocation");
}

static void free_buf(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

static int set_device(bem_ctx* c) { return cuda_check(c, cudaSetDevice(c->device), "cudaSetDevice"); }

// device tables and solutions sized by the number of boundary segments
static int alloc_boundary(bem_ctx* c) {
  const size_t Nb = (size_t)c->bd.Nb;
  int rc;
  if ((rc = alloc(c, c->bd.d_vert, 2 * (Nb + 1))) || (rc = alloc(c, c->bd.d_vert32, 2 * (Nb + 1))) ||
      (rc = alloc(c, c->bd.d_gp, 6 * Nb)) || (rc = alloc(c, c->bd.d_gp32, 6 * Nb)) ||
      (rc = alloc(c, c->bd.d_A, Nb * Nb)) || (rc = alloc(c, c->bd.d_W, Nb * Nb)) ||
      (rc = alloc(c, c->bd.d_WT, Nb * Nb)) || (rc = alloc(c, c->bd.d_W32, Nb * Nb)) ||
      (rc = alloc(c, c->bd.d_WT32, Nb * Nb)) || (rc = alloc(c, c->d_ub, 3 * Nb)) ||
      (rc = alloc(c, c->d_fb, 3 * Nb)) || (rc = alloc(c, c->d_q, 3 * Nb)) ||
      (rc = alloc(c, c->d_lb, 3 * Nb)))
    return rc;
  return BEM_OK;
}


int ctx_set_device(bem_ctx* c) { return set_device(c); }

// panels, compatibility weights and boundary solution of the current theta
static int refresh(bem_ctx* c, const double* theta) {
  int rc;
  if ((rc = geom_panelize(c, theta))) return rc;
  if ((rc = field_rhs(c))) return rc;
  return field_solve(c);
}
int ctx_refresh(bem_ctx* c, const double* theta) { return refresh(c, theta); }

static int need_ready(bem_ctx* c) {
  if (!c->have_scene) return fail(c, BEM_ESTATE, "bem_setup has not been called");
  if (!c->bd.factored) return fail(c, BEM_ESTATE, "bem_factor has not been called");
  return BEM_OK;
}
int ctx_ready(bem_ctx* c) { return need_ready(c); }

static cudaEvent_t prof_event(bem_ctx* c) {
  if (!c->prof_pool.empty()) {
    cudaEvent_t e = c->prof_pool.back();
    c->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(bem_ctx* ctx, const char* name) : c(ctx) {
  if (!c->prof) return;
  bem_ctx::ProfRec r{name, prof_event(c), prof_event(c)};
  cudaEventRecord(r.a, S(c));
  c->prof_pending.push_back(r);
  idx = (int)c->prof_pending.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx >= 0) cudaEventRecord(c->prof_pending[idx].b, S(c));
}

static void prof_resolve(bem_ctx* c) {
  for (auto& r : c->prof_pending) {
    cudaEventSynchronize(r.b);
    float ms = 0;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& t = c->prof_tot[r.name];
    t.first += ms;
    t.second += 1;
    c->prof_pool.push_back(r.a);
    c->prof_pool.push_back(r.b);
  }
  c->prof_pending.clear();
}

// out = a + b
__global__ void k_axpy(const double* __restrict__ a, const double* __restrict__ b, int n,
                       double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] + b[i];
}

// v *= s; *norm2 = |v|^2 after scaling (one block)
__global__ void k_scale_norm(double* __restrict__ v, int n, double s, double* __restrict__ norm2) {
  __shared__ double red[32];
  double acc = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double x = v[i] * s;
    v[i] = x;
    acc += x * x;
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    *norm2 = t;
  }
}

void ctx_axpy(bem_ctx* c, const double* a, const double* b, int n, double* out) {
  k_axpy<<<(n + 255) / 256, 256, 0, S(c)>>>(a, b, n, out);
  BEM_LAUNCHED(c);
}

void ctx_scale_norm(bem_ctx* c, double* v, int n, double s, double* norm2) {
  k_scale_norm<<<1, 1024, 0, S(c)>>>(v, n, s, norm2);
  BEM_LAUNCHED(c);
}

// which = 0: atan2(a, b); 1: log(a); 2: log1p(a).  Library approximation and
// CUDA's accurate float function side by side.
__global__ void k_fastmath(int which, int64_t n, const float* __restrict__ a,
                           const float* __restrict__ b, float* __restrict__ fast,
                           float* __restrict__ ref) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x = a[i];
  if (which == 0) {
    fast[i] = fm_atan2(x, b[i]);
    ref[i] = atan2f(x, b[i]);
  } else if (which == 1) {
    fast[i] = fm_log(x);
    ref[i] = logf(x);
  } else if (which == 2) {
    fast[i] = fm_log1p(x);
    ref[i] = log1pf(x);
  } else if (which == 3) {
    fast[i] = fm_atan2_ypos(fabsf(x), b[i]);
    ref[i] = atan2f(fabsf(x), b[i]);
  } else {
    fast[i] = fm_log1p_half(x);
    ref[i] = 0.5f * log1pf(x);
  }
}

// pixel centres ((i + 1/2)/W, (j + 1/2)/H) of pixels p0 .. p0 + cnt - 1 (row-major)
template <typename T>
__global__ void k_pixel_centres(int W, int H, int64_t p0, int64_t cnt, T* __restrict__ xy) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  const int64_t p = p0 + k;
  const int i = (int)(p % W), j = (int)(p / W);
  xy[2 * k] = T((i + 0.5) / W);
  xy[2 * k + 1] = T((j + 0.5) / H);
}

// panel midpoints a + (L/2) tau
template <typename T>
__global__ void k_panel_mids(const Panel<double>* __restrict__ pan, int P, T* __restrict__ xy) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const Panel<double> q = pan[p];
  xy[2 * p] = T(q.ax + 0.5 * q.L * q.tx);
  xy[2 * p + 1] = T(q.ay + 0.5 * q.L * q.ty);
}

// out[p][0] = u(mid) + w_d/2 (left of a->b), out[p][1] = u(mid) - w_d/2 (right)
template <typename T>
__global__ void k_two_sided(const T* __restrict__ u, const Panel<double>* __restrict__ pan, int P,
                            double* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  for (int ch = 0; ch < 3; ++ch) {
    const double avg = double(u[3 * p + ch]), h = 0.5 * pan[p].wd[ch];
    out[6 * p + ch] = avg + h;
    out[6 * p + 3 + ch] = avg - h;
  }
}

}  // namespace bem

using namespace bem;

extern "C" {

int bem_default_opts(bem_opts* o) {
  if (!o) return BEM_EINVAL;
  memset(o, 0, sizeof(*o));
  o->precision = BEM_FP64;
  o->eps_d = 1e-2;
  o->eps_c = 1e-2;
  o->segs_per_side = 256;
  o->near_factor = 0.5;
  o->jtj_mode = BEM_JTJ_FP64;
  o->lm_solver = BEM_LM_AUTO;
  o->galerkin_mode = 0;
  return BEM_OK;
}

int bem_create(bem_ctx** out, const bem_opts* opts, int device) {
  if (!out) return fail(nullptr, BEM_EINVAL, "out is NULL");
  *out = nullptr;
  bem_opts o;
  if (opts) o = *opts;
  else bem_default_opts(&o);
  if (o.precision != BEM_FP64 && o.precision != BEM_MIXED)
    return fail(nullptr, BEM_EINVAL, "precision must be BEM_FP64 or BEM_MIXED");
  if (!(o.eps_d > 0) || !(o.eps_c > 0) || !std::isfinite(o.eps_d) || !std::isfinite(o.eps_c))
    return fail(nullptr, BEM_EINVAL, "eps_d and eps_c must be positive");
  if (o.segs_per_side < 1 || o.segs_per_side > 4096)
    return fail(nullptr, BEM_EINVAL, "segs_per_side must be in [1, 4096]");
  if (!(o.near_factor >= 0)) return fail(nullptr, BEM_EINVAL, "near_factor must be >= 0");
  if (o.jtj_mode < BEM_JTJ_FP64 || o.jtj_mode > BEM_JTJ_BF16X3)
    return fail(nullptr, BEM_EINVAL, "unknown jtj_mode");
  if (o.lm_solver != BEM_LM_AUTO && o.lm_solver != BEM_LM_FP64)
    return fail(nullptr, BEM_EINVAL, "unknown lm_solver");
  if (o.galerkin_mode != 0 && o.galerkin_mode != 1)
    return fail(nullptr, BEM_EINVAL, "unknown galerkin_mode");
  if (o.gn_chunk != 0 && (o.gn_chunk < 128 || o.gn_chunk > (1 << 22) || o.gn_chunk % 128))
    return fail(nullptr, BEM_EINVAL, "gn_chunk must be 0 or a multiple of 128 in [128, 4194304]");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(nullptr, BEM_ECUDA, "no such CUDA device");
  bem_ctx* c = new (std::nothrow) bem_ctx();
  if (!c) return fail(nullptr, BEM_ENOMEM, "host allocation");
  c->device = device;
  c->opts = o;
  int rc;
  if ((rc = set_device(c))) { g_create_err = c->err; delete c; return rc; }
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      c->sms < 1) {
    g_create_err = "cannot read the multiprocessor count";
    delete c;
    return BEM_ECUDA;
  }
  c->bd.M = o.segs_per_side;
  c->bd.Nb = 4 * o.segs_per_side;
  if ((rc = alloc_boundary(c)) || (rc = alloc(c, c->d_scal, 64)) || (rc = alloc(c, c->d_status, 4))) {
    g_create_err = c->err;
    bem_destroy(c);
    return rc;
  }
  if ((rc = geom_boundary_tables(c))) { g_create_err = c->err; bem_destroy(c); return rc; }
  *out = c;
  return BEM_OK;
}

void bem_destroy(bem_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  void* ptrs[] = {c->bd.d_vert, c->bd.d_vert32, c->bd.d_gp, c->bd.d_gp32, c->bd.d_A, c->bd.d_W,
                  c->bd.d_WT, c->bd.d_W32, c->bd.d_WT32, c->d_ub, c->d_fb, c->d_q, c->d_lb,
                  c->d_scal, c->d_status, c->d_theta, c->d_trial, c->d_delta, c->d_pan64,
                  c->d_pan32, c->d_compat, c->sc.d_pcurve, c->sc.d_pk, c->sc.d_off, c->sc.d_K,
                  c->sc.d_closed};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  prof_resolve(c);
  for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
  DevBuf* bufs[] = {&c->part, &c->part2, &c->loss, &c->gpart, &c->jrow, &c->phi, &c->Hc, &c->Mc,
                    &c->Dfc, &c->Fg, &c->lmK, &c->lmL, &c->lmLt, &c->lmW, &c->H, &c->g, &c->rend,
                    &c->tcJ, &c->tcPart, &c->tcMt, &c->nearP, &c->nearS, &c->nearF, &c->gwork,
                    &c->regw, &c->hin_xy, &c->hin_t};
  for (DevBuf* b : bufs) free_buf(*b);
  if (c->hin_stream) cudaStreamDestroy(c->hin_stream);
  if (c->hin_start) cudaEventDestroy(c->hin_start);
  if (c->hin_xy_ready) cudaEventDestroy(c->hin_xy_ready);
  for (cudaEvent_t e : c->hin_t_ready) cudaEventDestroy(e);
  delete c;
}

const char* bem_last_error(const bem_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

}  // extern "C"

namespace bem {

// Scene of n_curves handles with the given panels per handle; pp = 2: cubic
// Bezier curves (4 control handles of 8 parameters), pp = 4: segment
// handles (10 parameters, one panel each).
static int setup_scene(bem_ctx* c, int n_curves, const int32_t* ppc, const uint8_t* closed,
                       const double* theta, const double* mean_color, int pp) {
  int rc;
  if ((rc = set_device(c))) return rc;
  Scene& s = c->sc;
  s.C = n_curves;
  s.K.assign(ppc, ppc + n_curves);
  s.closed.assign(closed, closed + n_curves);
  s.off.assign(n_curves + 1, 0);
  for (int i = 0; i < n_curves; ++i) {
    if (s.K[i] < 1 || s.K[i] > (1 << 20)) return fail(c, BEM_EINVAL, "panels_per_curve out of range");
    s.off[i + 1] = s.off[i] + s.K[i];
  }
  s.pp = pp;
  s.NH = pp == 4 ? n_curves : 4 * n_curves;
  s.nth = (pp + 6) * s.NH;
  s.nc = (pp + 2) * s.NH;
  for (int i = 0; i < s.nth; ++i)
    if (!std::isfinite(theta[i])) return fail(c, BEM_EINVAL, "theta has a non-finite entry");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(mean_color[k])) return fail(c, BEM_EINVAL, "mean colour not finite");
  s.P = s.off[n_curves];
  std::vector<int> pc(s.P), pk(s.P);
  for (int i = 0; i < n_curves; ++i)
    for (int k = 0; k < s.K[i]; ++k) { pc[s.off[i] + k] = i; pk[s.off[i] + k] = k; }
  if ((rc = alloc(c, s.d_pcurve, s.P)) || (rc = alloc(c, s.d_pk, s.P)) ||
      (rc = alloc(c, s.d_off, n_curves + 1)) || (rc = alloc(c, s.d_K, n_curves)) ||
      (rc = alloc(c, s.d_closed, n_curves)) || (rc = alloc(c, c->d_theta, s.nth)) ||
      (rc = alloc(c, c->d_trial, s.nth)) || (rc = alloc(c, c->d_delta, s.nth)) ||
      (rc = alloc(c, c->d_pan64, s.P)) || (rc = alloc(c, c->d_pan32, s.P)) ||
      (rc = alloc(c, c->d_compat, (size_t)s.NH)))
    return rc;
  if ((rc = cuda_check(c, cudaMemcpy(s.d_pcurve, pc.data(), 4 * s.P, cudaMemcpyHostToDevice), "copy")) ||
      (rc = cuda_check(c, cudaMemcpy(s.d_pk, pk.data(), 4 * s.P, cudaMemcpyHostToDevice), "copy")) ||
      (rc = cuda_check(c, cudaMemcpy(s.d_off, s.off.data(), 4 * (n_curves + 1), cudaMemcpyHostToDevice), "copy")) ||
      (rc = cuda_check(c, cudaMemcpy(s.d_K, s.K.data(), 4 * n_curves, cudaMemcpyHostToDevice), "copy")) ||
      (rc = cuda_check(c, cudaMemcpy(s.d_closed, s.closed.data(), n_curves, cudaMemcpyHostToDevice), "copy")) ||
      (rc = cuda_check(c, cudaMemcpy(c->d_theta, theta, 8 * s.nth, cudaMemcpyHostToDevice), "copy")))
    return rc;
  memcpy(c->mean, mean_color, sizeof(c->mean));
  c->have_scene = true;
  return BEM_OK;
}

}  // namespace bem

extern "C" {

int bem_setup(bem_ctx* c, int n_curves, const int32_t* ppc, const uint8_t* closed,
              const double* theta, const double* mean_color) {
  if (!c) return BEM_EINVAL;
  if (n_curves < 1 || !ppc || !closed || !theta || !mean_color)
    return fail(c, BEM_EINVAL, "bem_setup: n_curves >= 1 and non-NULL arrays required");
  return setup_scene(c, n_curves, ppc, closed, theta, mean_color, 2);
}

int bem_setup_segments(bem_ctx* c, int n_handles, const double* theta, const double* mean_color) {
  if (!c) return BEM_EINVAL;
  if (n_handles < 1 || n_handles > (1 << 20) || !theta || !mean_color)
    return fail(c, BEM_EINVAL, "bem_setup_segments: n_handles >= 1 and non-NULL arrays required");
  std::vector<int32_t> one(n_handles, 1);
  std::vector<uint8_t> open(n_handles, 0);
  return setup_scene(c, n_handles, one.data(), open.data(), theta, mean_color, 4);
}

int bem_set_regularizers(bem_ctx* c, const bem_reg* r) {
  if (!c) return BEM_EINVAL;
  if (!r) {
    c->reg = bem_reg{};
    return BEM_OK;
  }
  const double v[9] = {r->len_weight, r->len_max, r->snap_weight, r->snap_radius, r->snap_alpha,
                       r->sparse_wd, r->sparse_wc, r->sparse_eps, r->sparse_t};
  for (double x : v)
    if (!std::isfinite(x) || x < 0) return fail(c, BEM_EINVAL, "regulariser settings must be finite and >= 0");
  if (r->snap_weight > 0 && (!(r->snap_radius > 0) || r->snap_alpha > 1))
    return fail(c, BEM_EINVAL, "snapping needs snap_radius > 0 and snap_alpha in [0, 1]");
  if ((r->sparse_wd > 0 || r->sparse_wc > 0) && (!(r->sparse_eps > 0) || !(r->sparse_t > 0)))
    return fail(c, BEM_EINVAL, "sparsity needs sparse_eps > 0 and sparse_t > 0");
  if (!c->have_scene || c->sc.pp != 4)
    return fail(c, BEM_ESTATE, "regularisers need a scene of segment handles (bem_setup_segments)");
  c->reg = *r;
  return BEM_OK;
}

int bem_prune(bem_ctx* c, double threshold, int* n_kept, int32_t* kept_index, void* stream) {
  if (!c) return BEM_EINVAL;
  if (!n_kept || !(threshold >= 0) || !std::isfinite(threshold))
    return fail(c, BEM_EINVAL, "bem_prune: finite threshold >= 0 and n_kept required");
  int rc;
  if ((rc = need_ready(c)) || (rc = set_device(c))) return rc;
  if (c->sc.pp != 4) return fail(c, BEM_ESTATE, "bem_prune needs segment handles (bem_setup_segments)");
  c->cur = (cudaStream_t)stream;
  const int H = c->sc.NH;
  std::vector<double> th;
  std::vector<int> idx;
  if ((rc = reg_prune(c, threshold, th, idx))) return rc;
  const int n = (int)idx.size();
  *n_kept = n;
  if (n == 0) return BEM_OK;
  if (kept_index)
    for (int i = 0; i < n; ++i) kept_index[i] = idx[i];
  if (n == H) return BEM_OK;
  const double mean[3] = {c->mean[0], c->mean[1], c->mean[2]};
  std::vector<int32_t> one(n, 1);
  std::vector<uint8_t> open(n, 0);
  if ((rc = setup_scene(c, n, one.data(), open.data(), th.data(), mean, 4))) return rc;
  // w_c re-projected with the lengths of the kept handles (Sec. 4.3)
  if ((rc = geom_panelize(c, c->d_theta)) || (rc = geom_compat(c, c->d_theta, true))) return rc;
  return cuda_check(c, cudaStreamSynchronize(S(c)), "sync");
}

int bem_set_boundary(bem_ctx* c, int n_vertices, const double* vertices, int segs_per_edge) {
  if (!c) return BEM_EINVAL;
  if (n_vertices < 3 || !vertices || segs_per_edge < 1)
    return fail(c, BEM_EINVAL, "bem_set_boundary: bad arguments");
  const int64_t Nb = (int64_t)n_vertices * segs_per_edge;
  if (Nb > 8192) return fail(c, BEM_EINVAL, "bem_set_boundary: more than 8192 boundary segments");
  double area2 = 0;
  for (int e = 0; e < n_vertices; ++e) {
    const double ax = vertices[2 * e], ay = vertices[2 * e + 1];
    const double bx = vertices[2 * ((e + 1) % n_vertices)], by = vertices[2 * ((e + 1) % n_vertices) + 1];
    if (!(ax >= 0 && ax <= 1 && ay >= 0 && ay <= 1))
      return fail(c, BEM_EINVAL, "bem_set_boundary: vertices must lie in the unit square");
    if (ax == bx && ay == by) return fail(c, BEM_EINVAL, "bem_set_boundary: zero-length edge");
    area2 += ax * by - bx * ay;
  }
  if (!(area2 > 0)) return fail(c, BEM_EINVAL, "bem_set_boundary: polygon must be counter-clockwise");
  int rc;
  if ((rc = set_device(c))) return rc;
  c->bd.poly.assign(vertices, vertices + 2 * n_vertices);
  c->bd.M = segs_per_edge;
  c->bd.Nb = (int)Nb;
  c->bd.factored = false;
  if ((rc = cuda_check(c, cudaDeviceSynchronize(), "sync")) || (rc = alloc_boundary(c)))
    return rc;
  return geom_boundary_tables(c);
}

int bem_factor(bem_ctx* c, void* stream) {
  if (!c) return BEM_EINVAL;
  int rc;
  if ((rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  c->bd.factored = false;
  if ((rc = geom_assemble(c))) return rc;
  if ((rc = la_pinv(c))) return rc;
  c->bd.factored = true;
  return BEM_OK;
}

int bem_set_params(bem_ctx* c, const double* theta, int on_dev, void* stream) {
  if (!c || !theta) return c ? fail(c, BEM_EINVAL, "theta is NULL") : BEM_EINVAL;
  if (!c->have_scene) return fail(c, BEM_ESTATE, "bem_setup has not been called");
  int rc;
  if ((rc = set_device(c))) return rc;
  return cuda_check(c, cudaMemcpyAsync(c->d_theta, theta, 8 * (size_t)c->sc.nth,
                                       on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                       (cudaStream_t)stream),
                    "set params");
}

int bem_get_params(bem_ctx* c, double* out, void* stream) {
  if (!c || !out) return c ? fail(c, BEM_EINVAL, "out is NULL") : BEM_EINVAL;
  if (!c->have_scene) return fail(c, BEM_ESTATE, "bem_setup has not been called");
  int rc;
  if ((rc = set_device(c))) return rc;
  if ((rc = cuda_check(c, cudaMemcpyAsync(out, c->d_theta, 8 * (size_t)c->sc.nth,
                                          cudaMemcpyDeviceToHost, (cudaStream_t)stream), "get params")))
    return rc;
  return cuda_check(c, cudaStreamSynchronize((cudaStream_t)stream), "sync");
}

int bem_set_mean_color(bem_ctx* c, const double* m) {
  if (!c || !m) return c ? fail(c, BEM_EINVAL, "mean is NULL") : BEM_EINVAL;
  memcpy(c->mean, m, sizeof(c->mean));
  return BEM_OK;
}

int bem_sample_mean(bem_ctx* c, int64_t n, const void* target, double* mean_out, void* stream) {
  if (!c || !mean_out || n < 0 || (n > 0 && !target)) return c ? fail(c, BEM_EINVAL, "bad arguments") : BEM_EINVAL;
  int rc;
  if ((rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  return field_sample_mean(c, n, target, mean_out);
}

int bem_eval(bem_ctx* c, int64_t n, const void* xy, void* rgb, void* stream) {
  if (!c) return BEM_EINVAL;
  if (n < 0 || (n > 0 && (!xy || !rgb))) return fail(c, BEM_EINVAL, "bem_eval: bad arguments");
  int rc;
  if ((rc = need_ready(c)) || (rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  if ((rc = refresh(c, c->d_theta))) return rc;
  return field_eval(c, n, xy, rgb, nullptr, nullptr, false);
}

int bem_render(bem_ctx* c, int width, int height, void* rgb, void* stream) {
  if (!c) return BEM_EINVAL;
  if (width < 1 || height < 1 || !rgb) return fail(c, BEM_EINVAL, "bem_render: bad arguments");
  int rc;
  if ((rc = need_ready(c)) || (rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  if ((rc = refresh(c, c->d_theta))) return rc;
  const bool f64 = c->opts.precision == BEM_FP64;
  const size_t es = f64 ? 8 : 4;
  const int64_t total = (int64_t)width * height, chunk = std::min<int64_t>(total, 1 << 22);
  if ((rc = grow(c, c->rend, 2 * es * (size_t)chunk))) return rc;
  for (int64_t p0 = 0; p0 < total; p0 += chunk) {
    const int64_t cnt = std::min(chunk, total - p0);
    if (f64) k_pixel_centres<double><<<(unsigned)((cnt + 255) / 256), 256, 0, S(c)>>>(width, height, p0, cnt, (double*)c->rend.p);
    else k_pixel_centres<float><<<(unsigned)((cnt + 255) / 256), 256, 0, S(c)>>>(width, height, p0, cnt, (float*)c->rend.p);
    BEM_LAUNCHED(c);
    if ((rc = field_eval(c, cnt, c->rend.p, (char*)rgb + 3 * es * (size_t)p0, nullptr, nullptr, false)))
      return rc;
  }
  return cuda_check(c, cudaGetLastError(), "bem_render");
}

int bem_handle_colors(bem_ctx* c, double* out, void* stream) {
  if (!c) return BEM_EINVAL;
  if (!out) return fail(c, BEM_EINVAL, "bem_handle_colors: out is NULL");
  int rc;
  if ((rc = need_ready(c)) || (rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  if ((rc = refresh(c, c->d_theta))) return rc;
  const bool f64 = c->opts.precision == BEM_FP64;
  const size_t es = f64 ? 8 : 4;
  const int P = c->sc.P;
  // scratch: midpoints [P][2], colours [P][3] (sample type), result [P][2][3] double
  const size_t xyb = ((2 * es * (size_t)P + 255) / 256) * 256;
  const size_t ub = ((3 * es * (size_t)P + 255) / 256) * 256;
  if ((rc = grow(c, c->rend, xyb + ub + sizeof(double) * 6 * (size_t)P))) return rc;
  void* xy = c->rend.p;
  void* u = (char*)c->rend.p + xyb;
  double* o = (double*)((char*)u + ub);
  if (f64) k_panel_mids<double><<<(P + 127) / 128, 128, 0, S(c)>>>(c->d_pan64, P, (double*)xy);
  else k_panel_mids<float><<<(P + 127) / 128, 128, 0, S(c)>>>(c->d_pan64, P, (float*)xy);
  BEM_LAUNCHED(c);
  if ((rc = field_eval(c, P, xy, u, nullptr, nullptr, false))) return rc;
  if (f64) k_two_sided<double><<<(P + 127) / 128, 128, 0, S(c)>>>((const double*)u, c->d_pan64, P, o);
  else k_two_sided<float><<<(P + 127) / 128, 128, 0, S(c)>>>((const float*)u, c->d_pan64, P, o);
  BEM_LAUNCHED(c);
  if ((rc = cuda_check(c, cudaMemcpyAsync(out, o, sizeof(double) * 6 * (size_t)P,
                                          cudaMemcpyDeviceToHost, S(c)), "colors")))
    return rc;
  return cuda_check(c, cudaStreamSynchronize(S(c)), "sync");
}

int bem_loss(bem_ctx* c, int64_t n, const void* xy, const void* target, void* resid, double* loss,
             void* stream) {
  if (!c) return BEM_EINVAL;
  if (n < 0 || !loss || (n > 0 && (!xy || !target))) return fail(c, BEM_EINVAL, "bem_loss: bad arguments");
  int rc;
  if ((rc = need_ready(c)) || (rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  if ((rc = refresh(c, c->d_theta))) return rc;
  if ((rc = field_eval(c, n, xy, nullptr, target, resid, true))) return rc;
  double s = 0;
  if ((rc = cuda_check(c, cudaMemcpyAsync(&s, c->d_scal, 8, cudaMemcpyDeviceToHost, S(c)), "loss")))
    return rc;
  if ((rc = cuda_check(c, cudaStreamSynchronize(S(c)), "sync"))) return rc;
  *loss = n > 0 ? 0.5 * s / double(n) : 0.0;
  return BEM_OK;
}

int bem_vjp(bem_ctx* c, int64_t n, const void* xy, const void* resid, double* grad, void* stream) {
  if (!c) return BEM_EINVAL;
  if (n < 0 || !grad || (n > 0 && (!xy || !resid))) return fail(c, BEM_EINVAL, "bem_vjp: bad arguments");
  int rc;
  if ((rc = need_ready(c)) || (rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  if ((rc = geom_panelize(c, c->d_theta))) return rc;
  return adj_vjp(c, n, xy, resid, grad);
}

int bem_jtj(bem_ctx* c, int64_t n, const void* xy, double* H, void* stream) {
  if (!c) return BEM_EINVAL;
  if (n < 0 || (n > 0 && !xy)) return fail(c, BEM_EINVAL, "bem_jtj: bad arguments");
  int rc;
  if ((rc = need_ready(c)) || (rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  size_t nn = sizeof(double) * (size_t)c->sc.nth * c->sc.nth;
  if ((rc = grow(c, c->H, nn))) return rc;
  if ((rc = geom_panelize(c, c->d_theta))) return rc;
  if ((rc = jtj_build(c, n, xy, (double*)c->H.p))) return rc;
  if (H)
    return cuda_check(c, cudaMemcpyAsync(H, c->H.p, nn, cudaMemcpyDeviceToDevice, S(c)), "copy H");
  return BEM_OK;
}

}  // extern "C"

namespace bem {

// Loss sum, residual, g = (1/n) J^T r and H of one LM iteration at the
// context's theta, whose panels and boundary solution are current; with xy_h
// the Hessian integral uses those n_h points and the gradient comes from the
// adjoint over (xy, target).  *s0 receives sum |r|^2 (host) once the stream
// reaches it; |g|^2 lands in d_scal[1].
static int gn_at_theta(bem_ctx* c, int64_t n, const void* xy, const void* target, int64_t n_h,
                       const void* xy_h, void* resid, double* g, double* H, double* s0) {
  int rc;
  const int nth = c->sc.nth;
  if (!xy_h && jtj_fuses_eval(c)) {
    // one pass over the samples: the residual at theta (handle term as F w,
    // near-field correction, boundary term), g = (1/n) J^T r (Eq.
    // (lossjacobian)) and H from the same J rows
    if ((rc = jtj_build(c, n, xy, H, resid, g, target))) return rc;
    if ((rc = cuda_check(c, cudaMemcpyAsync(s0, c->d_scal, 8, cudaMemcpyDeviceToHost, S(c)), "loss")))
      return rc;
    k_scale_norm<<<1, 1024, 0, S(c)>>>(g, nth, 1.0, c->d_scal + 1);
    BEM_LAUNCHED(c);
  } else if (!xy_h && jtj_gives_gradient(c)) {
    if ((rc = field_eval(c, n, xy, nullptr, target, resid, true))) return rc;
    if ((rc = cuda_check(c, cudaMemcpyAsync(s0, c->d_scal, 8, cudaMemcpyDeviceToHost, S(c)), "loss")))
      return rc;
    // g = (1/n) J^T r from the J rows that also build H (Eq. (lossjacobian))
    if ((rc = jtj_build(c, n, xy, H, resid, g))) return rc;
    k_scale_norm<<<1, 1024, 0, S(c)>>>(g, nth, 1.0, c->d_scal + 1);
    BEM_LAUNCHED(c);
  } else {
    if ((rc = field_eval(c, n, xy, nullptr, target, resid, true))) return rc;
    if ((rc = cuda_check(c, cudaMemcpyAsync(s0, c->d_scal, 8, cudaMemcpyDeviceToHost, S(c)), "loss")))
      return rc;
    if ((rc = adj_vjp(c, n, xy, resid, g))) return rc;
    k_scale_norm<<<1, 1024, 0, S(c)>>>(g, nth, 1.0 / double(n), c->d_scal + 1);
    BEM_LAUNCHED(c);
    if ((rc = jtj_build(c, xy_h ? n_h : n, xy_h ? xy_h : xy, H))) return rc;
  }
  return BEM_OK;
}

// One LM iteration; with xy_h the Hessian integral uses those n_h points and
// the gradient comes from the adjoint over (xy, target).
static int lm_step_impl(bem_ctx* c, int64_t n, const void* xy, const void* target, int64_t n_h,
                        const void* xy_h, int n_trials, const double* lambdas, lm_result* out,
                        void* stream) {
  if (!c) return BEM_EINVAL;
  if (n <= 0 || !xy || !target || n_trials < 1 || n_trials > 64 || !lambdas || !out ||
      (xy_h && n_h <= 0))
    return fail(c, BEM_EINVAL, "lm_step: bad arguments");
  for (int t = 0; t < n_trials; ++t)
    if (!(lambdas[t] >= 0) || !std::isfinite(lambdas[t]))
      return fail(c, BEM_EINVAL, "lambda must be finite and >= 0");
  int rc;
  if ((rc = need_ready(c)) || (rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  const int nth = c->sc.nth;
  const size_t es = c->opts.precision == BEM_FP64 ? 8 : 4;
  const size_t nn = sizeof(double) * (size_t)nth * nth;
  if ((rc = grow(c, c->H, nn))) return rc;
  // residual (sample type), gradient, best trial theta
  const size_t roff = ((es * 3 * (size_t)n + 255) / 256) * 256;
  if ((rc = grow(c, c->phi, roff + 8 * (size_t)nth * 2 + 64))) return rc;
  void* resid = c->phi.p;
  double* g = (double*)((char*)c->phi.p + roff);
  double* best_theta = g + nth;
  // loss, residual and gradient at theta; compatibility weights with the
  // current lengths (the fixed-endpoint constraint of the step)
  if ((rc = refresh(c, c->d_theta))) return rc;
  if ((rc = geom_compat(c, c->d_theta, false))) return rc;
  double s0 = 0;
  if ((rc = gn_at_theta(c, n, xy, target, n_h, xy_h, resid, g, (double*)c->H.p, &s0))) return rc;
  // Sec. 4.4 regularisers: analytic gradient and Hessian added to g and H,
  // snapping pairs chosen here and kept for the trial losses
  const bool reg = reg_active(c);
  double R[2] = {0, 0};
  if (reg) {
    if ((rc = reg_pairs(c, c->d_theta)) || (rc = reg_add(c, c->d_theta, (double*)c->H.p, g)) ||
        (rc = reg_loss(c, c->d_theta, c->d_scal + 2)))
      return rc;
    k_scale_norm<<<1, 1024, 0, S(c)>>>(g, nth, 1.0, c->d_scal + 1);
    BEM_LAUNCHED(c);
    if ((rc = cuda_check(c, cudaMemcpyAsync(R, c->d_scal + 2, 8, cudaMemcpyDeviceToHost, S(c)), "reg")))
      return rc;
  }
  double gn2 = 0;
  if ((rc = cuda_check(c, cudaMemcpyAsync(&gn2, c->d_scal + 1, 8, cudaMemcpyDeviceToHost, S(c)), "norm")) ||
      (rc = cuda_check(c, cudaStreamSynchronize(S(c)), "sync")))
    return rc;
  const double L0 = 0.5 * s0 / double(n) + R[0];
  out->grad_norm = std::sqrt(gn2);
  double best = INFINITY;
  int best_t = -1;
  bool any_spd = false;
  double used[64];
  for (int t = 0; t < n_trials; ++t) {
    // H is positive semi-definite only up to rounding; if H + lambda D does
    // not factor, lambda is raised tenfold (at most 12 times) as LM does
    double lam = lambdas[t];
    for (int r = 0;; ++r) {
      rc = la_lm_solve(c, (const double*)c->H.p, g, lam, c->d_delta);
      if (rc != BEM_ENOTSPD || r == 12) break;
      lam = lam > 0 ? 10.0 * lam : 1e-9;
    }
    used[t] = lam;
    if (rc == BEM_ENOTSPD) continue;
    if (rc) return rc;
    any_spd = true;
    // trial theta = theta + delta, then w_c re-projected with the new lengths (Sec. 4.3)
    k_axpy<<<(nth + 255) / 256, 256, 0, S(c)>>>(c->d_theta, c->d_delta, nth, c->d_trial);
    BEM_LAUNCHED(c);
    if ((rc = geom_panelize(c, c->d_trial))) return rc;
    if ((rc = geom_compat(c, c->d_trial, true))) return rc;
    if ((rc = refresh(c, c->d_trial))) return rc;
    if ((rc = field_eval(c, n, xy, nullptr, target, nullptr, true))) return rc;
    if (reg && (rc = reg_loss(c, c->d_trial, c->d_scal + 3))) return rc;
    double s1 = 0;
    if ((rc = cuda_check(c, cudaMemcpyAsync(&s1, c->d_scal, 8, cudaMemcpyDeviceToHost, S(c)), "loss")) ||
        (reg && (rc = cuda_check(c, cudaMemcpyAsync(R + 1, c->d_scal + 3, 8, cudaMemcpyDeviceToHost,
                                                     S(c)), "reg"))) ||
        (rc = cuda_check(c, cudaStreamSynchronize(S(c)), "sync")))
      return rc;
    const double L1 = 0.5 * s1 / double(n) + R[1];
    if (L1 < best) {
      best = L1;
      best_t = t;
      if ((rc = cuda_check(c, cudaMemcpyAsync(best_theta, c->d_trial, 8 * (size_t)nth,
                                              cudaMemcpyDeviceToDevice, S(c)), "keep")))
        return rc;
    }
  }
  if (!any_spd) return fail(c, BEM_ENOTSPD, "LM matrix not positive definite for any trial lambda");
  out->loss_before = L0;
  out->loss_after = best;
  out->accepted = best < L0 ? 1 : 0;
  out->best_trial = out->accepted ? best_t : -1;
  if (out->accepted) {
    if ((rc = cuda_check(c, cudaMemcpyAsync(c->d_theta, best_theta, 8 * (size_t)nth,
                                            cudaMemcpyDeviceToDevice, S(c)), "theta")))
      return rc;
    out->lambda_next = used[best_t] / 3.0;
  } else {
    double mx = 0;
    for (int t = 0; t < n_trials; ++t) mx = std::fmax(mx, used[t]);
    out->lambda_next = n_trials == 1 ? 2.0 * used[0] : 10.0 * mx;
  }
  // panels and boundary solution are rebuilt from theta by the next call
  return cuda_check(c, cudaStreamSynchronize(S(c)), "sync");
}

}  // namespace bem

extern "C" {

int lm_step(bem_ctx* c, int64_t n, const void* xy, const void* target, int n_trials,
            const double* lambdas, lm_result* out, void* stream) {
  return lm_step_impl(c, n, xy, target, 0, nullptr, n_trials, lambdas, out, stream);
}

int lm_step_split(bem_ctx* c, int64_t n, const void* xy, const void* target, int64_t n_h,
                  const void* xy_h, int n_trials, const double* lambdas, lm_result* out,
                  void* stream) {
  if (c && !xy_h) return fail(c, BEM_EINVAL, "lm_step_split: xy_h is NULL");
  return lm_step_impl(c, n, xy, target, n_h, xy_h, n_trials, lambdas, out, stream);
}

int lm_step_host(bem_ctx* c, int64_t n, const void* xy, const void* target, int n_trials,
                 const double* lambdas, lm_result* out, void* stream) {
  if (!c) return BEM_EINVAL;
  if (n <= 0 || !xy || !target) return fail(c, BEM_EINVAL, "lm_step_host: bad arguments");
  int rc;
  if ((rc = need_ready(c)) || (rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  const size_t es = c->opts.precision == BEM_FP64 ? 8 : 4;
  if ((rc = grow(c, c->hin_xy, es * 2 * (size_t)n)) || (rc = grow(c, c->hin_t, es * 3 * (size_t)n)))
    return rc;
  const int64_t chunk = gn_chunk_tc(c, n);
  const int nchunks = (int)((n + chunk - 1) / chunk);
  if (!c->hin_stream &&
      (rc = cuda_check(c, cudaStreamCreateWithFlags(&c->hin_stream, cudaStreamNonBlocking), "stream")))
    return rc;
  if (!c->hin_start &&
      ((rc = cuda_check(c, cudaEventCreateWithFlags(&c->hin_start, cudaEventDisableTiming), "event")) ||
       (rc = cuda_check(c, cudaEventCreateWithFlags(&c->hin_xy_ready, cudaEventDisableTiming), "event"))))
    return rc;
  while ((int)c->hin_t_ready.size() < nchunks) {
    cudaEvent_t e;
    if ((rc = cuda_check(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event"))) return rc;
    c->hin_t_ready.push_back(e);
  }
  // the copies start once the work queued before this call (which may still
  // read the device copies) is done: the samples first, then the targets
  // chunk by chunk, each marked by its event
  char* dxy = (char*)c->hin_xy.p;
  char* dt = (char*)c->hin_t.p;
  if ((rc = cuda_check(c, cudaEventRecord(c->hin_start, S(c)), "record")) ||
      (rc = cuda_check(c, cudaStreamWaitEvent(c->hin_stream, c->hin_start, 0), "wait")))
    return rc;
  // from here on every exit waits for the copies already issued
  rc = cuda_check(c, cudaMemcpyAsync(dxy, xy, es * 2 * (size_t)n, cudaMemcpyHostToDevice,
                                     c->hin_stream), "copy xy");
  if (!rc) rc = cuda_check(c, cudaEventRecord(c->hin_xy_ready, c->hin_stream), "record");
  for (int k = 0; !rc && k < nchunks; ++k) {
    const int64_t s0 = (int64_t)k * chunk, m = std::min<int64_t>(chunk, n - s0);
    if ((rc = cuda_check(c, cudaMemcpyAsync(dt + es * 3 * (size_t)s0, (const char*)target + es * 3 * (size_t)s0,
                                            es * 3 * (size_t)m, cudaMemcpyHostToDevice, c->hin_stream),
                         "copy target")) == BEM_OK)
      rc = cuda_check(c, cudaEventRecord(c->hin_t_ready[k], c->hin_stream), "record");
  }
  // the one-pass Gauss-Newton pass consumes the targets chunk by chunk as
  // they arrive; every other path waits for all of them first
  if (!rc) {
    c->hin_on = jtj_fuses_eval(c);
    if (!c->hin_on)
      rc = cuda_check(c, cudaStreamWaitEvent(S(c), c->hin_t_ready[nchunks - 1], 0), "wait");
  }
  if (!rc) rc = lm_step_impl(c, n, dxy, dt, 0, nullptr, n_trials, lambdas, out, stream);
  c->hin_on = false;
  // the caller may reuse its host buffers once this returns
  const int rc2 = cuda_check(c, cudaStreamSynchronize(c->hin_stream), "sync");
  return rc ? rc : rc2;
}

int bem_gemm_bf16(bem_ctx* c, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                  float* D, int ldd, void* stream) {
  if (!c) return BEM_EINVAL;
  if (M < 1 || N < 1 || K < 1 || !A || !B || !D || lda < K || ldb < K || ldd < N || lda % 8 ||
      ldb % 8)
    return fail(c, BEM_EINVAL, "bem_gemm_bf16: bad sizes or strides");
  int rc;
  if ((rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  if ((rc = cuda_check(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), S(c)), "memset"))) return rc;
  if ((rc = tc_gemm_store(c, M, N, K, A, lda, B, ldb, D, ldd))) return rc;
  int st = 0;
  if ((rc = cuda_check(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, S(c)), "status")) ||
      (rc = cuda_check(c, cudaStreamSynchronize(S(c)), "sync")))
    return rc;
  if (st) return fail(c, BEM_ETIMEDOUT, "tensor-core GEMM: a bounded device wait ran out");
  return BEM_OK;
}

int bem_fastmath_eval(bem_ctx* c, int which, int64_t n, const float* a, const float* b,
                      float* out_fast, float* out_ref, void* stream) {
  if (!c) return BEM_EINVAL;
  if (which < 0 || which > 4 || n < 0 ||
      (n > 0 && (!a || !out_fast || !out_ref || ((which == 0 || which == 3) && !b))))
    return fail(c, BEM_EINVAL, "bem_fastmath_eval: bad arguments");
  int rc;
  if ((rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  if (n > 0) {
    k_fastmath<<<(unsigned)((n + 255) / 256), 256, 0, S(c)>>>(which, n, a, b, out_fast, out_ref);
    BEM_LAUNCHED(c);
  }
  return cuda_check(c, cudaGetLastError(), "k_fastmath");
}

int bem_gram_unit(int tiles, int rows, int unit, int32_t* out) {
  if (!out) return BEM_EINVAL;
  int v[4];
  const int rc = tc_gram_unit(tiles, rows, unit, v);
  if (rc) return rc;
  for (int k = 0; k < 4; ++k) out[k] = v[k];
  return BEM_OK;
}

int bem_sizes(const bem_ctx* c, int* n_theta, int* n_panels, int* n_boundary) {
  if (!c) return BEM_EINVAL;
  if (n_theta) *n_theta = c->sc.nth;
  if (n_panels) *n_panels = c->sc.P;
  if (n_boundary) *n_boundary = c->bd.Nb;
  return BEM_OK;
}

int bem_boundary_values(bem_ctx* c, double* ub, void* stream) {
  if (!c || !ub) return c ? fail(c, BEM_EINVAL, "ub is NULL") : BEM_EINVAL;
  int rc;
  if ((rc = need_ready(c)) || (rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  if ((rc = refresh(c, c->d_theta))) return rc;
  if ((rc = cuda_check(c, cudaMemcpyAsync(ub, c->d_ub, 24 * (size_t)c->bd.Nb, cudaMemcpyDeviceToHost, S(c)), "ub")))
    return rc;
  return cuda_check(c, cudaStreamSynchronize(S(c)), "sync");
}

int64_t bem_launch_count(const bem_ctx* c) { return c ? c->launches : 0; }

int64_t bem_alloc_count(const bem_ctx* c) { return c ? c->allocs : 0; }

int bem_set_wait_limit(bem_ctx* c, double seconds) {
  if (!c) return BEM_EINVAL;
  if (!(seconds >= 0) || !(seconds <= 60))
    return fail(c, BEM_EINVAL, "bem_set_wait_limit: seconds must be in [0, 60]");
  c->wait_ns = (uint64_t)std::llround(seconds * 1e9);
  return BEM_OK;
}

int bem_gn_products(bem_ctx* c, int64_t n, const void* xy, const void* target, double* loss_out,
                    double* g_out, double* H_out, void* stream) {
  if (!c) return BEM_EINVAL;
  if (n <= 0 || !xy || !target) return fail(c, BEM_EINVAL, "bem_gn_products: bad arguments");
  int rc;
  if ((rc = need_ready(c)) || (rc = set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  const int nth = c->sc.nth;
  const size_t es = c->opts.precision == BEM_FP64 ? 8 : 4;
  const size_t nn = sizeof(double) * (size_t)nth * nth;
  if ((rc = grow(c, c->H, nn))) return rc;
  const size_t roff = ((es * 3 * (size_t)n + 255) / 256) * 256;
  if ((rc = grow(c, c->phi, roff + 8 * (size_t)nth * 2 + 64))) return rc;
  double* g = (double*)((char*)c->phi.p + roff);
  if ((rc = refresh(c, c->d_theta))) return rc;
  double s0 = 0;
  if ((rc = gn_at_theta(c, n, xy, target, 0, nullptr, c->phi.p, g, (double*)c->H.p, &s0))) return rc;
  if (g_out &&
      (rc = cuda_check(c, cudaMemcpyAsync(g_out, g, 8 * (size_t)nth, cudaMemcpyDeviceToDevice, S(c)), "g")))
    return rc;
  if (H_out && (rc = cuda_check(c, cudaMemcpyAsync(H_out, c->H.p, nn, cudaMemcpyDeviceToDevice, S(c)), "H")))
    return rc;
  if ((rc = cuda_check(c, cudaStreamSynchronize(S(c)), "sync"))) return rc;
  if (loss_out) *loss_out = 0.5 * s0 / double(n);
  return BEM_OK;
}

int bem_profile_enable(bem_ctx* c, int on) {
  if (!c) return BEM_EINVAL;
  if (set_device(c)) return BEM_ECUDA;
  prof_resolve(c);
  c->prof_tot.clear();
  c->prof = on != 0;
  return BEM_OK;
}

int bem_profile_read(bem_ctx* c, int max_entries, char* names, double* total_ms, int64_t* counts,
                     int* n_entries) {
  if (!c || max_entries < 0 || !n_entries) return c ? fail(c, BEM_EINVAL, "bad arguments") : BEM_EINVAL;
  if (set_device(c)) return BEM_ECUDA;
  prof_resolve(c);
  int k = 0;
  for (auto& kv : c->prof_tot) {
    if (k >= max_entries) break;
    if (names) {
      strncpy(names + 32 * k, kv.first.c_str(), 31);
      names[32 * k + 31] = 0;
    }
    if (total_ms) total_ms[k] = kv.second.first;
    if (counts) counts[k] = kv.second.second;
    ++k;
  }
  *n_entries = k;
  return BEM_OK;
}

}  // extern "C"
