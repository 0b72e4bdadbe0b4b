// Batched LM iterations of many scenes of uneven size, several damping
// trials per scene (the batching part of the method's throughput study).
//
// One call steps every scene once, as lm_step does for a single scene
// (Sec. 4.3, Eq. (optimstep)):
//   A  per scene: panels, compatibility weights and boundary solution at
//      theta, double near-field sums at the samples;
//   A' one persistent launch over the sample tiles of all scenes: colours,
//      residuals and loss partials (k_field_batch_f32);
//   B  per scene: H and g = (1/n) J^T r from the J rows (tensor cores);
//   C  per scene and trial: the damped KKT solve, theta_t = theta + delta,
//      projection, panels, boundary solution and near sums of theta_t.
//   The scenes are independent in B and C, so each scene runs them on its
//      own stream, right after one another, driven by one of eight host
//      threads (worker w takes scenes w, w + 8, ...): the passes and the
//      chains of small, latency-bound kernels with host checks (the solves'
//      refinement) of different scenes overlap on the GPU;
//   D  one persistent launch over the sample tiles of all scenes: the trial
//      losses, the (up to four) trials of a scene on the same tile so that
//      they share the boundary angles of its points, which do not depend on
//      the handles;
//   E  per scene: the best trial is kept if it lowers the loss.
// The two persistent launches (with their counter reset and loss sums) are
// captured once into CUDA graphs and replayed: the job tables they read live
// in device memory and are rewritten per call.  On the first call a small
// autotuner times the tile shapes (128 or 256 points per tile) and CTAs per
// SM on the real job list and keeps the fastest.
//
// The batch runs on an internal stream (and, in B and C, one stream per
// scene), ordered after the caller's stream and before its next work; in B
// the Gauss-Newton chunk buffers of scene w serve the scenes of worker w.
#include <algorithm>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "ctx.h"

namespace bem {

// sums[j nt + t] = sum over the tiles of job j of part[t total + tile] (fixed
// order, one block per job and trial, blockIdx.y = trial)
__global__ void k_job_sums(const double* __restrict__ part, const BatchJob* __restrict__ jobs,
                           int njobs, const int64_t* __restrict__ total, double* __restrict__ sums) {
  __shared__ double red[32];
  const int j = blockIdx.x, t = blockIdx.y;
  part += (size_t)t * *total;
  const int64_t b = jobs[j].tile0, e = j + 1 < njobs ? jobs[j + 1].tile0 : *total;
  double s = 0.0;
  const int64_t m = e - b;
  const int64_t per = (m + blockDim.x - 1) / blockDim.x;
  const int64_t k0 = b + threadIdx.x * per, k1 = min(e, k0 + per);
  for (int64_t k = k0; k < k1; ++k) s += part[k];
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += red[w];
    sums[(size_t)j * gridDim.y + t] = acc;
  }
}

}  // namespace bem

using namespace bem;

struct bem_batch {
  std::vector<bem_ctx*> sc;
  bem_ctx* c0 = nullptr;                 // errors, device, shared chunk buffers
  cudaStream_t st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<cudaStream_t> sst;         // [S] the scenes' streams of phase C
  std::vector<cudaEvent_t> sev;          // [S] their ends
  cudaEvent_t ev_b = nullptr;            // end of phase B
  int T = 0;                             // trials the buffers are sized for
  std::vector<int64_t> n;                // samples the buffers are sized for
  std::vector<DevBuf> resid;             // [S] float [n][3]
  std::vector<DevBuf> nearb;             // [S (T+1)] double [n][3]: theta, trials
  std::vector<DevBuf> tpan, tub, ttheta; // [S T] trial panels, boundary solution, theta
  std::vector<DevBuf> gvec;              // [S] gradient
  DevBuf jobs[2], part[2], sums[2], counter[2], total[2], gn2;
  std::vector<BatchJob> hjobs[2];
  std::vector<int64_t> htotal;
  int spt = 1, bps = 8;
  int nt[2] = {1, 1};                    // trials per job of each job table
  bool tuned = false;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_njobs[2] = {-1, -1};
};

namespace {

void drop_graphs(bem_batch* b) {
  for (int k = 0; k < 2; ++k) {
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    b->graph[k] = nullptr;
    b->graph_njobs[k] = -1;
  }
}

void free_dev(DevBuf& d) {
  if (d.p) cudaFree(d.p);
  d.p = nullptr;
  d.cap = 0;
}

// tile list of the job table k: tile0 of each job for tiles of 128 * spt points
void number_tiles(bem_batch* b, int k, int spt) {
  int64_t t = 0;
  for (auto& j : b->hjobs[k]) {
    j.tile0 = t;
    const int64_t per = 128 * (int64_t)spt;
    t += (j.a.n + per - 1) / per;
  }
  b->htotal[k] = t;
}

// point every job's loss partials at its tiles (trial t of a multi-trial
// job: the t-th block of htotal partials)
void bind_partials(bem_batch* b, int k) {
  double* part = (double*)b->part[k].p;
  for (auto& j : b->hjobs[k]) {
    j.a.loss_part = part + j.tile0;
    for (int t = 0; t < j.nt && j.nt > 1; ++t) j.tloss[t] = part + (size_t)t * b->htotal[k] + j.tile0;
  }
}

int upload(bem_batch* b, int k) {
  bem_ctx* c = b->c0;
  const size_t bytes = sizeof(BatchJob) * b->hjobs[k].size();
  int rc;
  if ((rc = cuda_check(c, cudaMemcpyAsync(b->jobs[k].p, b->hjobs[k].data(), bytes,
                                          cudaMemcpyHostToDevice, b->st), "jobs")) ||
      (rc = cuda_check(c, cudaMemcpyAsync(b->total[k].p, &b->htotal[k], sizeof(int64_t),
                                          cudaMemcpyHostToDevice, b->st), "jobs")))
    return rc;
  // the host copies must outlive the asynchronous copies
  return cuda_check(c, cudaStreamSynchronize(b->st), "jobs");
}

int run_eval(bem_batch* b, int k) {
  bem_ctx* c = b->c0;
  const int nj = (int)b->hjobs[k].size();
  int rc;
  if ((rc = field_batch_launch(c, (const BatchJob*)b->jobs[k].p, nj, (const int64_t*)b->total[k].p,
                               (unsigned long long*)b->counter[k].p, b->spt, b->bps, b->nt[k])))
    return rc;
  k_job_sums<<<dim3(nj, b->nt[k]), 256, 0, b->st>>>((const double*)b->part[k].p,
                                                    (const BatchJob*)b->jobs[k].p, nj,
                                                    (const int64_t*)b->total[k].p,
                                                    (double*)b->sums[k].p);
  BEM_LAUNCHED(c);
  return cuda_check(c, cudaGetLastError(), "k_job_sums");
}

// evaluate job table k through its captured graph (captured on first use)
int eval_graph(bem_batch* b, int k) {
  bem_ctx* c = b->c0;
  const int nj = (int)b->hjobs[k].size();
  int rc;
  if (!b->graph[k] || b->graph_njobs[k] != nj) {
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    b->graph[k] = nullptr;
    cudaGraph_t g = nullptr;
    if ((rc = cuda_check(c, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal), "capture")))
      return rc;
    rc = run_eval(b, k);
    cudaError_t e = cudaStreamEndCapture(b->st, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if ((rc = cuda_check(c, e, "capture"))) return rc;
    e = cudaGraphInstantiate(&b->graph[k], g, 0);
    cudaGraphDestroy(g);
    if ((rc = cuda_check(c, e, "graph instantiate"))) return rc;
    b->graph_njobs[k] = nj;
  }
  ProfScope _ps(c, "k_field_batch");   // c->cur is b->st outside the per-scene phase
  return cuda_check(c, cudaGraphLaunch(b->graph[k], b->st), "graph launch");
}

// time the candidate tile shapes on job table k (idempotent) and keep the fastest
int autotune(bem_batch* b, int k) {
  bem_ctx* c = b->c0;
  const int spts[2] = {1, 2};
  const int bpss[3] = {4, 8, 12};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = INFINITY;
  int bs = 1, bb = 8, rc = BEM_OK;
  for (int spt : spts) {
    number_tiles(b, k, spt);
    bind_partials(b, k);
    if ((rc = upload(b, k))) break;
    b->spt = spt;
    for (int bps : bpss) {
      b->bps = bps;
      if ((rc = run_eval(b, k))) break;           // warm
      cudaEventRecord(e0, b->st);
      if ((rc = run_eval(b, k))) break;
      cudaEventRecord(e1, b->st);
      if ((rc = cuda_check(c, cudaEventSynchronize(e1), "autotune"))) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bs = spt; bb = bps; }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->spt = bs;
  b->bps = bb;
  b->tuned = true;
  return BEM_OK;
}

int size_buffers(bem_batch* b, const int64_t* n, int T) {
  bem_ctx* c = b->c0;
  const int S = (int)b->sc.size();
  bool same = T == b->T;
  for (int s = 0; s < S && same; ++s) same = n[s] == b->n[s];
  if (same) return BEM_OK;
  drop_graphs(b);
  b->T = T;
  b->n.assign(n, n + S);
  b->resid.resize(S);
  b->gvec.resize(S);
  b->nearb.resize((size_t)S * (T + 1));
  b->tpan.resize((size_t)S * T);
  b->tub.resize((size_t)S * T);
  b->ttheta.resize((size_t)S * T);
  int rc;
  int64_t tiles = 0;
  for (int s = 0; s < S; ++s) {
    bem_ctx* cs = b->sc[s];
    if ((rc = grow(c, b->resid[s], sizeof(float) * 3 * (size_t)n[s])) ||
        (rc = grow(c, b->gvec[s], sizeof(double) * (size_t)cs->sc.nth)))
      return rc;
    if (cs->opts.near_factor > 0)
      for (int t = 0; t <= T; ++t)
        if ((rc = grow(c, b->nearb[(size_t)s * (T + 1) + t], sizeof(double) * 3 * (size_t)n[s])))
          return rc;
    for (int t = 0; t < T; ++t) {
      const size_t i = (size_t)s * T + t;
      if ((rc = grow(c, b->tpan[i], sizeof(Panel<float>) * (size_t)cs->sc.P)) ||
          (rc = grow(c, b->tub[i], sizeof(double) * 3 * (size_t)cs->bd.Nb)) ||
          (rc = grow(c, b->ttheta[i], sizeof(double) * (size_t)cs->sc.nth)))
        return rc;
    }
    tiles += (n[s] + 127) / 128;
  }
  for (int k = 0; k < 2; ++k) {
    const int nj = k == 0 ? S : S * T;
    const int64_t pt = k == 0 ? tiles : tiles * T;
    if ((rc = grow(c, b->jobs[k], sizeof(BatchJob) * (size_t)nj)) ||
        (rc = grow(c, b->part[k], sizeof(double) * (size_t)(pt + 1))) ||
        (rc = grow(c, b->sums[k], sizeof(double) * (size_t)nj)) ||
        (rc = grow(c, b->counter[k], sizeof(unsigned long long))) ||
        (rc = grow(c, b->total[k], sizeof(int64_t))))
      return rc;
  }
  return grow(c, b->gn2, sizeof(double) * (size_t)S);
}

// the evaluation job of scene s with its current device state
BatchJob scene_job(bem_ctx* cs, int64_t n, const void* xy, const void* target) {
  BatchJob j{};
  j.nt = 1;
  j.a = field_args_f32(cs);
  j.a.xy = (const float*)xy;
  j.a.n = n;
  j.a.ub = cs->d_ub;
  j.a.mean0 = cs->mean[0];
  j.a.mean1 = cs->mean[1];
  j.a.mean2 = cs->mean[2];
  j.a.target = (const float*)target;
  return j;
}

int batch_lm(bem_batch* b, const int64_t* n, const void* const* xy, const void* const* target,
             int T, const double* lambdas, lm_result* out) {
  const int S = (int)b->sc.size();
  bem_ctx* c0 = b->c0;
  int rc;
  if ((rc = size_buffers(b, n, T))) return rc;
  // ---- A: state at theta, near sums at the samples.  A scene whose
  // residual comes out of its J-row pass (jtj_fuses_eval) gets no tiles here.
  b->hjobs[0].resize(S);
  bool any_eval = false;
  for (int s = 0; s < S; ++s) {
    bem_ctx* c = b->sc[s];
    if ((rc = ctx_refresh(c, c->d_theta)) || (rc = geom_compat(c, c->d_theta, false))) return rc;
    const bool fused = jtj_fuses_eval(c);
    double* nb = nullptr;
    if (!fused && c->opts.near_factor > 0) {
      nb = (double*)b->nearb[(size_t)s * (T + 1)].p;
      if ((rc = near_forward(c, n[s], (const float*)xy[s], nb))) return rc;
    }
    BatchJob j = scene_job(c, n[s], xy[s], target[s]);
    j.a.near_add = nb;
    j.a.resid = (float*)b->resid[s].p;
    if (fused) j.a.n = 0;
    any_eval = any_eval || !fused;
    b->hjobs[0][s] = j;
  }
  // ---- A': one persistent launch over the scenes evaluated here (the tile
  // shape is tuned once, on the first job table with work)
  if (any_eval && !b->tuned && (rc = autotune(b, 0))) return rc;
  number_tiles(b, 0, b->spt);
  bind_partials(b, 0);
  if ((rc = upload(b, 0)) || (rc = eval_graph(b, 0))) return rc;
  // ---- B: H and g per scene, the scenes on their own streams (after phase
  // A) from several host threads, each scene's trials (phase C) right after
  // its pass.  Worker w takes the scenes w, w + K, ... one after another and
  // lends them scene w's chunk buffers (the J-row pass ends with a
  // synchronisation of the scene's stream, so a worker's scenes never use
  // those buffers at the same time; the trials use none of them).
  if ((rc = cuda_check(c0, cudaEventRecord(b->ev_b, b->st), "event"))) return rc;
  for (int s = 0; s < S; ++s)
    if ((rc = cuda_check(c0, cudaStreamWaitEvent(b->sst[s], b->ev_b, 0), "event"))) return rc;
  std::vector<int> brc(S, BEM_OK);
  const int nworkers = std::min(S, 8);
  auto scene_gn = [&](int s, int w) -> int {
    int rc = BEM_OK;
    bem_ctx* c = b->sc[s];
    c->cur = b->sst[s];
    c->scratch = s == w ? nullptr : b->sc[w];
    const int nth = c->sc.nth;
    double* g = (double*)b->gvec[s].p;
    if ((rc = grow(c, c->H, sizeof(double) * (size_t)nth * nth))) return rc;
    if (jtj_fuses_eval(c)) {
      // residual, loss sum, g and H from one pass; the loss sum joins the others
      if ((rc = jtj_build(c, n[s], xy[s], (double*)c->H.p, b->resid[s].p, g, target[s])) ||
          (rc = cuda_check(c, cudaMemcpyAsync((double*)b->sums[0].p + s, c->d_scal, sizeof(double),
                                              cudaMemcpyDeviceToDevice, c->cur), "loss")))
        return rc;
      ctx_scale_norm(c, g, nth, 1.0, (double*)b->gn2.p + s);
    } else if (jtj_gives_gradient(c)) {
      if ((rc = jtj_build(c, n[s], xy[s], (double*)c->H.p, b->resid[s].p, g))) return rc;
      ctx_scale_norm(c, g, nth, 1.0, (double*)b->gn2.p + s);
    } else {
      if ((rc = adj_vjp(c, n[s], xy[s], b->resid[s].p, g))) return rc;
      ctx_scale_norm(c, g, nth, 1.0 / double(n[s]), (double*)b->gn2.p + s);
      if ((rc = jtj_build(c, n[s], xy[s], (double*)c->H.p))) return rc;
    }
    return rc;
  };
  // ---- C, in the same workers: each scene's trials (damped solves, trial
  // geometry, boundary values and near-field sums) on its stream right after
  // its Gauss-Newton pass, so that they overlap the other scenes' passes
  std::vector<double> used((size_t)S * T, 0.0);
  std::vector<char> ok((size_t)S * T, 0);
  std::vector<BatchJob> trial_jobs((size_t)S * T);
  auto scene_trials = [&](int s) -> int {
    int rc = BEM_OK;
    bem_ctx* c = b->sc[s];
    c->cur = b->sst[s];
    const int nth = c->sc.nth;
    const double* g = (const double*)b->gvec[s].p;
    for (int t = 0; t < T; ++t) {
      const size_t i = (size_t)s * T + t;
      double lam = lambdas[t];
      for (int r = 0;; ++r) {
        rc = la_lm_solve(c, (const double*)c->H.p, g, lam, c->d_delta);
        if (rc != BEM_ENOTSPD || r == 12) break;
        lam = lam > 0 ? 10.0 * lam : 1e-9;
      }
      used[i] = lam;
      BatchJob j{};
      if (rc == BEM_ENOTSPD) {
        j.a.n = 0;                   // no tiles; the trial is skipped
        trial_jobs[i] = j;
        rc = BEM_OK;
        continue;
      }
      if (rc) return rc;
      ok[i] = 1;
      double* th = (double*)b->ttheta[i].p;
      ctx_axpy(c, c->d_theta, c->d_delta, nth, th);
      if ((rc = geom_panelize(c, th)) || (rc = geom_compat(c, th, true)) ||
          (rc = ctx_refresh(c, th)))
        return rc;
      if ((rc = cuda_check(c, cudaMemcpyAsync(b->tpan[i].p, c->d_pan32,
                                              sizeof(Panel<float>) * (size_t)c->sc.P,
                                              cudaMemcpyDeviceToDevice, c->cur), "trial panels")) ||
          (rc = cuda_check(c, cudaMemcpyAsync(b->tub[i].p, c->d_ub, sizeof(double) * 3 * c->bd.Nb,
                                              cudaMemcpyDeviceToDevice, c->cur), "trial ub")))
        return rc;
      j = scene_job(c, n[s], xy[s], target[s]);
      j.a.pan = (const Panel<float>*)b->tpan[i].p;
      j.a.ub = (const double*)b->tub[i].p;
      if (c->opts.near_factor > 0) {
        double* nb = (double*)b->nearb[(size_t)s * (T + 1) + 1 + t].p;
        if ((rc = near_forward(c, n[s], (const float*)xy[s], nb))) return rc;
        j.a.near_add = nb;
      }
      trial_jobs[i] = j;
    }
    return rc;
  };
  {
    auto worker = [&](int w) {
      // the runtime's current device is per host thread
      if (cudaSetDevice(c0->device) != cudaSuccess) {
        for (int s = w; s < S; s += nworkers) brc[s] = BEM_ECUDA;
        return;
      }
      for (int s = w; s < S; s += nworkers) {
        brc[s] = scene_gn(s, w);
        if (brc[s] == BEM_OK) brc[s] = scene_trials(s);
      }
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < nworkers; ++w) pool.emplace_back(worker, w);
    worker(0);
    for (auto& th : pool) th.join();
  }
  for (int s = 0; s < S; ++s) {
    bem_ctx* c = b->sc[s];
    c->cur = b->st;
    c->scratch = s == 0 ? nullptr : c0;
    cudaEventRecord(b->sev[s], b->sst[s]);
    cudaStreamWaitEvent(b->st, b->sev[s], 0);
  }
  for (int s = 0; s < S; ++s)
    if (brc[s]) return brc[s];
  std::vector<double> L0(S), gn2(S);
  if ((rc = cuda_check(c0, cudaMemcpyAsync(L0.data(), b->sums[0].p, sizeof(double) * S,
                                           cudaMemcpyDeviceToHost, b->st), "loss")) ||
      (rc = cuda_check(c0, cudaMemcpyAsync(gn2.data(), b->gn2.p, sizeof(double) * S,
                                           cudaMemcpyDeviceToHost, b->st), "norm")) ||
      (rc = cuda_check(c0, cudaStreamSynchronize(b->st), "sync")))
    return rc;
  // ---- D: one persistent launch over all scenes and trials: with 2 to
  // kJobTrials trials one job per scene evaluates them all (a skipped
  // trial points at a factored one's data; its loss is not used), else one
  // job per (scene, trial)
  b->nt[1] = (T >= 2 && T <= kJobTrials) ? T : 1;
  if (b->nt[1] > 1) {
    b->hjobs[1].assign(S, BatchJob{});
    for (int s = 0; s < S; ++s) {
      int first = -1;
      for (int t = 0; t < T && first < 0; ++t)
        if (ok[(size_t)s * T + t]) first = t;
      BatchJob& j = b->hjobs[1][s];
      if (first < 0) {               // no trial factored: no tiles (reported below)
        j.a.n = 0;
        j.nt = T;
        continue;
      }
      j = trial_jobs[(size_t)s * T + first];
      j.nt = T;
      for (int t = 0; t < T; ++t) {
        const BatchJob& tj = trial_jobs[(size_t)s * T + (ok[(size_t)s * T + t] ? t : first)];
        j.tpan[t] = tj.a.pan;
        j.tub[t] = tj.a.ub;
        j.tnear[t] = tj.a.near_add;
      }
    }
  } else {
    b->hjobs[1] = trial_jobs;
    for (auto& j : b->hjobs[1]) j.nt = 1;
  }
  if (!b->tuned && (rc = autotune(b, 1))) return rc;
  number_tiles(b, 1, b->spt);
  bind_partials(b, 1);
  if ((rc = upload(b, 1)) || (rc = eval_graph(b, 1))) return rc;
  std::vector<double> L1((size_t)S * T);
  if ((rc = cuda_check(c0, cudaMemcpyAsync(L1.data(), b->sums[1].p, sizeof(double) * S * T,
                                           cudaMemcpyDeviceToHost, b->st), "loss")) ||
      (rc = cuda_check(c0, cudaStreamSynchronize(b->st), "sync")))
    return rc;
  // ---- E: the best trial per scene, damping update as lm_step
  for (int s = 0; s < S; ++s) {
    bem_ctx* c = b->sc[s];
    lm_result& o = out[s];
    const double l0 = 0.5 * L0[s] / double(n[s]);
    double best = INFINITY;
    int bt = -1;
    bool any = false;
    for (int t = 0; t < T; ++t) {
      const size_t i = (size_t)s * T + t;
      if (!ok[i]) continue;
      any = true;
      const double l1 = 0.5 * L1[i] / double(n[s]);
      if (l1 < best) { best = l1; bt = t; }
    }
    if (!any) return fail(c0, BEM_ENOTSPD, "LM matrix not positive definite for any trial lambda");
    o.loss_before = l0;
    o.loss_after = best;
    o.accepted = best < l0 ? 1 : 0;
    o.best_trial = o.accepted ? bt : -1;
    o.grad_norm = std::sqrt(gn2[s]);
    if (o.accepted) {
      if ((rc = cuda_check(c, cudaMemcpyAsync(c->d_theta, b->ttheta[(size_t)s * T + bt].p,
                                              sizeof(double) * c->sc.nth, cudaMemcpyDeviceToDevice,
                                              b->st), "theta")))
        return rc;
      o.lambda_next = used[(size_t)s * T + bt] / 3.0;
    } else {
      double mx = 0;
      for (int t = 0; t < T; ++t) mx = std::fmax(mx, used[(size_t)s * T + t]);
      o.lambda_next = T == 1 ? 2.0 * used[(size_t)s * T] : 10.0 * mx;
    }
  }
  return BEM_OK;
}

}  // namespace

extern "C" {

int bem_batch_create(bem_batch** out, bem_ctx* const* scenes, int n_scenes) {
  if (!out) return BEM_EINVAL;
  *out = nullptr;
  if (!scenes || n_scenes < 1) return BEM_EINVAL;
  bem_ctx* c0 = scenes[0];
  if (!c0) return BEM_EINVAL;
  for (int s = 0; s < n_scenes; ++s) {
    bem_ctx* c = scenes[s];
    if (!c) return fail(c0, BEM_EINVAL, "bem_batch_create: NULL scene");
    int rc;
    if ((rc = ctx_ready(c))) return fail(c0, rc, "bem_batch_create: scene not set up and factored");
    if (c->opts.precision != BEM_MIXED)
      return fail(c0, BEM_EINVAL, "bem_batch_create: scenes must be BEM_MIXED contexts");
    if (c->device != c0->device || c->opts.eps_c != c0->opts.eps_c ||
        c->opts.eps_d != c0->opts.eps_d || (c->opts.near_factor > 0) != (c0->opts.near_factor > 0))
      return fail(c0, BEM_EINVAL,
                  "bem_batch_create: scenes must share device, eps_c, eps_d and near-field use");
    for (int r = 0; r < s; ++r)
      if (scenes[r] == c) return fail(c0, BEM_EINVAL, "bem_batch_create: a scene appears twice");
  }
  int rc;
  if ((rc = ctx_set_device(c0))) return rc;
  bem_batch* b = new (std::nothrow) bem_batch;
  if (!b) return fail(c0, BEM_ENOMEM, "bem_batch_create: out of host memory");
  b->sc.assign(scenes, scenes + n_scenes);
  b->c0 = c0;
  b->htotal.assign(2, 0);
  if ((rc = cuda_check(c0, cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking), "stream")) ||
      (rc = cuda_check(c0, cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming), "event")) ||
      (rc = cuda_check(c0, cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming), "event")) ||
      (rc = cuda_check(c0, cudaEventCreateWithFlags(&b->ev_b, cudaEventDisableTiming), "event"))) {
    bem_batch_destroy(b);
    return rc;
  }
  b->sst.assign(n_scenes, nullptr);
  b->sev.assign(n_scenes, nullptr);
  for (int s = 0; s < n_scenes; ++s)
    if ((rc = cuda_check(c0, cudaStreamCreateWithFlags(&b->sst[s], cudaStreamNonBlocking), "stream")) ||
        (rc = cuda_check(c0, cudaEventCreateWithFlags(&b->sev[s], cudaEventDisableTiming), "event"))) {
      bem_batch_destroy(b);
      return rc;
    }
  *out = b;
  return BEM_OK;
}

void bem_batch_destroy(bem_batch* b) {
  if (!b) return;
  cudaSetDevice(b->c0->device);
  if (b->st) cudaStreamSynchronize(b->st);
  drop_graphs(b);
  for (auto* v : {&b->resid, &b->nearb, &b->tpan, &b->tub, &b->ttheta, &b->gvec})
    for (auto& d : *v) free_dev(d);
  for (int k = 0; k < 2; ++k) {
    free_dev(b->jobs[k]);
    free_dev(b->part[k]);
    free_dev(b->sums[k]);
    free_dev(b->counter[k]);
    free_dev(b->total[k]);
  }
  free_dev(b->gn2);
  for (bem_ctx* c : b->sc) c->scratch = nullptr;
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->ev_b) cudaEventDestroy(b->ev_b);
  for (cudaStream_t st : b->sst)
    if (st) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
  for (cudaEvent_t e : b->sev)
    if (e) cudaEventDestroy(e);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

int bem_batch_lm(bem_batch* b, const int64_t* n, const void* const* xy, const void* const* target,
                 int n_trials, const double* lambdas, lm_result* out, void* stream) {
  if (!b) return BEM_EINVAL;
  bem_ctx* c0 = b->c0;
  const int S = (int)b->sc.size();
  if (!n || !xy || !target || !out || !lambdas || n_trials < 1 || n_trials > 16)
    return fail(c0, BEM_EINVAL, "bem_batch_lm: bad arguments");
  for (int t = 0; t < n_trials; ++t)
    if (!(lambdas[t] >= 0) || !std::isfinite(lambdas[t]))
      return fail(c0, BEM_EINVAL, "bem_batch_lm: lambda must be finite and >= 0");
  for (int s = 0; s < S; ++s) {
    if (n[s] <= 0 || !xy[s] || !target[s])
      return fail(c0, BEM_EINVAL, "bem_batch_lm: every scene needs samples and targets");
    if (reg_active(b->sc[s]))
      return fail(c0, BEM_EINVAL, "bem_batch_lm: regularisers are applied by lm_step only");
  }
  int rc;
  if ((rc = ctx_set_device(c0))) return rc;
  // order after the caller's stream
  if ((rc = cuda_check(c0, cudaEventRecord(b->ev_in, (cudaStream_t)stream), "event")) ||
      (rc = cuda_check(c0, cudaStreamWaitEvent(b->st, b->ev_in, 0), "event")))
    return rc;
  for (int s = 0; s < S; ++s) {
    b->sc[s]->cur = b->st;
    b->sc[s]->scratch = s == 0 ? nullptr : c0;
    b->sc[s]->err.clear();
  }
  rc = batch_lm(b, n, xy, target, n_trials, lambdas, out);
  // the caller's stream continues after the batch's work
  cudaEventRecord(b->ev_out, b->st);
  cudaStreamWaitEvent((cudaStream_t)stream, b->ev_out, 0);
  if (rc) {
    // a failing scene reports into its own context; surface it on scene 0
    for (int s = 0; s < S; ++s)
      if (b->sc[s] != c0 && !b->sc[s]->err.empty()) {
        c0->err = "bem_batch_lm: scene " + std::to_string(s) + ": " + b->sc[s]->err;
        break;
      }
    return rc;
  }
  return cuda_check(c0, cudaStreamSynchronize(b->st), "sync");
}

int bem_batch_tile_shape(const bem_batch* b, int* points_per_tile, int* ctas_per_sm) {
  if (!b) return BEM_EINVAL;
  if (points_per_tile) *points_per_tile = b->tuned ? 128 * b->spt : 0;
  if (ctas_per_sm) *ctas_per_sm = b->tuned ? b->bps : 0;
  return BEM_OK;
}

}  // extern "C"
