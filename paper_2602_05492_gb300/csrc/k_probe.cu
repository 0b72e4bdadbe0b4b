// Throughput probes of the SM pipes the float pair kernels issue to: the
// fused multiply-add pipe (FP32) and the multi-function unit (MUFU: base-2
// logarithm, reciprocal, reciprocal square root).  They give the measured
// denominators of those kernels' roofline.  Each thread runs eight
// independent dependency chains of the probed operation, so that every SM
// has far more independent work in flight than the pipe's latency needs;
// the chains stay in a fixed numerical range (x <- a x + b with |a| < 1,
// x <- lg2 x + 2, x <- 1/x + 1, x <- 1/sqrt(x) + 1), and one improbable
// comparison keeps them from being removed.
#include <algorithm>
#include <vector>

#include "ctx.h"

namespace bem {

template <int WHICH>
__global__ void __launch_bounds__(256) k_pipe_probe(int iters, float a, float b, float* sink) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = 1.5f + 0.125f * i + 1e-6f * (float)threadIdx.x;
  // 16 x 8 operations per trip of the loop: its counter and branch cost
  // under 2 % of the issue slots
#pragma unroll 16
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if constexpr (WHICH == 0) x[i] = fmaf(x[i], a, b);
      else if constexpr (WHICH == 1) x[i] = mufu_lg2(x[i]) + b;
      else if constexpr (WHICH == 2) x[i] = mufu_rcp(x[i]) + b;
      else x[i] = mufu_rsqrt(x[i]) + b;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 1234.5f) sink[blockIdx.x] = s;
}

}  // namespace bem

using namespace bem;

extern "C" int bem_pipe_peak(bem_ctx* c, int which, int launches, double* ops_per_s,
                             void* stream) {
  if (!c) return BEM_EINVAL;
  if (which < 0 || which > 3 || launches < 1 || launches > 1000 || !ops_per_s)
    return fail(c, BEM_EINVAL, "bem_pipe_peak: bad arguments");
  int rc;
  if ((rc = ctx_set_device(c))) return rc;
  c->cur = (cudaStream_t)stream;
  // about 30 ms per launch at the nominal rates (FP32: 128 lanes per SM,
  // MUFU: 16), four CTAs of 256 threads per SM
  const int iters = which == 0 ? 1000000 : 100000;
  const unsigned grid = (unsigned)(4 * c->sms);
  if ((rc = grow(c, c->rend, sizeof(float) * grid))) return rc;
  float* sink = (float*)c->rend.p;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((rc = cuda_check(c, cudaEventCreate(&e0), "event")) ||
      (rc = cuda_check(c, cudaEventCreate(&e1), "event")))
    return rc;
  auto launch = [&]() {
    switch (which) {
      case 0: k_pipe_probe<0><<<grid, 256, 0, S(c)>>>(iters, 0.999f, 1e-3f, sink); break;
      case 1: k_pipe_probe<1><<<grid, 256, 0, S(c)>>>(iters, 0.f, 2.f, sink); break;
      case 2: k_pipe_probe<2><<<grid, 256, 0, S(c)>>>(iters, 0.f, 1.f, sink); break;
      default: k_pipe_probe<3><<<grid, 256, 0, S(c)>>>(iters, 0.f, 1.f, sink); break;
    }
    BEM_LAUNCHED(c);
  };
  launch();   // warm-up
  std::vector<double> rates;
  for (int k = 0; k < launches && rc == BEM_OK; ++k) {
    cudaEventRecord(e0, S(c));
    launch();
    cudaEventRecord(e1, S(c));
    if ((rc = cuda_check(c, cudaEventSynchronize(e1), "probe"))) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double ops = (double)grid * 256.0 * (double)iters * 8.0;
    rates.push_back(ops / (ms * 1e-3));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if ((rc = cuda_check(c, cudaGetLastError(), "k_pipe_probe"))) return rc;
  std::sort(rates.begin(), rates.end());
  *ops_per_s = rates[rates.size() / 2];
  return BEM_OK;
}
