// Arguments of the field kernels (k_field.cu) and the job record of the
// batched evaluation.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace bem {

template <typename T>
struct FieldArgs {
  const T* xy;
  int64_t n;
  const Panel<T>* pan;
  const Panel<double>* pan64;
  int P;
  int pchunk;          // panels per blockIdx.y slice (split mode)
  const T* vert;       // boundary vertices [(Nb+1)][2] or null
  const double* ub;    // boundary solution [Nb][3] or null
  int Nb;
  double mean0, mean1, mean2;
  T ec2, ed2;          // eps_c^2, eps_d^2
  double ec2d, ed2d;
  T near2;             // (near_factor)^2, mixed precision only
  float nfac;          // near_factor, mixed precision only
  const T* target;     // clamp target or null
  T* out;              // colours [n][3] or null
  T* resid;            // residual [n][3] or null
  double* loss_part;   // per-block sum of |r|^2 or null
  double* split_out;   // split mode: [gridDim.y][n][3] handle-term partials
  const double* near_add;  // double near-field sum [n][3] or null
};

// Most damping trials one job of the batched evaluation takes at once.
constexpr int kJobTrials = 4;

// One job of the batched evaluation, its tiles numbered from tile0 in the
// batch's tile list: a scene at one parameter vector (a), or, in the trial
// launch, a scene at nt trial parameter vectors, their panels, boundary
// solutions, double near-field sums and loss partials (per tile) given per
// trial.
struct BatchJob {
  FieldArgs<float> a;
  int64_t tile0;
  int nt;
  const Panel<float>* tpan[kJobTrials];
  const double* tub[kJobTrials];
  const double* tnear[kJobTrials];
  double* tloss[kJobTrials];
};

}  // namespace bem
