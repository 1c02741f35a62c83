// Evaluation kernels of the L2-staged path (not part of a frame step).
#pragma once

#include <cuda_runtime.h>

namespace ddh {

// Strehl ratio of a stream on the L2-staged path (512 x 512): a row pass and a column pass
// through an N x N complex scratch image; the maximum of |.|^2 is gathered as float bits.
struct StrehlL2Args {
  const float* phi_est;
  const float* phi_true;
  float2* work;        // N x N complex scratch, row-major (the pupil rows after the row pass)
  unsigned* max_bits;  // running maximum of |.|^2 (a non-negative float's bits); zero on entry
  const float2* tw;    // tw[t] = exp(-2 pi i t / N)
  int ap_lim;
};

cudaError_t launch_strehl_l2(int n, const StrehlL2Args& a, cudaStream_t st);  // n = 512

}  // namespace ddh
