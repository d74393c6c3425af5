// Entry points outside geo_step: measurement probes and the prism-zone predictor.
#pragma once
#include <cuda_runtime.h>

namespace geo {
// The predictor's derivative contraction alone (probe_contract.inc).
cudaError_t probe_contraction_any(int order, int tensor, long long Z, int reps, cudaStream_t st, float* out,
                                  float* ms);
// The ADER-CG predictor on the paper's prism zones (prism.inc).
cudaError_t launch_prism_predictor_any(int p, long long Z, const double* D, const double* R, const double* X,
                                       const double* U, double dt, double gam, double* Uh, cudaStream_t st);
}  // namespace geo
