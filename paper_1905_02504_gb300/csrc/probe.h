// Measurement probes of the library (not on the step's path).
#pragma once
#include <cuda_runtime.h>

namespace geo {
// The predictor's derivative contraction alone (probe_contract.inc).
cudaError_t probe_contraction_any(int order, int tensor, long long Z, int reps, cudaStream_t st, float* out,
                                  float* ms);
}  // namespace geo
