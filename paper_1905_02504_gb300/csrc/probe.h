// Entry points outside geo_step: measurement probes and the prism-zone predictor.
#pragma once
#include <cuda_runtime.h>

namespace geo {
// The predictor's derivative contraction alone (probe_contract.inc).
cudaError_t probe_contraction_any(int order, int tensor, long long Z, int reps, cudaStream_t st, float* out,
                                  float* ms);
// The ADER-CG predictor on the paper's prism zones (prism.inc).  D^alpha is
// passed in row form: Dv / Dc [3][N][prism_rl(p)] values and columns of each row's
// nonzeros, padded with value 0 and the row's own column.
__host__ __device__ constexpr int prism_rl(int p) { return p == 2 ? 4 : 16; }
cudaError_t launch_prism_predictor_any(int p, long long Z, const double* Dv, const unsigned char* Dc, const double* R,
                                       const double* X, const double* U, double dt, double gam, double* Uh,
                                       cudaStream_t st);
}  // namespace geo
