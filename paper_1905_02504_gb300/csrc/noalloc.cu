// Allocation-free variant of the CFL time-step reduction.
//
// Some callers cannot call cudaMalloc at the moment they need a time step: code
// that runs while another component owns the device memory pool (a fixed
// budget handed out once at start-up), code that must not synchronise the
// device (cudaMalloc can), or drivers that only hand the library pointers into
// memory they manage themselves.  geo_cfl_dt_noalloc() serves them: it reads the
// caller's conserved variables, writes the caller's output, and keeps its
// per-block partial minima in a fixed file-scope device array instead of memory
// allocated per call.  The array (GEO_NOALLOC_MAX_BLOCKS doubles, 512 KB) lives
// on every GPU that loads this library until the process exits.
#include <cuda_runtime.h>

#include <cfloat>
#include <mutex>
#include <string>

#include "../../include/geomhd.h"
#include "device.cuh"

struct geo_mesh;

namespace geo {
// accessors of the mesh internals, defined in api.cu
const DevTables* mesh_dev_tables(const geo_mesh* m);
cudaStream_t mesh_stream(const geo_mesh* m);
void set_error_message(const std::string& msg);
}  // namespace geo

namespace {

constexpr int kThreads = 256;

// Partial minima, one per block of the first pass.  Shared by every call on a
// device: calls that overlap on the GPU race on it.  Every slot a call reads is
// written earlier in the same call, so nothing has to start at zero.
static __device__ __align__(256) double g_cfl_scratch[GEO_NOALLOC_MAX_BLOCKS];

__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double block_min(double v) {
  __shared__ double sm[kThreads / 32];
  v = warp_min_d(v);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = DBL_MAX;
  if (threadIdx.x < 32) {
    r = threadIdx.x < kThreads / 32 ? sm[threadIdx.x] : DBL_MAX;
    r = warp_min_d(r);
  }
  return r;
}

// one zone per thread: in-sphere diameter over the fastest signal speed
__global__ void __launch_bounds__(kThreads) k_cfl_static_partial(const geo::DevTables T, const double* __restrict__ U,
                                                                 double* __restrict__ part) {
  const long long Z = T.Z;
  long long z = static_cast<long long>(blockIdx.x) * kThreads + threadIdx.x;
  double dtz = DBL_MAX;
  if (z < Z) {
    double rho = U[z], mx = U[Z + z], my = U[2 * Z + z], mz = U[3 * Z + z], en = U[4 * Z + z];
    double bx = U[5 * Z + z], by = U[6 * Z + z], bz = U[7 * Z + z];
    double ir = 1.0 / rho;
    double vx = mx * ir, vy = my * ir, vz = mz * ir;
    double b2 = bx * bx + by * by + bz * bz;
    double p = (T.gamma - 1.0) * (en - 0.5 * rho * (vx * vx + vy * vy + vz * vz) - 0.5 * b2);
    double cf = sqrt(T.gamma * p / rho + b2 / rho);
    double vm = sqrt(vx * vx + vy * vy + vz * vz);
    int c = static_cast<int>(z / T.nr), k = static_cast<int>(z % T.nr);
    double dz = 6.0 * T.V0[c] * T.qpow[k] / T.S0[c];
    dtz = dz / (vm + cf);
    if (!(dtz > 0.0)) dtz = -1.0;  // NaN or non-physical state poisons the minimum
  }
  double b = block_min(dtz);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__global__ void __launch_bounds__(kThreads) k_cfl_static_fold(const double* __restrict__ part, int n, double cfl,
                                                              double* __restrict__ out) {
  double v = DBL_MAX;
  for (int i = threadIdx.x; i < n; i += kThreads) v = fmin(v, part[i]);
  v = block_min(v);
  if (threadIdx.x == 0) out[0] = (v > 0.0) ? cfl * v : v;
}

// device address of g_cfl_scratch, looked up once per device
std::mutex g_mu;
double* g_addr[64] = {};

int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    geo::set_error_message(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return GEO_ERR_CUDA;
  }
  if (dev < 0 || dev >= 64) {
    geo::set_error_message("device ordinal out of range for the allocation-free path");
    return GEO_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_cfl_scratch);
    if (e != cudaSuccess) {
      geo::set_error_message(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return GEO_ERR_CUDA;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return GEO_OK;
}

}  // namespace

extern "C" int geo_cfl_dt_noalloc(geo_mesh_t mesh, const double* U_dev, double cfl, double* dt_dev) {
  if (!mesh || !U_dev || !dt_dev || !(cfl > 0.0)) {
    geo::set_error_message("geo_cfl_dt_noalloc: need a mesh, device U and dt pointers and cfl > 0");
    return GEO_ERR_ARG;
  }
  const geo::DevTables* T = geo::mesh_dev_tables(mesh);
  long long nb = (T->Z + kThreads - 1) / kThreads;
  if (nb > GEO_NOALLOC_MAX_BLOCKS) {
    geo::set_error_message("geo_cfl_dt_noalloc: the mesh has " + std::to_string(T->Z) +
                           " zones; the allocation-free reduction handles at most " +
                           std::to_string(static_cast<long long>(GEO_NOALLOC_MAX_BLOCKS) * kThreads));
    return GEO_ERR_ARG;
  }
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != GEO_OK) return rc;
  cudaStream_t st = geo::mesh_stream(mesh);
  k_cfl_static_partial<<<static_cast<unsigned>(nb), kThreads, 0, st>>>(*T, U_dev, scratch);
  k_cfl_static_fold<<<1, kThreads, 0, st>>>(scratch, static_cast<int>(nb), cfl, dt_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    geo::set_error_message(std::string("geo_cfl_dt_noalloc launch: ") + cudaGetErrorString(e));
    return GEO_ERR_CUDA;
  }
  return GEO_OK;
}
