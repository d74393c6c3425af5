// C ABI (include/geomhd.h) of the GB300 ADER-WENO-CT MHD library.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/geomhd.h"
#include "device.cuh"
#include "probe.h"
#include "host_tables.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return GEO_ERR_CUDA;
}

struct PendingTiming {
  int stage;
  cudaEvent_t a, b;
};

}  // namespace

struct geo_mesh {
  geo::Tables T;
  geo::DevTables dt{};
  geo::DevState ds{};
  cudaStream_t st = nullptr;
  int order = 0;
  int prec = GEO_FP64;
  bool have_state = false;
  std::vector<void*> allocs;
  bool timing = false;
  std::vector<PendingTiming> pending;
  // adjoint work buffers (allocated on the first geo_step_adjoint call)
  bool adj_ready = false;
  geo::DevState adj_fwd{};
  geo::AdjState adj{};
  double* adj_U0 = nullptr;
  double* adj_It = nullptr;  // stored Picard iterates of the node-team reverse sweep
  double ms[geo::N_STAGES] = {};
  int64_t cnt[geo::N_STAGES] = {};
  // physical-state flag of the last step, copied to pinned host memory after
  // each step and looked at by the next geo_step once that copy has landed
  int* status_host = nullptr;
  cudaEvent_t status_ev = nullptr;
  bool status_pending = false;

  template <typename Tv>
  const Tv* upload(const std::vector<Tv>& v, cudaError_t& err) {
    if (err != cudaSuccess) return nullptr;
    void* p = nullptr;
    size_t bytes = v.size() * sizeof(Tv);
    if (bytes == 0) bytes = sizeof(Tv);
    err = cudaMalloc(&p, bytes);
    if (err != cudaSuccess) return nullptr;
    allocs.push_back(p);
    if (!v.empty()) err = cudaMemcpy(p, v.data(), v.size() * sizeof(Tv), cudaMemcpyHostToDevice);
    return static_cast<const Tv*>(p);
  }
  // FP32 copy of an FP64 table (made once; the FP64 master stays on the device)
  const float* upload_f32(const std::vector<double>& v, cudaError_t& err) {
    std::vector<float> f(v.size());
    for (size_t i = 0; i < v.size(); ++i) f[i] = static_cast<float>(v[i]);
    return upload(f, err);
  }
  void* alloc_bytes(size_t n, cudaError_t& err) {
    if (err != cudaSuccess) return nullptr;
    void* p = nullptr;
    err = cudaMalloc(&p, n ? n : 1);
    if (err != cudaSuccess) return nullptr;
    allocs.push_back(p);
    return p;
  }
  double* alloc(size_t n, cudaError_t& err) {
    if (err != cudaSuccess) return nullptr;
    void* p = nullptr;
    err = cudaMalloc(&p, (n ? n : 1) * sizeof(double));
    if (err != cudaSuccess) return nullptr;
    allocs.push_back(p);
    return static_cast<double*>(p);
  }
  void release() {
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    if (status_host) cudaFreeHost(status_host);
    status_host = nullptr;
    if (status_ev) cudaEventDestroy(status_ev);
    status_ev = nullptr;
    for (auto& t : pending) {
      cudaEventDestroy(t.a);
      cudaEventDestroy(t.b);
    }
    pending.clear();
  }
};

static int run_stage(geo_mesh* m, int stage, double dt) {
  cudaError_t e = cudaSuccess;
  PendingTiming pt{stage, nullptr, nullptr};
  if (m->timing) {
    cudaEventCreate(&pt.a);
    cudaEventCreate(&pt.b);
    cudaEventRecord(pt.a, m->st);
  }
  const bool f32 = m->prec == GEO_FP32_BULK;
  switch (m->order) {
    case 2: e = f32 ? geo::launch_stage<2, float>(stage, m->dt, m->ds, dt, m->st)
                    : geo::launch_stage<2, double>(stage, m->dt, m->ds, dt, m->st); break;
    case 3: e = f32 ? geo::launch_stage<3, float>(stage, m->dt, m->ds, dt, m->st)
                    : geo::launch_stage<3, double>(stage, m->dt, m->ds, dt, m->st); break;
    default: e = f32 ? geo::launch_stage<4, float>(stage, m->dt, m->ds, dt, m->st)
                     : geo::launch_stage<4, double>(stage, m->dt, m->ds, dt, m->st); break;
  }
  if (m->timing) {
    cudaEventRecord(pt.b, m->st);
    m->pending.push_back(pt);
  }
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return GEO_OK;
}

namespace geo {
// accessors used by the allocation-free entry point (noalloc.cu)
const DevTables* mesh_dev_tables(const geo_mesh* m) { return &m->dt; }
cudaStream_t mesh_stream(const geo_mesh* m) { return m->st; }
void set_error_message(const std::string& msg) { g_err = msg; }
}  // namespace geo

extern "C" {

const char* geo_last_error(void) { return g_err.c_str(); }

int geo_mesh_create(int subdiv, int nr, double r_in, double r_out, int order, int prec, void* stream,
                    geo_mesh_t* out) {
  if (!out) return fail(GEO_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (prec != GEO_FP64 && prec != GEO_FP32_BULK) return fail(GEO_ERR_ARG, "prec must be GEO_FP64 or GEO_FP32_BULK");
  auto* m = new (std::nothrow) geo_mesh();
  if (!m) return fail(GEO_ERR_OOM, "host allocation failed");
  std::string msg = geo::build_tables(subdiv, nr, r_in, r_out, order, m->T);
  if (!msg.empty()) {
    delete m;
    return fail(GEO_ERR_ARG, msg);
  }
  m->order = order;
  m->prec = prec;
  m->st = static_cast<cudaStream_t>(stream);
  const geo::Tables& T = m->T;
  const geo::Dims& d = T.d;
  cudaError_t err = cudaSuccess;
  geo::DevTables& D = m->dt;
  D.n = T.n;
  D.nr = T.nr;
  D.ncol = T.ncol;
  D.nsv = T.nsv;
  D.nse = T.nse;
  D.Z = T.Z;
  D.F = T.F;
  D.E = T.E;
  D.F_rad = T.F_rad;
  D.E_rad = T.E_rad;
  D.gamma = 5.0 / 3.0;
  D.positivity = 0;
  // default schedule: the variable-layout team where it measured faster (orders
  // 2, 3, and the FP32-bulk form at order 4), the node team for FP64 at order 4
  // (3 % faster there)
  D.predictor = (order <= 3 || prec == GEO_FP32_BULK) ? GEO_PRED_VAR_TEAM : GEO_PRED_NODE_TEAM;
  D.riemann = GEO_RIEMANN_HLL;
  std::vector<double> qpow(T.nr + 2);
  for (int k = 0; k < T.nr + 2; ++k) qpow[k] = std::pow(T.q, k);
  D.qpow = m->upload(qpow, err);
  {
    std::vector<double> iA0(T.A0.size()), iq2(T.nr + 2);
    for (size_t i = 0; i < T.A0.size(); ++i) iA0[i] = 1.0 / T.A0[i];
    for (int k = 0; k < T.nr + 2; ++k) iq2[k] = 1.0 / (qpow[k] * qpow[k]);
    D.iA0 = m->upload(iA0, err);
    D.iq2 = m->upload(iq2, err);
  }
  D.D = m->upload(T.D, err);
  D.R = m->upload(T.R, err);
  D.wt = m->upload(T.wt, err);
  D.psiF = m->upload(T.psiF, err);
  D.psiE = m->upload(T.psiE, err);
  D.wE = m->upload(T.wE, err);
  D.st_n = m->upload(T.st_n, err);
  D.st_nb = m->upload(T.st_nb, err);
  D.pinvH = m->upload(T.pinvH, err);
  D.oct_nb = m->upload(T.oct_nb, err);
  D.oct_inv = m->upload(T.oct_inv, err);
  D.Q = m->upload(T.Q, err);
  D.V0 = m->upload(T.V0, err);
  D.l0 = m->upload(T.l0, err);
  D.S0 = m->upload(T.S0, err);
  D.A0 = m->upload(T.A0, err);
  D.TF = m->upload(T.TF, err);
  D.nF = m->upload(T.nF, err);
  D.wF = m->upload(T.wF, err);
  D.WF = m->upload(T.WF, err);
  // GB and TN transposed per column (team threads read consecutive rows)
  const int NR = 3 + 3 * d.N;
  std::vector<double> GBt(T.GB.size()), TNt(T.TN.size());
  for (int c = 0; c < T.ncol; ++c) {
    const size_t g0 = static_cast<size_t>(c) * NR * d.NBIN, t0 = static_cast<size_t>(c) * d.N * d.NC1;
    for (int r = 0; r < NR; ++r)
      for (int b = 0; b < d.NBIN; ++b) GBt[g0 + static_cast<size_t>(b) * NR + r] = T.GB[g0 + static_cast<size_t>(r) * d.NBIN + b];
    for (int i = 0; i < d.N; ++i)
      for (int mm = 0; mm < d.NC1; ++mm) TNt[t0 + static_cast<size_t>(mm) * d.N + i] = T.TN[t0 + static_cast<size_t>(i) * d.NC1 + mm];
  }
  D.GB = m->upload(GBt, err);
  D.TN = m->upload(TNt, err);
  D.J0 = m->upload(T.J0, err);
  D.iJ0 = m->upload(T.iJ0, err);
  D.Sm = m->upload(T.Sm, err);
  D.gcl = m->upload(T.gcl, err);
  D.JF = m->upload(T.JF, err);
  D.JE = m->upload(T.JE, err);
  D.col_side_se = m->upload(T.col_side_se, err);
  D.col_side_sgn = m->upload(T.col_side_sgn, err);
  D.se_v = m->upload(T.se_v, err);
  D.se_col = m->upload(T.se_col, err);
  D.se_lf = m->upload(T.se_lf, err);
  D.se_perm = m->upload(T.se_perm, err);
  D.se_le = m->upload(T.se_le, err);
  D.se_rev = m->upload(T.se_rev, err);
  D.se_t = m->upload(T.se_t, err);
  D.se_dlw = m->upload(T.se_dlw, err);
  D.se_nang = m->upload(T.se_nang, err);
  D.se_nradL = m->upload(T.se_nradL, err);
  D.se_nradR = m->upload(T.se_nradR, err);
  D.sv_nc = m->upload(T.sv_nc, err);
  D.sv_col = m->upload(T.sv_col, err);
  D.sv_le = m->upload(T.sv_le, err);
  D.sv_fL = m->upload(T.sv_fL, err);
  D.sv_fR = m->upload(T.sv_fR, err);
  D.sv_fse = m->upload(T.sv_fse, err);
  D.sv_fn = m->upload(T.sv_fn, err);
  D.sv_t = m->upload(T.sv_t, err);
  D.sv_dlw = m->upload(T.sv_dlw, err);
  // (l_0 / |x_0|)^2 per column: the WENO-AO eps scale
  std::vector<double> weta(T.ncol);
  for (int c = 0; c < T.ncol; ++c) {
    const double* x = &T.xc0[3 * c];
    weta[c] = T.l0[c] * T.l0[c] / (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  }
  // bulk-arithmetic views of the per-column matrices
  std::vector<double> iJF(T.JF.size()), iJE(T.JE.size());
  for (size_t t = 0; t < iJF.size(); ++t) iJF[t] = 1.0 / T.JF[t];
  for (size_t t = 0; t < iJE.size(); ++t) iJE[t] = 1.0 / T.JE[t];
  D.b64 = geo::BulkTables<double>{D.pinvH, D.oct_inv, D.Q,        D.TF,       D.nF,       D.wF,
                                  D.GB,    D.TN,      D.J0,       D.iJ0,      D.Sm,       D.gcl,
                                  D.JF,    D.JE,      D.se_t,     D.se_nang,  D.se_nradL, D.se_nradR,
                                  D.sv_fn, D.sv_t,    m->upload(weta, err), m->upload(iJF, err),
                                  m->upload(iJE, err)};
  const bool f32 = prec == GEO_FP32_BULK;
  if (f32) {
    geo::BulkTables<float>& b = D.b32;
    b.pinvH = m->upload_f32(T.pinvH, err);
    b.oct_inv = m->upload_f32(T.oct_inv, err);
    b.weta = m->upload_f32(weta, err);
    b.iJF = m->upload_f32(iJF, err);
    b.iJE = m->upload_f32(iJE, err);
    b.Q = m->upload_f32(T.Q, err);
    b.TF = m->upload_f32(T.TF, err);
    b.nF = m->upload_f32(T.nF, err);
    b.wF = m->upload_f32(T.wF, err);
    b.GB = m->upload_f32(GBt, err);
    b.TN = m->upload_f32(TNt, err);
    b.J0 = m->upload_f32(T.J0, err);
    b.iJ0 = m->upload_f32(T.iJ0, err);
    b.Sm = m->upload_f32(T.Sm, err);
    b.gcl = m->upload_f32(T.gcl, err);
    b.JF = m->upload_f32(T.JF, err);
    b.JE = m->upload_f32(T.JE, err);
    b.se_t = m->upload_f32(T.se_t, err);
    b.se_nang = m->upload_f32(T.se_nang, err);
    b.se_nradL = m->upload_f32(T.se_nradL, err);
    b.se_nradR = m->upload_f32(T.se_nradR, err);
    b.sv_fn = m->upload_f32(T.sv_fn, err);
    b.sv_t = m->upload_f32(T.sv_t, err);
  }
  if (err == cudaSuccess) {
    if (order == 2) err = f32 ? geo::upload_reference_constants<2, float>(T) : geo::upload_reference_constants<2, double>(T);
    else if (order == 3) err = f32 ? geo::upload_reference_constants<3, float>(T) : geo::upload_reference_constants<3, double>(T);
    else err = f32 ? geo::upload_reference_constants<4, float>(T) : geo::upload_reference_constants<4, double>(T);
  }
  const size_t Z = T.Z, F = T.F, E = T.E;
  const int nqmax = d.NQR > d.NQS ? d.NQR : d.NQS;
  geo::DevState& S = m->ds;
  S.U = m->alloc(8 * Z, err);
  S.phi = m->alloc(F, err);
  const size_t rb = f32 ? sizeof(float) : sizeof(double);
  S.Wc = m->alloc_bytes(rb * 8 * d.NC1 * Z, err);
  S.Bp = m->alloc_bytes(rb * nqmax * F, err);
  S.trF = m->alloc_bytes(rb * (d.M - 1) * d.NQT * 8 * Z, err);
  S.trE = m->alloc_bytes(rb * (d.M - 1) * 12 * d.NS * 8 * Z, err);
  S.Ff = m->alloc(8 * F, err);
  S.Ee = m->alloc(E, err);
  S.red = m->alloc(4096, err);
  S.Uhl = f32 ? static_cast<float*>(m->alloc_bytes(sizeof(float) * 16 * Z, err)) : nullptr;
  m->dt.status = static_cast<int*>(m->alloc_bytes(sizeof(int), err));
  if (err == cudaSuccess) err = cudaMemset(m->dt.status, 0, sizeof(int));
  if (err == cudaSuccess) err = cudaMallocHost(&m->status_host, sizeof(int));
  if (err == cudaSuccess) {
    *m->status_host = 0;
    err = cudaEventCreateWithFlags(&m->status_ev, cudaEventDisableTiming);
  }
  if (err != cudaSuccess) {
    int code = (err == cudaErrorMemoryAllocation) ? GEO_ERR_OOM : GEO_ERR_CUDA;
    std::string s = std::string("device setup: ") + cudaGetErrorString(err);
    m->release();
    delete m;
    cudaGetLastError();
    return fail(code, s);
  }
  *out = m;
  return GEO_OK;
}

int geo_mesh_destroy(geo_mesh_t m) {
  if (!m) return fail(GEO_ERR_ARG, "mesh is NULL");
  cudaStreamSynchronize(m->st);
  m->release();
  delete m;
  return GEO_OK;
}

int geo_mesh_sizes(geo_mesh_t m, int64_t* nz, int64_t* nf, int64_t* ne) {
  if (!m) return fail(GEO_ERR_ARG, "mesh is NULL");
  if (nz) *nz = m->T.Z;
  if (nf) *nf = m->T.F;
  if (ne) *ne = m->T.E;
  return GEO_OK;
}

int geo_set_gamma(geo_mesh_t m, double gamma) {
  if (!m || !(gamma > 1.0)) return fail(GEO_ERR_ARG, "need a mesh and gamma > 1");
  m->dt.gamma = gamma;
  return GEO_OK;
}

int geo_set_positivity(geo_mesh_t m, int enable) {
  if (!m) return fail(GEO_ERR_ARG, "mesh is NULL");
  m->dt.positivity = enable ? 1 : 0;
  return GEO_OK;
}

int geo_set_riemann(geo_mesh_t m, int solver) {
  if (!m) return fail(GEO_ERR_ARG, "mesh is NULL");
  if (solver != GEO_RIEMANN_HLL && solver != GEO_RIEMANN_HLLD) return fail(GEO_ERR_ARG, "unknown face solver");
  m->dt.riemann = solver;
  return GEO_OK;
}

int geo_set_predictor(geo_mesh_t m, int schedule) {
  if (!m) return fail(GEO_ERR_ARG, "mesh is NULL");
  if (schedule != GEO_PRED_ZONE_THREAD && schedule != GEO_PRED_NODE_TEAM && schedule != GEO_PRED_VAR_TEAM)
    return fail(GEO_ERR_ARG, "unknown predictor schedule");
  m->dt.predictor = schedule;
  return GEO_OK;
}

int geo_zone_cubature(geo_mesh_t m, int nq, double* pts, double* w) {
  if (!m || !pts || !w || nq < 1 || nq > 12) return fail(GEO_ERR_ARG, "bad cubature arguments");
  geo::zone_cubature(m->T, nq, pts, w);
  return GEO_OK;
}

int geo_edge_quadrature(geo_mesh_t m, int nq, double* pts, double* tw) {
  if (!m || !pts || !tw || nq < 1 || nq > 12) return fail(GEO_ERR_ARG, "bad quadrature arguments");
  geo::edge_quadrature(m->T, nq, pts, tw);
  return GEO_OK;
}

int geo_radial_face_quadrature(geo_mesh_t m, int nq, double* pts, double* wn) {
  if (!m || !pts || !wn || nq < 1 || nq > 12) return fail(GEO_ERR_ARG, "bad quadrature arguments");
  geo::radial_face_quadrature(m->T, nq, pts, wn);
  return GEO_OK;
}

int geo_phi_from_edge_circulation(geo_mesh_t m, const double* circ, double* phi) {
  if (!m || !circ || !phi) return fail(GEO_ERR_ARG, "bad arguments");
  geo::phi_from_circulation(m->T, circ, phi);
  return GEO_OK;
}

int geo_zone_geometry(geo_mesh_t m, double* xc, double* vol) {
  if (!m || !xc || !vol) return fail(GEO_ERR_ARG, "bad arguments");
  geo::zone_centroids(m->T, xc, vol);
  return GEO_OK;
}

int geo_host_geometry(int subdiv, int nr, double r_in, double r_out, int order, int64_t zones, int64_t faces,
                      double* centroid, double* volume, double* area, double* normal) {
  if (!centroid || !volume || !area || !normal) return fail(GEO_ERR_ARG, "geo_host_geometry: bad arguments");
  if (subdiv < 1 || nr < 1 || !(r_in > 0.0) || !(r_out > r_in) || order < 2 || order > 4)
    return fail(GEO_ERR_ARG, "geo_host_geometry: bad mesh");
  geo::Tables T;
  const std::string err = geo::build_tables(subdiv, nr, r_in, r_out, order, T);
  if (!err.empty()) return fail(GEO_ERR_ARG, err);
  if (zones != static_cast<int64_t>(T.Z) || faces != static_cast<int64_t>(T.F))
    return fail(GEO_ERR_ARG, "geo_host_geometry: zones / faces do not match the mesh");
  geo::zone_centroids(T, centroid, volume);
  geo::face_geometry(T, area, normal);
  return GEO_OK;
}

int geo_face_geometry(geo_mesh_t m, double* area, double* normal) {
  if (!m || !area || !normal) return fail(GEO_ERR_ARG, "bad arguments");
  geo::face_geometry(m->T, area, normal);
  return GEO_OK;
}

int geo_state_upload(geo_mesh_t m, const double* U, const double* phi, int on_device) {
  if (!m || !U || !phi) return fail(GEO_ERR_ARG, "bad arguments");
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpyAsync(m->ds.U, U, 8 * m->T.Z * sizeof(double), kind, m->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->ds.phi, phi, m->T.F * sizeof(double), kind, m->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->dt.status, 0, sizeof(int), m->st);
  if (e == cudaSuccess) e = geo::launch_split_u(m->dt, m->ds, m->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) return cuda_fail(e, "state upload");
  m->status_pending = false;
  *m->status_host = 0;
  m->have_state = true;
  return GEO_OK;
}

int geo_state_download(geo_mesh_t m, double* U, double* phi, int on_device) {
  if (!m || !U || !phi) return fail(GEO_ERR_ARG, "bad arguments");
  if (!m->have_state) return fail(GEO_ERR_STATE, "no state uploaded");
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaMemcpyAsync(U, m->ds.U, 8 * m->T.Z * sizeof(double), kind, m->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(phi, m->ds.phi, m->T.F * sizeof(double), kind, m->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) return cuda_fail(e, "state download");
  return GEO_OK;
}

int geo_cfl_dt(geo_mesh_t m, double cfl, double* dt) {
  if (!m || !dt || !(cfl > 0.0)) return fail(GEO_ERR_ARG, "bad arguments");
  if (!m->have_state) return fail(GEO_ERR_STATE, "no state uploaded");
  cudaError_t e = geo::launch_cfl(m->dt, m->ds, cfl, dt, m->st);
  if (e != cudaSuccess) return cuda_fail(e, "cfl reduction");
  if (!(*dt > 0.0) || !std::isfinite(*dt)) return fail(GEO_ERR_NONPHYSICAL, "non-physical state in CFL reduction");
  return GEO_OK;
}

int geo_step(geo_mesh_t m, double dt) {
  if (!m || !(dt > 0.0) || !std::isfinite(dt)) return fail(GEO_ERR_ARG, "bad arguments");
  if (!m->have_state) return fail(GEO_ERR_STATE, "no state uploaded");
  if (m->status_pending && cudaEventQuery(m->status_ev) == cudaSuccess) {
    m->status_pending = false;
    if (*m->status_host) return fail(GEO_ERR_NONPHYSICAL, "an earlier step produced a non-physical state");
  }
  for (int s = 0; s < geo::N_STAGES; ++s) {
    int rc = run_stage(m, s, dt);
    if (rc != GEO_OK) return rc;
  }
  cudaError_t e = cudaMemcpyAsync(m->status_host, m->dt.status, sizeof(int), cudaMemcpyDeviceToHost, m->st);
  if (e == cudaSuccess) e = cudaEventRecord(m->status_ev, m->st);
  if (e != cudaSuccess) return cuda_fail(e, "status copy");
  m->status_pending = true;
  return GEO_OK;
}

int geo_check_state(geo_mesh_t m, int* flags) {
  if (!m || !flags) return fail(GEO_ERR_ARG, "bad arguments");
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, m->dt.status, sizeof(int), cudaMemcpyDeviceToHost, m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->dt.status, 0, sizeof(int), m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) return cuda_fail(e, "state check");
  *m->status_host = 0;
  m->status_pending = false;
  *flags = h;
  return h ? fail(GEO_ERR_NONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or not finite) in a zone") : GEO_OK;
}

int geo_divB_max(geo_mesh_t m, double* abs_max, double* rel_max) {
  if (!m || !abs_max || !rel_max) return fail(GEO_ERR_ARG, "bad arguments");
  if (!m->have_state) return fail(GEO_ERR_STATE, "no state uploaded");
  double out[2] = {0, 0};
  cudaError_t e = geo::launch_divb(m->dt, m->ds, out, m->st);
  if (e != cudaSuccess) return cuda_fail(e, "divB reduction");
  *abs_max = out[0];
  *rel_max = out[1];
  return GEO_OK;
}

int geo_set_stage_timing(geo_mesh_t m, int enable) {
  if (!m) return fail(GEO_ERR_ARG, "mesh is NULL");
  m->timing = enable != 0;
  return GEO_OK;
}

int geo_get_stage_timing(geo_mesh_t m, double* ms, int64_t* counts) {
  if (!m || !ms || !counts) return fail(GEO_ERR_ARG, "bad arguments");
  cudaError_t e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) return cuda_fail(e, "timing sync");
  for (auto& t : m->pending) {
    float x = 0.f;
    cudaEventElapsedTime(&x, t.a, t.b);
    m->ms[t.stage] += x;
    m->cnt[t.stage] += 1;
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  m->pending.clear();
  for (int s = 0; s < geo::N_STAGES; ++s) {
    ms[s] = m->ms[s];
    counts[s] = m->cnt[s];
    m->ms[s] = 0.0;
    m->cnt[s] = 0;
  }
  return GEO_OK;
}

int geo_stage_flops(geo_mesh_t m, double* fl, int64_t* units) {
  if (!m || !fl || !units) return fail(GEO_ERR_ARG, "bad arguments");
  const geo::Dims& d = m->T.d;
  const double N = d.N, M = d.M, NC1 = d.NC1, NQT = d.NQT, NS = d.NS, P = d.P, NBIN = d.NBIN;
  const double nq_mean = NQT / 6.0;
  double ns = 0;
  for (int v : m->T.st_n) ns += v;
  ns /= m->T.ncol;
  const double flux1 = 40.0;  // one physical flux F(U).n with its primitive recovery
  const double hll = 2 * flux1 + 60.0;
  // WENO-AO, per zone and variable: central LSQ apply, smoothness form, 8 octant fits
  fl[geo::ST_WENO] = 8.0 * (ns * (1 + 2 * NC1) + 2 * NC1 * NC1 + 2 * NC1 + 8 * (3 + 18 + 6 + 4) + 3 * 48 + 2 * NC1);
  units[geo::ST_WENO] = m->T.Z;
  // nodal normal B per face: two polynomial evaluations per point, MinMod, shift
  fl[geo::ST_BPERP] = nq_mean * (2 * (3 * 2 * NC1 + 5) + 8);
  units[geo::ST_BPERP] = m->T.F;
  // ADER: KKT apply + node values, then 1 + (p-1)(M-1) flux-difference levels (the
  // first Picard iteration reuses level 1's), each
  // with N primitive recoveries, 4 physical fluxes per node (3 metric directions
  // + the geometric-conservation residual) and the 3 NNZ nonzero couplings of the
  // serendipity derivative matrices over 8 variables; p Picard updates of M-1
  // levels; point values at the face (edge) points from the face's (edge's) nodes
  const double levels = 1 + (P - 1) * (M - 1);
  const double flux = 45.0, prim = 17.0;
  const double per_level = N * (8 + prim + 4 * flux + 8) + 3.0 * d.NNZ * 8 * 2;
  fl[geo::ST_ADER] = 2 * (3 + 3 * N) * NBIN + N * 5 * 2 * NC1 + levels * per_level +
                     P * (M - 1) * N * 8 * 2 * M +
                     (M - 1) * (NQT * (d.NFN * 16 + 8) + 12 * NS * (d.NEN * 16 + 8));
  units[geo::ST_ADER] = m->T.Z;
  fl[geo::ST_FACE] = (M - 1) * nq_mean * (hll + 16);
  units[geo::ST_FACE] = m->T.F;
  fl[geo::ST_EDGE] = (M - 1) * NS * (4 * 16 + 4 * (2 * 45 + 20) + 4);
  units[geo::ST_EDGE] = m->T.E;
  fl[geo::ST_UPD_U] = 6 * 8 * 2 + 8;
  units[geo::ST_UPD_U] = m->T.Z;
  fl[geo::ST_UPD_PHI] = 4;
  units[geo::ST_UPD_PHI] = m->T.F;
  return GEO_OK;
}

int geo_debug_buffer(geo_mesh_t m, int which, double* host, int64_t count) {
  if (!m || !host) return fail(GEO_ERR_ARG, "bad arguments");
  const geo::Dims& d = m->T.d;
  const int64_t Z = m->T.Z, F = m->T.F, E = m->T.E;
  const int nqmax = d.NQR > d.NQS ? d.NQR : d.NQS;
  const void* src = nullptr;
  int64_t n = 0;
  bool bulk = true;
  switch (which) {
    case 0: src = m->ds.Wc; n = 8LL * d.NC1 * Z; break;
    case 1: src = m->ds.Bp; n = static_cast<int64_t>(nqmax) * F; break;
    case 2: src = m->ds.trF; n = static_cast<int64_t>(d.M - 1) * d.NQT * 8 * Z; break;
    case 3: src = m->ds.trE; n = static_cast<int64_t>(d.M - 1) * 12 * d.NS * 8 * Z; break;
    case 4: src = m->ds.Ff; n = 8 * F; bulk = false; break;
    case 5: src = m->ds.Ee; n = E; bulk = false; break;
    default: return fail(GEO_ERR_ARG, "unknown buffer");
  }
  if (count < n) return fail(GEO_ERR_ARG, "host buffer too small");
  cudaError_t e;
  if (bulk && m->prec == GEO_FP32_BULK) {
    std::vector<float> tmp(n);
    e = cudaMemcpyAsync(tmp.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost, m->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    for (int64_t i = 0; i < n; ++i) host[i] = tmp[i];
  } else {
    e = cudaMemcpyAsync(host, src, n * sizeof(double), cudaMemcpyDeviceToHost, m->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "debug copy");
  return GEO_OK;
}

static int ensure_adjoint_buffers(geo_mesh* m) {
  if (m->adj_ready) return GEO_OK;
  const geo::Dims& d = m->T.d;
  const size_t Z = m->T.Z, F = m->T.F, E = m->T.E;
  const int nqmax = d.NQR > d.NQS ? d.NQR : d.NQS;
  cudaError_t err = cudaSuccess;
  geo::DevState& S = m->adj_fwd;
  S.U = m->alloc(8 * Z, err);
  S.phi = m->alloc(F, err);
  S.Wc = m->alloc(static_cast<size_t>(8) * d.NC1 * Z, err);
  S.Bp = m->alloc(static_cast<size_t>(nqmax) * F, err);
  S.trF = m->alloc(static_cast<size_t>(d.M - 1) * d.NQT * 8 * Z, err);
  S.trE = m->alloc(static_cast<size_t>(d.M - 1) * 12 * d.NS * 8 * Z, err);
  S.Ff = m->alloc(8 * F, err);
  S.Ee = m->alloc(E, err);
  S.red = m->ds.red;
  m->adj_U0 = m->alloc(8 * Z, err);
  geo::AdjState& A = m->adj;
  A.gFf = m->alloc(8 * F, err);
  A.gEe = m->alloc(E, err);
  A.gtrF = m->alloc(static_cast<size_t>(d.M - 1) * d.NQT * 8 * Z, err);
  A.gtrE = m->alloc(static_cast<size_t>(d.M - 1) * 12 * d.NS * 8 * Z, err);
  A.gW = m->alloc(static_cast<size_t>(8) * d.NC1 * Z, err);
  A.gBpz = m->alloc(static_cast<size_t>(d.NQT) * Z, err);
  A.gphiz = m->alloc(6 * Z, err);
  A.U0 = m->adj_U0;
  // [P-1][M-1][8][N][Z]: the linearisation points of the reverse predictor
  m->adj_It = m->alloc(static_cast<size_t>(d.P - 1) * (d.M - 1) * 8 * d.N * Z, err);
  if (err != cudaSuccess) return cuda_fail(err, "adjoint buffers");
  m->adj_ready = true;
  return GEO_OK;
}

int geo_step_adjoint(geo_mesh_t m, double dt, const double* U_in, const double* phi_in, const double* gU_out,
                     const double* gphi_out, double* gU_in, double* gphi_in) {
  if (!m || !U_in || !phi_in || !gU_out || !gphi_out || !gU_in || !gphi_in || !(dt > 0.0))
    return fail(GEO_ERR_ARG, "geo_step_adjoint: bad arguments");
  if (m->prec != GEO_FP64) return fail(GEO_ERR_ARG, "geo_step_adjoint: the adjoint is available for GEO_FP64 meshes");
  if (m->dt.positivity)
    return fail(GEO_ERR_ARG, "geo_step_adjoint: the positivity scaling is not differentiated; switch it off");
  if (m->dt.riemann != GEO_RIEMANN_HLL)
    return fail(GEO_ERR_ARG, "geo_step_adjoint: the reverse sweep differentiates the HLL face solver only");
  int rc = ensure_adjoint_buffers(m);
  if (rc != GEO_OK) return rc;
  const size_t Z = m->T.Z, F = m->T.F;
  cudaError_t e = cudaMemcpyAsync(m->adj_U0, U_in, 8 * Z * sizeof(double), cudaMemcpyDeviceToDevice, m->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->adj_fwd.U, U_in, 8 * Z * sizeof(double), cudaMemcpyDeviceToDevice, m->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->adj_fwd.phi, phi_in, F * sizeof(double), cudaMemcpyDeviceToDevice, m->st);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint checkpoint copy");
  // forward intermediates of the checkpoint state; with a team schedule the
  // predictor is the node team that also stores its Picard iterates, which the
  // reverse predictor then reads instead of recomputing them
  const bool store = m->dt.predictor != GEO_PRED_ZONE_THREAD;
  for (int s = geo::ST_WENO; s <= geo::ST_ADER && e == cudaSuccess; ++s) {
    if (s == geo::ST_ADER && store) {
      switch (m->order) {
        case 2: e = geo::launch_ader_store_iterates<2>(m->dt, m->adj_fwd, m->adj_It, dt, m->st); break;
        case 3: e = geo::launch_ader_store_iterates<3>(m->dt, m->adj_fwd, m->adj_It, dt, m->st); break;
        default: e = geo::launch_ader_store_iterates<4>(m->dt, m->adj_fwd, m->adj_It, dt, m->st); break;
      }
      continue;
    }
    switch (m->order) {
      case 2: e = geo::launch_stage<2, double>(s, m->dt, m->adj_fwd, dt, m->st); break;
      case 3: e = geo::launch_stage<3, double>(s, m->dt, m->adj_fwd, dt, m->st); break;
      default: e = geo::launch_stage<4, double>(s, m->dt, m->adj_fwd, dt, m->st); break;
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "adjoint forward recompute");
  geo::AdjState A = m->adj;
  A.It = store ? m->adj_It : nullptr;
  A.gUp = gU_out;
  A.gphip = gphi_out;
  A.gU = gU_in;
  A.gphi = gphi_in;
  // the forward k_ader overwrote the zone B of the working copy; the adjoint
  // kernels read the pristine checkpoint (A.U0) and the pre-step face fluxes
  geo::DevState S = m->adj_fwd;
  switch (m->order) {
    case 2: e = geo::launch_adjoint<2>(m->dt, S, A, dt, m->st); break;
    case 3: e = geo::launch_adjoint<3>(m->dt, S, A, dt, m->st); break;
    default: e = geo::launch_adjoint<4>(m->dt, S, A, dt, m->st); break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
  return GEO_OK;
}

// ---- test support: one stage forward or reversed, on host buffers (FP64 meshes)
static int debug_buffer_slot(geo_mesh* m, int which, void** ptr, int64_t* n) {
  const geo::Dims& d = m->T.d;
  const int64_t Z = m->T.Z, F = m->T.F, E = m->T.E;
  const int nqmax = d.NQR > d.NQS ? d.NQR : d.NQS;
  switch (which) {
    case 0: *ptr = m->ds.Wc; *n = 8LL * d.NC1 * Z; return GEO_OK;
    case 1: *ptr = m->ds.Bp; *n = static_cast<int64_t>(nqmax) * F; return GEO_OK;
    case 2: *ptr = m->ds.trF; *n = static_cast<int64_t>(d.M - 1) * d.NQT * 8 * Z; return GEO_OK;
    case 3: *ptr = m->ds.trE; *n = static_cast<int64_t>(d.M - 1) * 12 * d.NS * 8 * Z; return GEO_OK;
    case 4: *ptr = m->ds.Ff; *n = 8 * F; return GEO_OK;
    case 5: *ptr = m->ds.Ee; *n = E; return GEO_OK;
    default: return fail(GEO_ERR_ARG, "unknown buffer");
  }
}

int geo_debug_set_buffer(geo_mesh_t m, int which, const double* host, int64_t count) {
  if (!m || !host) return fail(GEO_ERR_ARG, "bad arguments");
  if (m->prec != GEO_FP64) return fail(GEO_ERR_ARG, "geo_debug_set_buffer: FP64 meshes only");
  void* dst = nullptr;
  int64_t n = 0;
  int rc = debug_buffer_slot(m, which, &dst, &n);
  if (rc != GEO_OK) return rc;
  if (count != n) return fail(GEO_ERR_ARG, "geo_debug_set_buffer: count must equal the buffer size");
  cudaError_t e = cudaMemcpyAsync(dst, host, n * sizeof(double), cudaMemcpyHostToDevice, m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) return cuda_fail(e, "debug copy");
  return GEO_OK;
}

int geo_debug_run_stage(geo_mesh_t m, int stage, double dt) {
  if (!m || stage < 0 || stage >= geo::N_STAGES) return fail(GEO_ERR_ARG, "bad arguments");
  cudaError_t e;
  switch (m->order) {
    case 2: e = m->prec == GEO_FP64 ? geo::launch_stage<2, double>(stage, m->dt, m->ds, dt, m->st)
                                    : geo::launch_stage<2, float>(stage, m->dt, m->ds, dt, m->st); break;
    case 3: e = m->prec == GEO_FP64 ? geo::launch_stage<3, double>(stage, m->dt, m->ds, dt, m->st)
                                    : geo::launch_stage<3, float>(stage, m->dt, m->ds, dt, m->st); break;
    default: e = m->prec == GEO_FP64 ? geo::launch_stage<4, double>(stage, m->dt, m->ds, dt, m->st)
                                     : geo::launch_stage<4, float>(stage, m->dt, m->ds, dt, m->st); break;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) return cuda_fail(e, "geo_debug_run_stage");
  return GEO_OK;
}

int geo_debug_stage_vjp(geo_mesh_t m, int stage, double dt, const double* U, const double* phi, const double* g_out,
                        int64_t n_out, double* g_in, int64_t n_in) {
  if (!m || !U || !phi || !g_out || !g_in || !(dt > 0.0)) return fail(GEO_ERR_ARG, "bad arguments");
  if (m->prec != GEO_FP64) return fail(GEO_ERR_ARG, "geo_debug_stage_vjp: FP64 meshes only");
  int rc = ensure_adjoint_buffers(m);
  if (rc != GEO_OK) return rc;
  const geo::Dims& d = m->T.d;
  const size_t Z = m->T.Z, F = m->T.F, E = m->T.E;
  const int64_t nW = 8LL * d.NC1 * Z, nF = static_cast<int64_t>(d.M - 1) * d.NQT * 8 * Z,
                nE = static_cast<int64_t>(d.M - 1) * 12 * d.NS * 8 * Z;
  geo::AdjState A = m->adj;
  double *dst_out = nullptr, *src_in = nullptr;
  int64_t want_out = 0, want_in = 0;
  switch (stage) {
    case geo::ST_WENO: dst_out = A.gW; want_out = nW; want_in = 8 * Z; break;
    case geo::ST_ADER: dst_out = A.gtrF; want_out = nF + nE; src_in = A.gW; want_in = nW; break;
    case geo::ST_FACE: dst_out = A.gFf; want_out = 8 * F; src_in = A.gtrF; want_in = nF; break;
    case geo::ST_EDGE: dst_out = A.gEe; want_out = E; src_in = A.gtrE; want_in = nE; break;
    default: return fail(GEO_ERR_ARG, "geo_debug_stage_vjp: stage must be WENO, ADER, FACE or EDGE");
  }
  if (n_out != want_out || n_in != want_in) return fail(GEO_ERR_ARG, "geo_debug_stage_vjp: wrong buffer sizes");
  // the zone cotangents: a zero incoming one, and the WENO stage's output
  double* gU0 = nullptr;
  double* gU = nullptr;
  cudaError_t e = cudaMalloc(&gU0, 8 * Z * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&gU, 8 * Z * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(gU0, 0, 8 * Z * sizeof(double), m->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(gU, 0, 8 * Z * sizeof(double), m->st);
  // forward intermediates of (U, phi), as in geo_step_adjoint
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->adj_U0, U, 8 * Z * sizeof(double), cudaMemcpyHostToDevice, m->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->adj_fwd.U, U, 8 * Z * sizeof(double), cudaMemcpyHostToDevice, m->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->adj_fwd.phi, phi, F * sizeof(double), cudaMemcpyHostToDevice, m->st);
  for (int s = geo::ST_WENO; s <= geo::ST_ADER && e == cudaSuccess; ++s) {
    switch (m->order) {
      case 2: e = geo::launch_stage<2, double>(s, m->dt, m->adj_fwd, dt, m->st); break;
      case 3: e = geo::launch_stage<3, double>(s, m->dt, m->adj_fwd, dt, m->st); break;
      default: e = geo::launch_stage<4, double>(s, m->dt, m->adj_fwd, dt, m->st); break;
    }
  }
  A.gUp = gU0;
  A.gphip = nullptr;
  A.gU = gU;
  if (stage == geo::ST_ADER) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(A.gtrF, g_out, nF * sizeof(double), cudaMemcpyHostToDevice, m->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(A.gtrE, g_out + nF, nE * sizeof(double), cudaMemcpyHostToDevice, m->st);
  } else if (e == cudaSuccess) {
    e = cudaMemcpyAsync(dst_out, g_out, want_out * sizeof(double), cudaMemcpyHostToDevice, m->st);
  }
  if (e == cudaSuccess) {
    switch (m->order) {
      case 2: e = geo::launch_adjoint_stage<2>(stage, m->dt, m->adj_fwd, A, dt, m->st); break;
      case 3: e = geo::launch_adjoint_stage<3>(stage, m->dt, m->adj_fwd, A, dt, m->st); break;
      default: e = geo::launch_adjoint_stage<4>(stage, m->dt, m->adj_fwd, A, dt, m->st); break;
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g_in, stage == geo::ST_WENO ? gU : src_in, want_in * sizeof(double), cudaMemcpyDeviceToHost,
                        m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  cudaFree(gU0);
  cudaFree(gU);
  if (e != cudaSuccess) return cuda_fail(e, "geo_debug_stage_vjp");
  return GEO_OK;
}

int geo_outer_Br2(geo_mesh_t m, const double* phi_dev, double* J, double* gphi_dev) {
  if (!m || !phi_dev || !J) return fail(GEO_ERR_ARG, "geo_outer_Br2: bad arguments");
  cudaError_t e = cudaSuccess;
  if (gphi_dev) e = cudaMemsetAsync(gphi_dev, 0, m->T.F * sizeof(double), m->st);
  if (e == cudaSuccess) e = geo::launch_outer_br2(m->dt, phi_dev, m->ds.red + 3000, gphi_dev, m->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(J, m->ds.red + 3000, sizeof(double), cudaMemcpyDeviceToHost, m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) return cuda_fail(e, "geo_outer_Br2");
  return GEO_OK;
}

int geo_probe_fma_peak(int prec, void* stream, double* flops_per_s) {
  if (!flops_per_s) return fail(GEO_ERR_ARG, "bad arguments");
  cudaError_t e = geo::probe_fma(prec, static_cast<cudaStream_t>(stream), flops_per_s);
  if (e != cudaSuccess) return cuda_fail(e, "fma probe");
  return GEO_OK;
}

// prism tables per order on the device, built on first use and kept until exit
namespace {
struct PrismTables {
  std::once_flag once;
  int status = GEO_ERR_CUDA;
  std::string err;
  int N = 0;
  std::vector<double> nodes;
  double* Dv = nullptr;         // [3][N][RL] nonzeros of each row of D^alpha
  unsigned char* Dc = nullptr;  // [3][N][RL] their columns (padding: value 0, the row's own column)
  double* R = nullptr;          // [M][M]
};
PrismTables g_prism[3];

PrismTables& prism_tables_for(int p) {
  PrismTables& P = g_prism[p - 2];
  std::call_once(P.once, [&]() {
    std::vector<double> D, wt, R;
    if (!geo::prism_element(p, P.nodes, D)) {
      P.status = GEO_ERR_ARG;
      P.err = "prism element: singular basis";
      return;
    }
    geo::time_tables(p, wt, R);
    const int N = static_cast<int>(P.nodes.size() / 3), RL = geo::prism_rl(p);
    P.N = N;
    std::vector<double> Dv(static_cast<size_t>(3) * N * RL, 0.0);
    std::vector<unsigned char> Dc(static_cast<size_t>(3) * N * RL, 0);
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < N; ++i) {
        int r = 0;
        for (int j = 0; j < N; ++j) {
          const double d = D[(static_cast<size_t>(a) * N + i) * N + j];
          if (d == 0.0) continue;
          if (r == RL) {
            P.status = GEO_ERR_ARG;
            P.err = "prism element: a row of D has more nonzeros than the row form holds";
            return;
          }
          Dv[(static_cast<size_t>(a) * N + i) * RL + r] = d;
          Dc[(static_cast<size_t>(a) * N + i) * RL + r] = static_cast<unsigned char>(j);
          ++r;
        }
        for (; r < RL; ++r) Dc[(static_cast<size_t>(a) * N + i) * RL + r] = static_cast<unsigned char>(i);
      }
    cudaError_t e = cudaMalloc(&P.Dv, Dv.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&P.Dc, Dc.size());
    if (e == cudaSuccess) e = cudaMalloc(&P.R, R.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(P.Dv, Dv.data(), Dv.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P.Dc, Dc.data(), Dc.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P.R, R.data(), R.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      P.err = std::string("prism tables: ") + cudaGetErrorString(e);
      return;
    }
    P.status = GEO_OK;
  });
  return P;
}
}  // namespace

int geo_prism_nodes(int order, double* nodes, int64_t count) {
  if (order < 2 || order > 4 || !nodes) return fail(GEO_ERR_ARG, "geo_prism_nodes: bad arguments");
  std::vector<double> n, D;
  if (!geo::prism_element(order, n, D)) return fail(GEO_ERR_ARG, "geo_prism_nodes: singular basis");
  if (count < static_cast<int64_t>(n.size())) return fail(GEO_ERR_ARG, "geo_prism_nodes: host buffer too small");
  std::memcpy(nodes, n.data(), n.size() * sizeof(double));
  return GEO_OK;
}

int geo_time_matrix(int order, double* R, int64_t count) {
  if (order < 2 || order > 4 || !R) return fail(GEO_ERR_ARG, "geo_time_matrix: bad arguments");
  if (count < static_cast<int64_t>(order) * order) return fail(GEO_ERR_ARG, "geo_time_matrix: host buffer too small");
  std::vector<double> wt, r;
  geo::time_tables(order, wt, r);
  std::memcpy(R, r.data(), r.size() * sizeof(double));
  return GEO_OK;
}

int geo_prism_derivatives(int order, double* D, int64_t count) {
  if (order < 2 || order > 4 || !D) return fail(GEO_ERR_ARG, "geo_prism_derivatives: bad arguments");
  std::vector<double> n, d;
  if (!geo::prism_element(order, n, d)) return fail(GEO_ERR_ARG, "geo_prism_derivatives: singular basis");
  if (count < static_cast<int64_t>(d.size())) return fail(GEO_ERR_ARG, "geo_prism_derivatives: host buffer too small");
  std::memcpy(D, d.data(), d.size() * sizeof(double));
  return GEO_OK;
}

int geo_prism_predictor(int order, int64_t zones, const double* X_dev, const double* U_dev, double dt, double gamma,
                        double* Uh_dev, void* stream) {
  if (order < 2 || order > 4 || zones < 1 || !X_dev || !U_dev || !Uh_dev || !(dt > 0.0) || !(gamma > 1.0))
    return fail(GEO_ERR_ARG, "geo_prism_predictor: bad arguments");
  PrismTables& P = prism_tables_for(order);
  if (P.status != GEO_OK) return fail(P.status, P.err);
  cudaError_t e = geo::launch_prism_predictor_any(order, zones, P.Dv, P.Dc, P.R, X_dev, U_dev, dt, gamma, Uh_dev,
                                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "geo_prism_predictor");
  return GEO_OK;
}

int geo_probe_contraction(geo_mesh_t m, int tensor, int64_t zones, int reps, float* out_dev, float* ms) {
  if (!m || !out_dev || !ms || zones < 1 || reps < 1 || (tensor != 0 && tensor != 1))
    return fail(GEO_ERR_ARG, "geo_probe_contraction: bad arguments");
  if (m->prec != GEO_FP32_BULK) return fail(GEO_ERR_ARG, "geo_probe_contraction: needs a GEO_FP32_BULK mesh");
  if (zones > (int64_t(1) << 31) / 8) return fail(GEO_ERR_ARG, "geo_probe_contraction: too many zones");
  cudaError_t e = geo::probe_contraction_any(m->order, tensor, zones, reps, m->st, out_dev, ms);
  if (e != cudaSuccess) return cuda_fail(e, "geo_probe_contraction");
  return GEO_OK;
}

}  // extern "C"
