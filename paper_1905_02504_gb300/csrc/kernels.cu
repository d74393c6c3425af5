// CUDA kernels of one ADER-WENO-CT step (arXiv 1905.02504, Sec. VI).
//
// One thread per zone / face / edge.  Zones of a radial column share their
// tables (self-similar log shells, Sec. IV.b step 7 and Sec. V.b): zone (c, k)
// reads column c's tables and rescales lengths by q^k, areas by q^2k and
// volumes by q^3k.  Per-zone arrays are structure-of-arrays ([component][Z]) so
// consecutive threads touch consecutive addresses.
//
// Precision: the reconstruction, the predictor and the Riemann solvers run in
// the bulk type R (double for the FP64 form, float for the FP32-bulk form);
// the time-integrated face fluxes and edge EMFs are accumulated in FP64 and the
// updates of U and Phi are FP64 in both forms, so div B stays at FP64 rounding.
#include "device.cuh"
#include "probe.h"
#include "geomhd.h"
#include "host_tables.h"
#include "mhd_device.cuh"
#include "refpattern.h"  // generated at build time (refpattern.py)

#include <cfloat>
#include <utility>
#include <vector>

namespace geo {

__constant__ RefConst<2, double> c_ref2d;
__constant__ RefConst<3, double> c_ref3d;
__constant__ RefConst<4, double> c_ref4d;
__constant__ RefConst<2, float> c_ref2f;
__constant__ RefConst<3, float> c_ref3f;
__constant__ RefConst<4, float> c_ref4f;

template <int P, typename R> struct RC;
#define GEO_RC(P, R, SYM)                                                              \
  template <> struct RC<P, R> {                                                         \
    static __device__ __forceinline__ const RefConst<P, R>& get() { return SYM; }       \
    static const RefConst<P, R>& sym() { return SYM; }                                  \
  };
GEO_RC(2, double, c_ref2d)
GEO_RC(3, double, c_ref3d)
GEO_RC(4, double, c_ref4d)
GEO_RC(2, float, c_ref2f)
GEO_RC(3, float, c_ref3f)
GEO_RC(4, float, c_ref4f)
#undef GEO_RC

namespace {

using namespace dev;

// ----------------------------------------------------------------------------
// a1: WENO-AO reconstruction (Sec. III); one thread per zone and conserved
// variable (grid row y = variable)
// ----------------------------------------------------------------------------
template <int P, typename R>
__global__ void __launch_bounds__(TPB) k_weno(const DevTables T, const double* __restrict__ U,
                                              const float* __restrict__ Uhl, R* __restrict__ Wc) {
  using Dm = Dim<P>;
  constexpr int NC1 = Dm::NC1, SMAX = Dm::SMAX;
  const R GH = R(0.85), GK = R(0.15 / 8.0), EPS0 = R(1e-12);
  long long z = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (z >= T.Z) return;
  const BulkTables<R>& B = bulk<R>(T);
  const long long Z = T.Z;
  int nr = T.nr;
  int c = static_cast<int>(z / nr), k = static_cast<int>(z % nr);
  int ns = T.st_n[c];
  long long zs[SMAX];
  for (int j = 0; j < ns; ++j) {
    int pk = T.st_nb[c * SMAX + j];
    int cc = pk >> 3, dk = (pk & 7) - 3;
    int kk = min(max(k + dk, 0), nr - 1);
    zs[j] = static_cast<long long>(cc) * nr + kk;
  }
  long long zo[24];
#pragma unroll
  for (int j = 0; j < 24; ++j) {
    int pk = T.oct_nb[c * 24 + j];
    int cc = pk >> 3, dk = (pk & 7) - 3;
    int kk = min(max(k + dk, 0), nr - 1);
    zo[j] = static_cast<long long>(cc) * nr + kk;
  }
  const R* pinv = B.pinvH + static_cast<size_t>(c) * NC1 * SMAX;
  const R* oinv = B.oct_inv + static_cast<size_t>(c) * 72;
  const R* Qm = B.Q + static_cast<size_t>(c) * NC1 * NC1;
  {
    const int v = blockIdx.y;  // one conserved variable per grid row
    const double* Uv = U + v * Z;
    // zone-average differences U_j - U_0: in FP64 for the FP64 form; in the
    // FP32-bulk form from the hi/lo split, (hi_j - hi_0) + (lo_j - lo_0), which
    // carries the FP64 difference to FP32 rounding without FP64 arithmetic
    const float* Hv = Uhl ? Uhl + static_cast<size_t>(v) * Z : nullptr;
    const float* Lv = Uhl ? Uhl + static_cast<size_t>(8 + v) * Z : nullptr;
    const double u0d = (sizeof(R) == 8) ? Uv[z] : 0.0;
    const float h0 = (sizeof(R) == 4) ? Hv[z] : 0.f, l0 = (sizeof(R) == 4) ? Lv[z] : 0.f;
    // eps = eps_0 + K (l_0/r_0)^2 u_0^2 with K = 1 (Arandiga et al. 2011: eps ~ h^2)
    const R u0 = (sizeof(R) == 8) ? static_cast<R>(u0d) : static_cast<R>(h0);
    const R EPS = EPS0 + B.weta[c] * u0 * u0;
    auto diff = [&](long long zz) -> R {
      if constexpr (sizeof(R) == 4) return (Hv[zz] - h0) + (Lv[zz] - l0);
      else return static_cast<R>(Uv[zz] - u0d);
    };
    R uH[NC1];
#pragma unroll
    for (int m = 0; m < NC1; ++m) uH[m] = R(0);
    for (int j = 0; j < ns; ++j) {
      R du = diff(zs[j]);
#pragma unroll
      for (int m = 0; m < NC1; ++m) uH[m] += pinv[m * SMAX + j] * du;
    }
    R bH = R(0);
#pragma unroll
    for (int i = 0; i < NC1; ++i) {
      R s = R(0);
#pragma unroll
      for (int j = 0; j < NC1; ++j) s += Qm[i * NC1 + j] * uH[j];
      bH += uH[i] * s;
    }
    R uK[8][3], wK[8];
    R tau = R(0);
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      R d0 = diff(zo[3 * o]), d1 = diff(zo[3 * o + 1]), d2 = diff(zo[3 * o + 2]);
      const R* A = oinv + 9 * o;
#pragma unroll
      for (int a = 0; a < 3; ++a) uK[o][a] = A[3 * a] * d0 + A[3 * a + 1] * d1 + A[3 * a + 2] * d2;
      wK[o] = uK[o][0] * uK[o][0] + uK[o][1] * uK[o][1] + uK[o][2] * uK[o][2];  // beta_k for now
      tau += fabs(bH - wK[o]);
    }
    // WENO-Z type weights g (1 + (tau / (beta + eps))^2), tau = mean |beta_H - beta_k|
    // (Borges, Carmona, Costa & Don 2008), with the mesh-dependent eps above
    tau *= R(0.125);
    const R rH = tau / (bH + EPS);
    R wH = GH * (R(1) + rH * rH);
    R tot = wH;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const R r = tau / (wK[o] + EPS);
      wK[o] = GK * (R(1) + r * r);
      tot += wK[o];
    }
    R itot = R(1) / tot;
    wH *= itot;
    R fH = wH / GH;
    R* out = Wc + static_cast<size_t>(v) * NC1 * Z;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R sk = R(0), wk = R(0);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        sk += uK[o][a];
        wk += wK[o] * itot * uK[o][a];
      }
      out[a * Z + z] = fH * (uH[a] - GK * sk) + wk;
    }
#pragma unroll
    for (int m = 3; m < NC1; ++m) out[m * Z + z] = fH * uH[m];
  }
}

// ----------------------------------------------------------------------------
// a2 (face part): nodal normal fields by MinMod + mean shift (Eqs. 4.11-4.12)
// ----------------------------------------------------------------------------
template <int P, typename R>
__global__ void __launch_bounds__(TPB) k_bperp(const DevTables T, const double* __restrict__ U,
                                               const double* __restrict__ phi, const R* __restrict__ Wc,
                                               R* __restrict__ Bp) {
  using Dm = Dim<P>;
  constexpr int NC1 = Dm::NC1, NQT = Dm::NQT, NQMAX = (Dm::NQR > Dm::NQS ? Dm::NQR : Dm::NQS);
  long long f = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (f >= T.F) return;
  const BulkTables<R>& BT = bulk<R>(T);
  const long long Z = T.Z, F = T.F;
  FaceInfo fi = face_info(T, f);
  int nq = nq_of<P>(fi.lfg);
  // face mean <B_perp> = Phi / A with the tabulated reciprocal area
  const R mean = static_cast<R>(phi[f] * T.iA0[6 * fi.cg + fi.lfg] * T.iq2[fi.k]);
  const R gs = static_cast<R>(fi.gsign);
  int cL = fi.zL >= 0 ? static_cast<int>(fi.zL / T.nr) : -1;
  int cR = fi.zR >= 0 ? static_cast<int>(fi.zR / T.nr) : -1;
  // zone-mean B of both sides, converted once
  R UB[2][3];
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const long long zz = sd == 0 ? fi.zL : fi.zR;
#pragma unroll
    for (int d = 0; d < 3; ++d) UB[sd][d] = zz >= 0 ? static_cast<R>(U[(5 + d) * Z + zz]) : R(0);
  }
  R b[NQMAX];
  R wsum = R(0);
  for (int q = 0; q < nq; ++q) {
    int ig = foff<P>(fi.lfg) + q;
    const R* nv = BT.nF + (static_cast<size_t>(fi.cg) * NQT + ig) * 3;
    R nx = gs * nv[0], ny = gs * nv[1], nz = gs * nv[2];
    R bside[2];
    bool have[2] = {false, false};
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      long long zz = sd == 0 ? fi.zL : fi.zR;
      if (zz < 0) continue;
      int cc = sd == 0 ? cL : cR;
      int lf = sd == 0 ? fi.lfL : fi.lfR;
      int ql = q;
      if (sd == 1 && fi.se >= 0) ql = T.se_perm[fi.se * Dm::NQS + q];
      const R* tf = BT.TF + (static_cast<size_t>(cc) * NQT + foff<P>(lf) + ql) * NC1;
      R Bv[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        R s = UB[sd][d];
#pragma unroll
        for (int m = 0; m < NC1; ++m) s += tf[m] * Wc[((5 + d) * NC1 + m) * Z + zz];
        Bv[d] = s;
      }
      bside[sd] = nx * Bv[0] + ny * Bv[1] + nz * Bv[2];
      have[sd] = true;
    }
    if (!have[0]) bside[0] = bside[1];
    if (!have[1]) bside[1] = bside[0];
    b[q] = mean + minmod(bside[0] - mean, bside[1] - mean);
    wsum += BT.wF[static_cast<size_t>(fi.cg) * NQT + ig] * b[q];
  }
  R shift = mean - wsum;
  for (int q = 0; q < nq; ++q) Bp[static_cast<size_t>(q) * F + f] = b[q] + shift;
}

// ----------------------------------------------------------------------------
// a2 (zone part) + a3: divergence-free B (KKT apply) and the ADER predictor
// ----------------------------------------------------------------------------
// dF_i = sum_j sum_alpha D^alpha_ij F^alpha(U_j) - F(U_i).g_i, unscaled by dt (Eq. C.34
// with the geometric-conservation residual); D^alpha is walked in its sparse
// column form, so only the nonzero couplings of the serendipity element are formed.
template <int P, typename R>
__device__ void flux_difference(const DevTables& T, int c, const R (*Uh)[8], R (*dF)[8]) {
  using Dm = Dim<P>;
  constexpr int N = Dm::N;
  const RefConst<P, R>& K = RC<P, R>::get();
  const BulkTables<R>& B = bulk<R>(T);
  const R* iJ0 = B.iJ0 + static_cast<size_t>(c) * N;
  const R* Sm = B.Sm + static_cast<size_t>(c) * 9 * N;
  const R* gc = B.gcl + static_cast<size_t>(c) * N * 3;
  const R g = static_cast<R>(T.gamma);
#pragma unroll 1
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int v = 0; v < 8; ++v) dF[i][v] = R(0);
#pragma unroll 1
  for (int j = 0; j < N; ++j) {
    R u[8];
    const R iJ = iJ0[j];
#pragma unroll
    for (int v = 0; v < 8; ++v) u[v] = Uh[j][v] * iJ;
    Prim<R> w = to_prim(u, g);
    R Gj[8];
    flux_n(u, w, gc[3 * j], gc[3 * j + 1], gc[3 * j + 2], Gj);
#pragma unroll
    for (int v = 0; v < 8; ++v) dF[j][v] -= Gj[v];
#pragma unroll
    for (int al = 0; al < 3; ++al) {
      const R* s = Sm + (al * N + j) * 3;
      R Fa[8];
      flux_n(u, w, s[0], s[1], s[2], Fa);
      const int t0 = K.Dptr[al * (N + 1) + j], t1 = K.Dptr[al * (N + 1) + j + 1];
#pragma unroll 1
      for (int t = t0; t < t1; ++t) {
        const int i = K.Drow[al * Dm::NNZ + t];
        const R d = K.Dval[al * Dm::NNZ + t];
#pragma unroll
        for (int v = 0; v < 8; ++v) dF[i][v] += d * Fa[v];
      }
    }
  }
}

// POS: the positivity scaling of the nodal states (Sec. VI step 3) is compiled in only
// when the switch is on, so the plain predictor keeps its register budget
template <int P, typename R, bool POS>
__global__ void __launch_bounds__(TPB) k_ader(const DevTables T, double* __restrict__ U,
                                              const double* __restrict__ phi, const R* __restrict__ Wc,
                                              const R* __restrict__ Bp, R* __restrict__ trF,
                                              R* __restrict__ trE, double dt) {
  using Dm = Dim<P>;
  constexpr int N = Dm::N, M = Dm::M, NC1 = Dm::NC1, NC = Dm::NC, NQT = Dm::NQT, NS = Dm::NS,
                NBIN = Dm::NBIN;
  long long z = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (z >= T.Z) return;
  const BulkTables<R>& BT = bulk<R>(T);
  const RefConst<P, R>& K = RC<P, R>::get();
  const long long Z = T.Z, F = T.F;
  const int nr = T.nr;
  const int c = static_cast<int>(z / nr), k = static_cast<int>(z % nr);
  const double s1 = T.qpow[k];
  const double s2 = s1 * s1;
  // ---- inputs of the divergence-free reconstruction
  R in[NBIN];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    in[d * NC] = static_cast<R>(U[(5 + d) * Z + z]);
#pragma unroll
    for (int m = 0; m < NC1; ++m) in[d * NC + 1 + m] = Wc[((5 + d) * NC1 + m) * Z + z];
  }
#pragma unroll 1
  for (int lf = 0; lf < 6; ++lf) {
    long long f;
    int sg;
    int se = -1;
    if (lf < 4) {
      int sd = side_of_lf(lf);
      se = T.col_side_se[4 * c + sd];
      sg = T.col_side_sgn[4 * c + sd];
      f = T.F_rad + static_cast<long long>(se) * nr + k;
    } else {
      f = static_cast<long long>(c) * (nr + 1) + k + (lf == 5 ? 1 : 0);
      sg = lf == 5 ? 1 : -1;
    }
    const R rsg = static_cast<R>(sg);
    int nq = nq_of<P>(lf);
    for (int q = 0; q < nq; ++q) {
      int ql = q;
      if (lf < 4 && sg < 0) ql = T.se_perm[se * Dm::NQS + q];
      in[3 * NC + foff<P>(lf) + ql] = rsg * Bp[static_cast<size_t>(q) * F + f];
    }
    in[3 * NC + NQT + lf] = static_cast<R>(sg * phi[f] / (T.A0[6 * c + lf] * s2));
  }
  const R* GB = BT.GB + static_cast<size_t>(c) * (3 + 3 * N) * NBIN;
  R Uz[8];
#pragma unroll
  for (int v = 0; v < 5; ++v) Uz[v] = static_cast<R>(U[v * Z + z]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R s = R(0);
    for (int b = 0; b < NBIN; ++b) s += GB[b * (3 + 3 * N) + d] * in[b];
    Uz[5 + d] = s;
    U[(5 + d) * Z + z] = static_cast<double>(s);  // Sec. IV.b step 10: zone B <- divergence-free mean
  }
  // ---- initial nodal states U_hat_1 = J U(x_i)
  R Uh[M][N][8];
  const R* TN = BT.TN + static_cast<size_t>(c) * N * NC1;
  const R* J0 = BT.J0 + static_cast<size_t>(c) * N;
#pragma unroll 1
  for (int i = 0; i < N; ++i) {
    R u[8];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R s = Uz[v];
      for (int m = 0; m < NC1; ++m) s += TN[m * N + i] * Wc[(v * NC1 + m) * Z + z];
      u[v] = s;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      R s = R(0);
      for (int b = 0; b < NBIN; ++b) s += GB[b * (3 + 3 * N) + 3 + d * N + i] * in[b];
      u[5 + d] = s;
    }
    const R jf = POS ? R(1) : J0[i];
#pragma unroll
    for (int v = 0; v < 8; ++v) Uh[0][i][v] = jf * u[v];
  }
  if constexpr (POS) {
    const R gR = static_cast<R>(T.gamma);
    const R pbar = pressure_of(Uz, gR);
    const R eps_r = fmin(R(1e-13), Uz[0]), eps_p = fmin(R(1e-13), pbar);
    R th_r = R(1), th_p = R(1);
#pragma unroll 1
    for (int i = 0; i < N; ++i) pos_rho(Uh[0][i], Uz, eps_r, th_r);
#pragma unroll 1
    for (int i = 0; i < N; ++i) pos_p(Uh[0][i], Uz, th_r, gR, pbar, eps_p, th_p);
    const R th = th_r * th_p;
#pragma unroll 1
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const R uv = th < R(1) ? Uz[v] + th * (Uh[0][i][v] - Uz[v]) : Uh[0][i][v];
        Uh[0][i][v] = J0[i] * uv;
      }
  }
#pragma unroll 1
  for (int m = 1; m < M; ++m)
#pragma unroll 1
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int v = 0; v < 8; ++v) Uh[m][i][v] = Uh[0][i][v];
  // ---- Picard iterations (Eqs. C.34-C.36)
  const R fs = static_cast<R>(dt / s1);  // dt * l_0 / l_k (Eq. 5.21)
  R dF1[N][8];
  R dFm[M - 1][N][8];
  flux_difference<P, R>(T, c, Uh[0], dF1);
#pragma unroll 1
  for (int it = 0; it < P; ++it) {
    // in the first iteration every level still equals level 1, so its flux
    // difference is dF1 bit for bit
#pragma unroll 1
    for (int m = 1; m < M; ++m) {
      if (it == 0) {
#pragma unroll 1
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int v = 0; v < 8; ++v) dFm[m - 1][i][v] = dF1[i][v];
      } else {
        flux_difference<P, R>(T, c, Uh[m], dFm[m - 1]);
      }
    }
#pragma unroll 1
    for (int kk = 1; kk < M; ++kk) {
      R rk[M];
#pragma unroll
      for (int m = 0; m < M; ++m) rk[m] = fs * K.R_[kk * M + m];
#pragma unroll 1
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          R s = Uh[0][i][v] - rk[0] * dF1[i][v];
#pragma unroll
          for (int m = 1; m < M; ++m) s -= rk[m] * dFm[m - 1][i][v];
          Uh[kk][i][v] = s;
        }
    }
  }
  // ---- traces at the zone's face and edge points, Gauss times tau_2..tau_M;
  // a face (edge) point only sees the nodes of its face (edge)
  const R* JF = BT.JF + static_cast<size_t>(c) * NQT;
#pragma unroll 1
  for (int m = 1; m < M; ++m)
#pragma unroll 1
    for (int lf = 0; lf < 6; ++lf) {
      const int nq = nq_of<P>(lf), f0 = foff<P>(lf);
#pragma unroll 1
      for (int q = 0; q < nq; ++q) {
        const int idx = f0 + q;
        R acc[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[v] = R(0);
#pragma unroll
        for (int a = 0; a < Dm::NFN; ++a) {
          const R w = K.psiFc[idx * Dm::NFN + a];
          const int i = K.fnode[lf * Dm::NFN + a];
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[v] += w * Uh[m][i][v];
        }
        const R iJ = R(1) / JF[idx];
        R* out = trF + (static_cast<size_t>((m - 1) * NQT + idx) * 8) * Z + z;
#pragma unroll
        for (int v = 0; v < 8; ++v) out[v * Z] = acc[v] * iJ;
      }
    }
  const R* JE = BT.JE + static_cast<size_t>(c) * 12 * NS;
#pragma unroll 1
  for (int m = 1; m < M; ++m)
#pragma unroll 1
    for (int le = 0; le < 12; ++le)
#pragma unroll 1
      for (int s = 0; s < NS; ++s) {
        const int idx = le * NS + s;
        R acc[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[v] = R(0);
#pragma unroll
        for (int a = 0; a < Dm::NEN; ++a) {
          const R w = K.psiEc[idx * Dm::NEN + a];
          const int i = K.enode[le * Dm::NEN + a];
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[v] += w * Uh[m][i][v];
        }
        const R iJ = R(1) / JE[idx];
        R* out = trE + (static_cast<size_t>((m - 1) * 12 * NS + idx) * 8) * Z + z;
#pragma unroll
        for (int v = 0; v < 8; ++v) out[v * Z] = acc[v] * iJ;
      }
}

// Positivity scaling of the predicted face and edge point states (Sec. VI step 3):
// one theta per zone over all its traces at all Gauss times, about the zone mean
// (whose B the predictor has just replaced by the divergence-free mean).
template <int P, typename R>
__global__ void __launch_bounds__(TPB) k_pos_traces(const DevTables T, const double* __restrict__ U,
                                                    R* __restrict__ trF, R* __restrict__ trE) {
  using Dm = Dim<P>;
  constexpr int M = Dm::M, NQT = Dm::NQT, NS = Dm::NS;
  constexpr int NPF = (M - 1) * NQT, NPE = (M - 1) * 12 * NS;
  long long z = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (z >= T.Z) return;
  const long long Z = T.Z;
  R Uz[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) Uz[v] = static_cast<R>(U[v * Z + z]);
  const R gR = static_cast<R>(T.gamma);
  const R pbar = pressure_of(Uz, gR);
  const R eps_r = fmin(R(1e-13), Uz[0]), eps_p = fmin(R(1e-13), pbar);
  R th_r = R(1), th_p = R(1);
  for (int pass = 0; pass < 3; ++pass) {
    const R th = th_r * th_p;
    if (pass == 2 && !(th < R(1))) break;
#pragma unroll 1
    for (int t = 0; t < NPF + NPE; ++t) {
      R* base = (t < NPF) ? trF + (static_cast<size_t>(t) * 8) * Z + z
                          : trE + (static_cast<size_t>(t - NPF) * 8) * Z + z;
      R s[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) s[v] = base[v * Z];
      if (pass == 0) pos_rho(s, Uz, eps_r, th_r);
      else if (pass == 1) pos_p(s, Uz, th_r, gR, pbar, eps_p, th_p);
      else
#pragma unroll
        for (int v = 0; v < 8; ++v) base[v * Z] = Uz[v] + th * (s[v] - Uz[v]);
    }
  }
}


// ----------------------------------------------------------------------------
// a2 (zone part) + a3 with one thread per serendipity node: a team of N threads
// per zone, ZB zones per block.  Node i's M time levels and flux differences
// live in its thread's registers; at each flux evaluation the team exchanges
// the three metric fluxes of its nodes through shared memory and each thread
// gathers its own row of D^alpha (row form, RL entries).  Point values at the
// zone's face and edge points are then formed from the final levels in shared
// memory by threads mapped zone-fastest, so that the SoA trace writes of the ZB
// zones of a block are contiguous.
// ----------------------------------------------------------------------------
template <int P> struct Team;
template <> struct Team<2> { static constexpr int ZB = 16; };
template <> struct Team<3> { static constexpr int ZB = 8; };
template <> struct Team<4> { static constexpr int ZB = 4; };

// 8-vectors in shared memory are split into 16-byte chunks stored chunk-major,
// [alpha][chunk][node] within a zone.  Threads are mapped zone-fastest (thread =
// node * ZB + zone), so the 8 threads of a quarter warp, which share one 16-byte
// access phase, handle the same node (P = 2, 3) or two nodes (P = 4) of several
// zones; the per-zone stride XS is padded to 1 (2) modulo the 8 bank groups so
// that those zones' copies of one chunk sit in distinct bank groups.
template <typename R> struct Chunk { static constexpr int CH = 16 / sizeof(R), NCH = 8 / CH; };

template <typename R>
__device__ __forceinline__ void ld16(const R* p, R* out) {
  if constexpr (sizeof(R) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
  } else {
    const double2 q = *reinterpret_cast<const double2*>(p);
    out[0] = q.x; out[1] = q.y;
  }
}
template <typename R>
__device__ __forceinline__ void st16(R* p, const R* in) {
  if constexpr (sizeof(R) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(in[0], in[1], in[2], in[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(in[0], in[1]);
  }
}

template <int P, typename R>
struct TeamSmem {
  using Dm = Dim<P>;
  static constexpr int ZB = Team<P>::ZB, CH = Chunk<R>::CH, NCH = Chunk<R>::NCH;
  static constexpr int XS0 = 3 * NCH * Dm::N, XT = ZB >= 8 ? 1 : 2;
  static constexpr int XS = XS0 + ((XT - XS0 % 8) + 8) % 8;  // chunks per zone, XS % 8 == XT
  alignas(16) R X[ZB][XS][CH];       // fluxes of one level / the final levels
  R in[ZB][Dm::NBIN];                // inputs of the divergence-free reconstruction
  R W[ZB][5 * Dm::NC1];              // fluid Taylor coefficients
  R Uz[ZB][8];                       // zone means (B: the divergence-free mean)
  R Ev[3 * Dm::RL * Dm::N];
  R psiF[Dm::NQT * Dm::NFN];
  R psiE[12 * Dm::NS * Dm::NEN];
  R th[ZB][5];                       // positivity factors (min-reduced)
  R fs[ZB];                          // dt l_0 / l_k of the zone (Eq. 5.21)
  unsigned char Ec[3 * Dm::RL * Dm::N];
  unsigned char fnode[6 * Dm::NFN];
  unsigned char enode[12 * Dm::NEN];
};

// min-reduction of a non-negative factor in shared memory (the bit patterns of
// non-negative IEEE numbers order like the numbers)
__device__ __forceinline__ void smem_min_nonneg(float* a, float v) {
  atomicMin(reinterpret_cast<int*>(a), __float_as_int(v));
}
__device__ __forceinline__ void smem_min_nonneg(double* a, double v) {
  atomicMin(reinterpret_cast<unsigned long long*>(a), static_cast<unsigned long long>(__double_as_longlong(v)));
}

// FP32 order 3 runs at its register limit (5 blocks per SM): its column indices
// stay in shared memory
template <int P, typename R> struct EcInRegs { static constexpr bool value = !(P == 3 && sizeof(R) == 4); };

// one flux difference of node i of a team: dF = sum_alpha sum_j D^alpha_ij F^alpha_j - F_i . g_i;
// X is the zone's exchange buffer, chunk (alpha * NCH + c) * N + node
template <int P, typename R>
__device__ __forceinline__ void team_flux_difference(const R* Uh, R* dF, R iJ, const R* g, const R* Sa, R gam,
                                                     R (*X)[Chunk<R>::CH], const R* Ev, const unsigned char* Ec,
                                                     const unsigned* Ecr, int i, bool valid) {
  using Dm = Dim<P>;
  constexpr int N = Dm::N, RL = Dm::RL, CH = Chunk<R>::CH, NCH = Chunk<R>::NCH;
  if (valid) {
    R u[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) u[v] = Uh[v] * iJ;
    Prim<R> w = to_prim(u, gam);
    R G[8];
    flux_n(u, w, g[0], g[1], g[2], G);
#pragma unroll
    for (int v = 0; v < 8; ++v) dF[v] = -G[v];
#pragma unroll
    for (int al = 0; al < 3; ++al) {
      R Fa[8];
      flux_n(u, w, Sa[3 * al], Sa[3 * al + 1], Sa[3 * al + 2], Fa);
#pragma unroll
      for (int c = 0; c < NCH; ++c) st16(&X[(al * NCH + c) * N + i][0], &Fa[c * CH]);
    }
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
      for (int sl = 0; sl < RL; ++sl) {
        const R d = Ev[(al * RL + sl) * N + i];
        if (d != R(0)) {  // padding entries of short rows: no shared-memory traffic
          // column index: from registers (four per register, static shifts), or
          // from shared memory where the registers are needed elsewhere
          const int j = EcInRegs<P, R>::value ? (Ecr[(al * RL + sl) / 4] >> (8 * ((al * RL + sl) % 4))) & 0xff
                                              : Ec[(al * RL + sl) * N + i];
#pragma unroll
          for (int c = 0; c < NCH; ++c) {
            R f[CH];
            ld16(&X[(al * NCH + c) * N + j][0], f);
#pragma unroll
            for (int t = 0; t < CH; ++t) dF[c * CH + t] += d * f[t];
          }
        }
      }
  }
  __syncthreads();
}

// Zone inputs of a team block into shared memory: the WENO-AO coefficients,
// the zone means, the KKT right-hand side of the divergence-free reconstruction
// (zone B modes, nodal normal fields, face means; Sec. IV.b steps 5-8), then the
// zone-mean B of step 10 (written back to U) and the time-step factor dt / q^k.
// SM is any shared-memory struct with members in, W, Uz and fs per zone.  With
// WRITE_U false (the reverse sweep, which reads a pristine checkpoint) the
// zone-mean B is not written back.
template <int P, typename R, typename SM, bool WRITE_U = true>
__device__ __forceinline__ void team_load_inputs(SM& S, const DevTables& T, double* __restrict__ U,
                                                 const double* __restrict__ phi, const R* __restrict__ Wc,
                                                 const R* __restrict__ Bp, double dt, long long zbase, int tid) {
  using Dm = Dim<P>;
  constexpr int NC1 = Dm::NC1, NC = Dm::NC, NQT = Dm::NQT, NBIN = Dm::NBIN, NR = 3 + 3 * Dm::N,
                ZB = Team<P>::ZB, NT = ZB * Dm::N;
  const BulkTables<R>& BT = bulk<R>(T);
  const long long Z = T.Z, F = T.F;
  const int nr = T.nr;
  for (int w = tid; w < ZB * 3 * NC; w += NT) {
    const int zl = w % ZB, e = w / ZB, d = e / NC, t = e % NC;
    const long long z = zbase + zl;
    if (z < Z) S.in[zl][e] = (t == 0) ? static_cast<R>(U[(5 + d) * Z + z]) : Wc[((5 + d) * NC1 + t - 1) * Z + z];
  }
  for (int w = tid; w < ZB * 5 * NC1; w += NT) {
    const int zl = w % ZB, e = w / ZB;
    const long long z = zbase + zl;
    if (z < Z) S.W[zl][e] = Wc[static_cast<size_t>(e) * Z + z];
  }
  for (int w = tid; w < ZB * 5; w += NT) {
    const int zl = w % ZB, v = w / ZB;
    const long long z = zbase + zl;
    if (z < Z) S.Uz[zl][v] = static_cast<R>(U[v * Z + z]);
  }
  for (int w = tid; w < ZB * 6; w += NT) {
    const int zl = w % ZB, lf = w / ZB;
    const long long z = zbase + zl;
    if (z >= Z) continue;
    const int c = static_cast<int>(z / nr), k = static_cast<int>(z % nr);
    long long f;
    int sg, se = -1;
    if (lf < 4) {
      const int sd = side_of_lf(lf);
      se = T.col_side_se[4 * c + sd];
      sg = T.col_side_sgn[4 * c + sd];
      f = T.F_rad + static_cast<long long>(se) * nr + k;
    } else {
      f = static_cast<long long>(c) * (nr + 1) + k + (lf == 5 ? 1 : 0);
      sg = lf == 5 ? 1 : -1;
    }
    const R rsg = static_cast<R>(sg);
    const int nq = nq_of<P>(lf);
    for (int q = 0; q < nq; ++q) {
      const int ql = (lf < 4 && sg < 0) ? T.se_perm[se * Dm::NQS + q] : q;
      S.in[zl][3 * NC + foff<P>(lf) + ql] = rsg * Bp[static_cast<size_t>(q) * F + f];
    }
    // face mean <B_perp> = Phi / A with the tabulated reciprocal area (no FP64 division)
    S.in[zl][3 * NC + NQT + lf] = static_cast<R>(sg * phi[f] * T.iA0[6 * c + lf] * T.iq2[k]);
  }
  __syncthreads();
  // ---- zone-mean B (Sec. IV.b step 10)
  if (tid < 3 * ZB) {
    const int zl = tid % ZB, d = tid / ZB;
    const long long z = zbase + zl;
    if (z < Z) {
      const int c = static_cast<int>(z / nr);
      const R* GB = BT.GB + static_cast<size_t>(c) * NR * NBIN;
      R s = R(0);
      for (int b = 0; b < NBIN; ++b) s += GB[b * NR + d] * S.in[zl][b];
      S.Uz[zl][5 + d] = s;
      if constexpr (WRITE_U) U[(5 + d) * Z + z] = static_cast<double>(s);
      if (d == 0) S.fs[zl] = static_cast<R>(dt / T.qpow[z % nr]);  // one FP64 division per zone
    }
  }
  __syncthreads();
}

// Reconstructed conserved values at node i of zone zl (Sec. V.d steps 5-6): the
// fluid variables from the WENO-AO Taylor coefficients, B from the
// divergence-free KKT solution; u = 1 for the padding threads of a partial block.
template <int P, typename R, typename SM>
__device__ __forceinline__ void team_nodal_values(const SM& S, const BulkTables<R>& BT, int c, int i, int zl,
                                                  bool valid, R* u) {
  using Dm = Dim<P>;
  constexpr int N = Dm::N, NC1 = Dm::NC1, NBIN = Dm::NBIN, NR = 3 + 3 * Dm::N;
  if (valid) {
    const R* TN = BT.TN + static_cast<size_t>(c) * N * NC1;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R s = S.Uz[zl][v];
      for (int m = 0; m < NC1; ++m) s += TN[m * N + i] * S.W[zl][v * NC1 + m];
      u[v] = s;
    }
    const R* GB = BT.GB + static_cast<size_t>(c) * NR * NBIN;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      R s = R(0);
      for (int b = 0; b < NBIN; ++b) s += GB[b * NR + 3 + d * N + i] * S.in[zl][b];
      u[5 + d] = s;
    }
  } else {
#pragma unroll
    for (int v = 0; v < 8; ++v) u[v] = R(1);
  }
}

// Metric terms of node i (Eqs. 5.5-5.11): 1/J, the discrete GCL residual g_i and
// the three contravariant area vectors S^alpha (zeros for padding threads).
template <int P, typename R>
__device__ __forceinline__ void team_node_metrics(const BulkTables<R>& BT, int c, int i, bool valid, R& iJ,
                                                  R* g, R* Sa) {
  constexpr int N = Dim<P>::N;
  iJ = R(1);
#pragma unroll
  for (int t = 0; t < 3; ++t) g[t] = R(0);
#pragma unroll
  for (int t = 0; t < 9; ++t) Sa[t] = R(0);
  if (valid) {
    iJ = BT.iJ0[static_cast<size_t>(c) * N + i];
    const R* gc = BT.gcl + (static_cast<size_t>(c) * N + i) * 3;
#pragma unroll
    for (int t = 0; t < 3; ++t) g[t] = gc[t];
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
      for (int t = 0; t < 3; ++t) Sa[3 * al + t] = BT.Sm[static_cast<size_t>(c) * 9 * N + (al * N + i) * 3 + t];
  }
}

// resident blocks per SM the register budget is sized for
template <int P, typename R> struct TeamOcc;
template <> struct TeamOcc<2, float> { static constexpr int MINB = 8; };   // 128 threads
template <> struct TeamOcc<3, float> { static constexpr int MINB = 5; };   // 160 threads (72 registers, a few spilled)
template <> struct TeamOcc<4, float> { static constexpr int MINB = 4; };   // 128 threads (128 registers, a few spilled)
template <> struct TeamOcc<2, double> { static constexpr int MINB = 4; };
template <> struct TeamOcc<3, double> { static constexpr int MINB = 2; };
template <> struct TeamOcc<4, double> { static constexpr int MINB = 2; };

// STORE: also write the levels after each of the first P-1 Picard iterations to
// itS ([P-1][M-1][8][N][Z]), the linearisation points of the reverse sweep
template <int P, typename R, bool POS, bool STORE = false>
__global__ void __launch_bounds__(Team<P>::ZB * Dim<P>::N, TeamOcc<P, R>::MINB)
    k_ader_team(const DevTables T, double* __restrict__ U, const double* __restrict__ phi,
                const R* __restrict__ Wc, const R* __restrict__ Bp, R* __restrict__ trF, R* __restrict__ trE,
                double dt, R* __restrict__ itS) {
  using Dm = Dim<P>;
  constexpr int N = Dm::N, M = Dm::M, NC1 = Dm::NC1, NC = Dm::NC, NQT = Dm::NQT, NS = Dm::NS,
                NBIN = Dm::NBIN, NR = 3 + 3 * Dm::N, ZB = Team<P>::ZB, NT = ZB * N;
  __shared__ TeamSmem<P, R> S;
  const RefConst<P, R>& K = RC<P, R>::get();
  const BulkTables<R>& BT = bulk<R>(T);
  const long long Z = T.Z, F = T.F;
  const int nr = T.nr;
  const int tid = threadIdx.x;
  const long long zbase = static_cast<long long>(blockIdx.x) * ZB;
  // ---- reference tables and zone inputs into shared memory
  for (int t = tid; t < 3 * Dm::RL * N; t += NT) {
    S.Ev[t] = K.Eval[t];
    S.Ec[t] = K.Ecol[t];
  }
  for (int t = tid; t < NQT * Dm::NFN; t += NT) S.psiF[t] = K.psiFc[t];
  for (int t = tid; t < 6 * Dm::NFN; t += NT) S.fnode[t] = K.fnode[t];
  for (int t = tid; t < 12 * NS * Dm::NEN; t += NT) S.psiE[t] = K.psiEc[t];
  for (int t = tid; t < 12 * Dm::NEN; t += NT) S.enode[t] = K.enode[t];
  for (int w = tid; w < ZB * 5; w += NT) S.th[w / 5][w % 5] = R(1);
  team_load_inputs<P, R>(S, T, U, phi, Wc, Bp, dt, zbase, tid);
  // ---- node of this thread (zone-fastest mapping)
  const int zl = tid % ZB, i = tid / ZB;
  const long long z = zbase + zl;
  const bool valid = z < Z;
  const int c = valid ? static_cast<int>(z / nr) : 0;
  const R gam = static_cast<R>(T.gamma);
  R Uh[M][8];
  {
    R u[8];
    team_nodal_values<P, R>(S, BT, c, i, zl, valid, u);
    if constexpr (POS) {
      const R* Uz = S.Uz[zl];
      const R pbar = pressure_of(Uz, gam);
      const R eps_r = fmin(R(1e-13), Uz[0]), eps_p = fmin(R(1e-13), pbar);
      R th_r = R(1), th_p = R(1);
      pos_rho(u, Uz, eps_r, th_r);
      if (valid && th_r < R(1)) smem_min_nonneg(&S.th[zl][0], th_r);
      __syncthreads();
      th_r = S.th[zl][0];
      pos_p(u, Uz, th_r, gam, pbar, eps_p, th_p);
      if (valid && th_p < R(1)) smem_min_nonneg(&S.th[zl][1], th_p);
      __syncthreads();
      const R th = th_r * S.th[zl][1];
      if (th < R(1)) {
#pragma unroll
        for (int v = 0; v < 8; ++v) u[v] = Uz[v] + th * (u[v] - Uz[v]);
      }
    }
    const R j0 = valid ? BT.J0[static_cast<size_t>(c) * N + i] : R(1);
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int v = 0; v < 8; ++v) Uh[m][v] = j0 * u[v];
  }
  // ---- metric terms of the node, kept for all flux evaluations
  R iJ, g[3], Sa[9];
  team_node_metrics<P, R>(BT, c, i, valid, iJ, g, Sa);
  // ---- Picard iterations (Eqs. C.34-C.36); in the first iteration every level
  // equals level 1, so its flux difference is reused
  const R fs = S.fs[zl];
  constexpr int CH = Chunk<R>::CH, NCH = Chunk<R>::NCH;
  R (*X)[CH] = S.X[zl];
  // the node's row of every D^alpha: values stay in shared memory, the column
  // indices are packed into registers once
  constexpr int NEC = (3 * Dm::RL + 3) / 4;
  unsigned Ecr[NEC];
#pragma unroll
  for (int t = 0; t < NEC; ++t) Ecr[t] = 0u;
  if constexpr (EcInRegs<P, R>::value) {
#pragma unroll
    for (int t = 0; t < 3 * Dm::RL; ++t) Ecr[t / 4] |= static_cast<unsigned>(S.Ec[t * N + i]) << (8 * (t % 4));
  }
  R dF[M][8];
  team_flux_difference<P, R>(Uh[0], dF[0], iJ, g, Sa, gam, X, S.Ev, S.Ec, Ecr, i, valid);
#pragma unroll
  for (int m = 1; m < M; ++m)
#pragma unroll
    for (int v = 0; v < 8; ++v) dF[m][v] = dF[0][v];
#pragma unroll 1
  for (int it = 0; it < P; ++it) {
    if (it > 0) {
#pragma unroll
      for (int m = 1; m < M; ++m) team_flux_difference<P, R>(Uh[m], dF[m], iJ, g, Sa, gam, X, S.Ev, S.Ec, Ecr, i, valid);
    }
#pragma unroll
    for (int kk = 1; kk < M; ++kk) {
      R rk[M];
#pragma unroll
      for (int m = 0; m < M; ++m) rk[m] = fs * K.R_[kk * M + m];
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        R s = Uh[0][v] - rk[0] * dF[0][v];
#pragma unroll
        for (int m = 1; m < M; ++m) s -= rk[m] * dF[m][v];
        Uh[kk][v] = s;
      }
      if constexpr (STORE) {
        if (it < P - 1 && valid) {
#pragma unroll
          for (int v = 0; v < 8; ++v) itS[((static_cast<size_t>(it * (M - 1) + kk - 1) * 8 + v) * N + i) * Z + z] = Uh[kk][v];
        }
      }
    }
  }
  // ---- final levels to shared memory (the exchange buffer is free after the
  // last flux difference's closing barrier)
#pragma unroll
  for (int m = 1; m < M; ++m)
#pragma unroll
    for (int c = 0; c < NCH; ++c) st16(&X[((m - 1) * NCH + c) * N + i][0], &Uh[m][c * CH]);
  __syncthreads();
  // ---- point values; thread -> (zone zl2 = tid % ZB, point slots tid / ZB + N s)
  {
    constexpr int NPF = (M - 1) * NQT, NPE = (M - 1) * 12 * NS, NPT = NPF + NPE;
    const int zl2 = tid % ZB;
    const long long z2 = zbase + zl2;
    const bool valid2 = z2 < Z;
    const int c2 = valid2 ? static_cast<int>(z2 / nr) : 0;
    const R* JF = BT.JF + static_cast<size_t>(c2) * NQT;
    const R* JE = BT.JE + static_cast<size_t>(c2) * 12 * NS;
    const R(*X2)[CH] = S.X[zl2];
    const R* Uz = S.Uz[zl2];
    // with positivity: pass 0 writes the unscaled values and min-reduces theta_rho
    // and the pressure factor for theta_rho = 1; pass 1 (only if some zone of the
    // block has theta_rho < 1) recomputes the pressure factor of those zones; pass 2
    // (only if some zone has theta < 1) rewrites those zones' values scaled
    constexpr int NPASS = POS ? 3 : 1;
    R pbar = R(0), eps_r = R(0), eps_p = R(0), th = R(1);
    bool redo = true;  // this zone takes part in the current pass
    if constexpr (POS) {
      pbar = pressure_of(Uz, gam);
      eps_r = fmin(R(1e-13), Uz[0]);
      eps_p = fmin(R(1e-13), pbar);
    }
#pragma unroll 1
    for (int pass = 0; pass < NPASS; ++pass) {
      if constexpr (POS) {
        if (pass == 1) {
          redo = valid2 && S.th[zl2][2] < R(1);
          if (!__syncthreads_or(redo)) continue;  // block-uniform
        }
        if (pass == 2) {
          const R thp = S.th[zl2][2] < R(1) ? S.th[zl2][3] : S.th[zl2][4];
          th = S.th[zl2][2] * thp;
          redo = valid2 && th < R(1);
          if (!__syncthreads_or(redo)) continue;  // block-uniform
        }
      }
#pragma unroll 1
      for (int t = tid / ZB; t < NPT; t += N) {
        if (!redo) break;
        R s[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) s[v] = R(0);
        R* out;
        if (t < NPF) {
          const int m = t / NQT, idx = t % NQT;
          const int lf = idx < 4 * Dm::NQS ? idx / Dm::NQS : 4 + (idx - 4 * Dm::NQS) / Dm::NQR;
#pragma unroll
          for (int a = 0; a < Dm::NFN; ++a) {
            const R w = S.psiF[idx * Dm::NFN + a];
            const int nd = S.fnode[lf * Dm::NFN + a];
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
              R x[CH];
              ld16(&X2[(m * NCH + c) * N + nd][0], x);
#pragma unroll
              for (int t = 0; t < CH; ++t) s[c * CH + t] += w * x[t];
            }
          }
          const R ij = valid2 ? R(1) / JF[idx] : R(1);
#pragma unroll
          for (int v = 0; v < 8; ++v) s[v] *= ij;
          out = trF + (static_cast<size_t>(t) * 8) * Z + z2;
        } else {
          const int tt = t - NPF, m = tt / (12 * NS), idx = tt % (12 * NS), le = idx / NS;
#pragma unroll
          for (int a = 0; a < Dm::NEN; ++a) {
            const R w = S.psiE[idx * Dm::NEN + a];
            const int nd = S.enode[le * Dm::NEN + a];
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
              R x[CH];
              ld16(&X2[(m * NCH + c) * N + nd][0], x);
#pragma unroll
              for (int t = 0; t < CH; ++t) s[c * CH + t] += w * x[t];
            }
          }
          const R ij = valid2 ? R(1) / JE[idx] : R(1);
#pragma unroll
          for (int v = 0; v < 8; ++v) s[v] *= ij;
          out = trE + (static_cast<size_t>(tt) * 8) * Z + z2;
        }
        if (!valid2) continue;
        if constexpr (POS) {
          if (pass == 0) {
            R th_r = R(1), th_p1 = R(1);
            pos_rho(s, Uz, eps_r, th_r);
            if (th_r < R(1)) smem_min_nonneg(&S.th[zl2][2], th_r);
            pos_p(s, Uz, R(1), gam, pbar, eps_p, th_p1);
            if (th_p1 < R(1)) smem_min_nonneg(&S.th[zl2][4], th_p1);
          } else if (pass == 1) {
            R th_p = R(1);
            pos_p(s, Uz, S.th[zl2][2], gam, pbar, eps_p, th_p);
            if (th_p < R(1)) smem_min_nonneg(&S.th[zl2][3], th_p);
            continue;
          } else {
#pragma unroll
            for (int v = 0; v < 8; ++v) s[v] = Uz[v] + th * (s[v] - Uz[v]);
          }
        }
#pragma unroll
        for (int v = 0; v < 8; ++v) out[v * Z] = s[v];
      }
      if constexpr (POS) __syncthreads();
    }
  }
}

#include "ader_vt.cuh"

// ----------------------------------------------------------------------------
// a4: face fluxes (HLL at face points x Gauss times, FP64 accumulation)
// ----------------------------------------------------------------------------
template <int P, typename R, bool HLLD>
__global__ void __launch_bounds__(TPB) k_face_flux(const DevTables T, const R* __restrict__ trF,
                                                   double* __restrict__ Ff, double dt) {
  using Dm = Dim<P>;
  constexpr int M = Dm::M, NQT = Dm::NQT;
  long long f = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (f >= T.F) return;
  const BulkTables<R>& BT = bulk<R>(T);
  const long long Z = T.Z, F = T.F;
  FaceInfo fi = face_info(T, f);
  int nq = nq_of<P>(fi.lfg);
  double s2 = T.qpow[fi.k] * T.qpow[fi.k];
  const R gs = static_cast<R>(fi.gsign);
  const R g = static_cast<R>(T.gamma);
  // quadrature sum over the face's points and Gauss times in the bulk type (the
  // zone update that sums the faces is FP64)
  R acc[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) acc[v] = R(0);
#pragma unroll 1
  for (int m = 1; m < M; ++m) {
    double wt = T.wt[m - 1];
#pragma unroll 1
    for (int q = 0; q < nq; ++q) {
      int ig = foff<P>(fi.lfg) + q;
      const R* nv = BT.nF + (static_cast<size_t>(fi.cg) * NQT + ig) * 3;
      R nx = gs * nv[0], ny = gs * nv[1], nz = gs * nv[2];
      const R W = static_cast<R>(wt * T.WF[static_cast<size_t>(fi.cg) * NQT + ig] * s2);
      R uL[8], uR[8];
      if (fi.zL >= 0) {
        const R* src = trF + trF_at<P>(fi.zL, m, foff<P>(fi.lfL) + q, Z);
#pragma unroll
        for (int v = 0; v < 8; ++v) uL[v] = src[v * Z];
      }
      if (fi.zR >= 0) {
        int ql = q;
        if (fi.se >= 0) ql = T.se_perm[fi.se * Dm::NQS + q];
        const R* src = trF + trF_at<P>(fi.zR, m, foff<P>(fi.lfR) + ql, Z);
#pragma unroll
        for (int v = 0; v < 8; ++v) uR[v] = src[v * Z];
      }
      if (fi.zL < 0) {
#pragma unroll
        for (int v = 0; v < 8; ++v) uL[v] = uR[v];
      }
      if (fi.zR < 0) {
#pragma unroll
        for (int v = 0; v < 8; ++v) uR[v] = uL[v];
      }
      if constexpr (HLLD) hlld_acc(uL, uR, nx, ny, nz, g, W, acc);
      else hll_acc(uL, uR, nx, ny, nz, g, W, acc);
    }
  }
#pragma unroll
  for (int v = 0; v < 8; ++v) Ff[v * F + f] = dt * static_cast<double>(acc[v]);
}

// ----------------------------------------------------------------------------
// a5: edge EMFs (multidimensional Rusanov at edge points x Gauss times, FP64
// accumulation)
// ----------------------------------------------------------------------------
template <int P, typename R>
__global__ void __launch_bounds__(TPB) k_edge_emf(const DevTables T, const R* __restrict__ trE,
                                                  double* __restrict__ Ee, double dt) {
  using Dm = Dim<P>;
  constexpr int M = Dm::M, NS = Dm::NS;
  long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= T.E) return;
  const long long Z = T.Z;
  const int nr = T.nr;
  const R g = static_cast<R>(T.gamma);
  long long zs[4];
  int les[4], revs[4];
  int nz = 0, nf = 0;
  int fL[4], fR[4];
  const BulkTables<R>& BT = bulk<R>(T);
  const R* fn[4];  // normals [NS][3] of each face
  R tv[NS][3], dlw[NS];
  if (e < T.E_rad) {
    int sv = static_cast<int>(e / nr), k = static_cast<int>(e % nr);
    nz = T.sv_nc[sv];
    nf = nz;
    for (int j = 0; j < nz; ++j) {
      zs[j] = static_cast<long long>(T.sv_col[4 * sv + j]) * nr + k;
      les[j] = T.sv_le[4 * sv + j];
      revs[j] = 0;
      fL[j] = T.sv_fL[4 * sv + j];
      fR[j] = T.sv_fR[4 * sv + j];
      fn[j] = BT.sv_fn + static_cast<size_t>(sv * 4 + j) * NS * 3;
    }
    for (int s = 0; s < NS; ++s) {
      for (int a = 0; a < 3; ++a) tv[s][a] = BT.sv_t[3 * sv + a];
      dlw[s] = static_cast<R>(T.sv_dlw[sv * NS + s] * T.qpow[k]);
    }
  } else {
    long long r = e - T.E_rad;
    int se = static_cast<int>(r / (nr + 1)), kk = static_cast<int>(r % (nr + 1));
    int cL = T.se_col[2 * se], cR = T.se_col[2 * se + 1];
    int revL = T.se_rev[2 * se], revR = T.se_rev[2 * se + 1];
    const R* nang = BT.se_nang + static_cast<size_t>(se) * NS * 3;
    if (kk >= 1 && kk <= nr - 1) {
      nz = 4;
      zs[0] = static_cast<long long>(cL) * nr + kk - 1; les[0] = T.se_le[(2 * se) * 2 + 1]; revs[0] = revL;
      zs[1] = static_cast<long long>(cL) * nr + kk;     les[1] = T.se_le[(2 * se) * 2 + 0]; revs[1] = revL;
      zs[2] = static_cast<long long>(cR) * nr + kk - 1; les[2] = T.se_le[(2 * se + 1) * 2 + 1]; revs[2] = revR;
      zs[3] = static_cast<long long>(cR) * nr + kk;     les[3] = T.se_le[(2 * se + 1) * 2 + 0]; revs[3] = revR;
      nf = 4;
      fL[0] = 0; fR[0] = 2; fn[0] = nang;
      fL[1] = 1; fR[1] = 3; fn[1] = nang;
      fL[2] = 0; fR[2] = 1; fn[2] = BT.se_nradL + static_cast<size_t>(se) * NS * 3;
      fL[3] = 2; fR[3] = 3; fn[3] = BT.se_nradR + static_cast<size_t>(se) * NS * 3;
    } else {
      nz = 2;
      int top = (kk == nr) ? 1 : 0;
      int kz = top ? nr - 1 : 0;
      zs[0] = static_cast<long long>(cL) * nr + kz; les[0] = T.se_le[(2 * se) * 2 + top]; revs[0] = revL;
      zs[1] = static_cast<long long>(cR) * nr + kz; les[1] = T.se_le[(2 * se + 1) * 2 + top]; revs[1] = revR;
      nf = 1;
      fL[0] = 0; fR[0] = 1; fn[0] = nang;
    }
    for (int s = 0; s < NS; ++s) {
      for (int a = 0; a < 3; ++a) tv[s][a] = BT.se_t[(static_cast<size_t>(se) * NS + s) * 3 + a];
      dlw[s] = static_cast<R>(T.se_dlw[se * NS + s] * T.qpow[kk]);
    }
  }
  const R inz = R(1) / static_cast<R>(nz);
  R acc = R(0);  // quadrature sum in the bulk type; the Phi update is FP64
#pragma unroll 1
  for (int m = 1; m < M; ++m) {
    const R wt = static_cast<R>(T.wt[m - 1]);
#pragma unroll 1
    for (int s = 0; s < NS; ++s) {
      // primitive state of each zone at the point, 1/rho formed once per zone
      // (register arrays: every index below is static or goes through sel4)
      R ir[4], vx[4], vy[4], vz[4], pr[4], bx[4], by[4], bz[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        R u[8] = {R(1), R(0), R(0), R(0), R(1), R(0), R(0), R(0)};
        if (j < nz) {
          const int sl = revs[j] ? NS - 1 - s : s;
          const R* src = trE + trE_at<P>(zs[j], m, les[j] * NS + sl, Z);
#pragma unroll
          for (int v = 0; v < 8; ++v) u[v] = src[v * Z];
        }
        const Prim<R> w = to_prim(u, g);
        ir[j] = R(1) / u[0];
        vx[j] = w.vx; vy[j] = w.vy; vz[j] = w.vz; pr[j] = w.p;
        bx[j] = w.bx; by[j] = w.by; bz[j] = w.bz;
      }
      R tx = tv[s][0], ty = tv[s][1], tz = tv[s][2];
      R E = R(0);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        // (-v x B) . t
        if (j < nz)
          E -= (vy[j] * bz[j] - vz[j] * by[j]) * tx + (vz[j] * bx[j] - vx[j] * bz[j]) * ty +
               (vx[j] * by[j] - vy[j] * bx[j]) * tz;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j >= nf) continue;
        const R* nvd = fn[j] + 3 * s;
        R nx = nvd[0], ny = nvd[1], nzz = nvd[2];
        const int qL = fL[j], qR = fR[j];
        R a = fmax(rusanov_speed_ir(sel4(ir, qL), sel4(vx, qL), sel4(vy, qL), sel4(vz, qL), sel4(pr, qL),
                                    sel4(bx, qL), sel4(by, qL), sel4(bz, qL), nx, ny, nzz, g),
                   rusanov_speed_ir(sel4(ir, qR), sel4(vx, qR), sel4(vy, qR), sel4(vz, qR), sel4(pr, qR),
                                    sel4(bx, qR), sel4(by, qR), sel4(bz, qR), nx, ny, nzz, g));
        // t x n
        R cx = ty * nzz - tz * ny, cy = tz * nx - tx * nzz, cz = tx * ny - ty * nx;
        R dbx = sel4(bx, qR) - sel4(bx, qL), dby = sel4(by, qR) - sel4(by, qL), dbz = sel4(bz, qR) - sel4(bz, qL);
        E += a * (dbx * cx + dby * cy + dbz * cz);
      }
      acc += wt * dlw[s] * (E * inz);
    }
  }
  Ee[e] = dt * static_cast<double>(acc);
}

// ----------------------------------------------------------------------------
// a6: conservative and constrained-transport updates
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(TPB) k_update_u(const DevTables T, double* __restrict__ U,
                                                  const double* __restrict__ Ff, float* __restrict__ Uhl) {
  long long z = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (z >= T.Z) return;
  const long long Z = T.Z, F = T.F;
  const int nr = T.nr;
  int c = static_cast<int>(z / nr), k = static_cast<int>(z % nr);
  double s1 = T.qpow[k];
  double iV = 1.0 / (T.V0[c] * s1 * s1 * s1);
  double acc[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) acc[v] = 0.0;
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) {
    long long f;
    double sg;
    if (lf < 4) {
      int sd = side_of_lf(lf);
      f = T.F_rad + static_cast<long long>(T.col_side_se[4 * c + sd]) * nr + k;
      sg = T.col_side_sgn[4 * c + sd];
    } else {
      f = static_cast<long long>(c) * (nr + 1) + k + (lf == 5 ? 1 : 0);
      sg = lf == 5 ? 1.0 : -1.0;
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[v] += sg * Ff[v * F + f];
  }
  double u[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    u[v] = U[v * Z + z] - iV * acc[v];
    U[v * Z + z] = u[v];
    if (Uhl) {
      const float hi = static_cast<float>(u[v]);
      Uhl[v * Z + z] = hi;
      Uhl[(8 + v) * Z + z] = static_cast<float>(u[v] - static_cast<double>(hi));
    }
  }
  // physical-state flag (read by the host between steps)
  const double p = pressure_of(u, T.gamma);
  if (!(u[0] > 0.0) || !(p > 0.0) || !isfinite(u[4])) atomicOr(T.status, 1);
}

__global__ void __launch_bounds__(TPB) k_split_u(const DevTables T, const double* __restrict__ U,
                                                 float* __restrict__ Uhl) {
  long long z = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (z >= T.Z) return;
  const long long Z = T.Z;
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const double u = U[v * Z + z];
    const float hi = static_cast<float>(u);
    Uhl[v * Z + z] = hi;
    Uhl[(8 + v) * Z + z] = static_cast<float>(u - static_cast<double>(hi));
  }
}

__global__ void __launch_bounds__(TPB) k_update_phi(const DevTables T, double* __restrict__ phi,
                                                    const double* __restrict__ Ee) {
  long long f = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (f >= T.F) return;
  const int nr = T.nr;
  double s;
  if (f < T.F_rad) {
    int c = static_cast<int>(f / (nr + 1)), k = static_cast<int>(f % (nr + 1));
    s = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      s += T.col_side_sgn[4 * c + q] * Ee[T.E_rad + static_cast<long long>(T.col_side_se[4 * c + q]) * (nr + 1) + k];
  } else {
    long long r = f - T.F_rad;
    int se = static_cast<int>(r / nr), k = static_cast<int>(r % nr);
    long long base = T.E_rad + static_cast<long long>(se) * (nr + 1);
    s = Ee[base + k] + Ee[static_cast<long long>(T.se_v[2 * se + 1]) * nr + k] - Ee[base + k + 1] -
        Ee[static_cast<long long>(T.se_v[2 * se]) * nr + k];
  }
  phi[f] -= s;
}

// ----------------------------------------------------------------------------
// a8 / a9: CFL time step and div B (deterministic two-pass reductions)
// ----------------------------------------------------------------------------
constexpr int RED_TPB = 256;

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void __launch_bounds__(RED_TPB) k_cfl_partial(const DevTables T, const double* __restrict__ U,
                                                         double* __restrict__ part) {
  __shared__ double sm[RED_TPB / 32];
  const long long Z = T.Z;
  const int nr = T.nr;
  double best = DBL_MAX;
  for (long long z = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; z < Z;
       z += static_cast<long long>(gridDim.x) * blockDim.x) {
    double u[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) u[v] = U[v * Z + z];
    Prim w = to_prim(u, T.gamma);
    double cf = sqrt(T.gamma * w.p / w.rho + (w.bx * w.bx + w.by * w.by + w.bz * w.bz) / w.rho);
    double vm = sqrt(w.vx * w.vx + w.vy * w.vy + w.vz * w.vz);
    int c = static_cast<int>(z / nr), k = static_cast<int>(z % nr);
    double s1 = T.qpow[k];
    double dz = 6.0 * T.V0[c] * s1 / T.S0[c];
    double dtz = dz / (vm + cf);
    if (!(dtz > 0.0)) dtz = -1.0;  // NaN or non-physical state poisons the minimum
    best = fmin(best, dtz);
  }
  best = warp_min(best);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < RED_TPB / 32 ? sm[threadIdx.x] : DBL_MAX;
    v = warp_min(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

__global__ void __launch_bounds__(RED_TPB) k_divb_partial(const DevTables T, const double* __restrict__ phi,
                                                          double* __restrict__ part) {
  __shared__ double sa[RED_TPB / 32], sr[RED_TPB / 32];
  const long long Z = T.Z;
  const int nr = T.nr;
  double ba = 0.0, br = 0.0;
  for (long long z = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; z < Z;
       z += static_cast<long long>(gridDim.x) * blockDim.x) {
    int c = static_cast<int>(z / nr), k = static_cast<int>(z % nr);
    double dv = 0.0, sc = 0.0;
#pragma unroll
    for (int lf = 0; lf < 6; ++lf) {
      long long f;
      double sg;
      if (lf < 4) {
        int sd = side_of_lf(lf);
        f = T.F_rad + static_cast<long long>(T.col_side_se[4 * c + sd]) * nr + k;
        sg = T.col_side_sgn[4 * c + sd];
      } else {
        f = static_cast<long long>(c) * (nr + 1) + k + (lf == 5 ? 1 : 0);
        sg = lf == 5 ? 1.0 : -1.0;
      }
      double p = phi[f];
      dv += sg * p;
      sc += fabs(p);
    }
    ba = fmax(ba, fabs(dv));
    br = fmax(br, sc > 0.0 ? fabs(dv) / sc : 0.0);
  }
  ba = warp_max(ba);
  br = warp_max(br);
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = ba;
    sr[threadIdx.x >> 5] = br;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double a = threadIdx.x < RED_TPB / 32 ? sa[threadIdx.x] : 0.0;
    double r = threadIdx.x < RED_TPB / 32 ? sr[threadIdx.x] : 0.0;
    a = warp_max(a);
    r = warp_max(r);
    if (threadIdx.x == 0) {
      part[2 * blockIdx.x] = a;
      part[2 * blockIdx.x + 1] = r;
    }
  }
}

// final pass: one block folds the partials (min for stride 1, max for stride 2)
__global__ void __launch_bounds__(RED_TPB) k_fold(const double* __restrict__ part, int n, int stride,
                                                  double* __restrict__ out) {
  __shared__ double s0[RED_TPB / 32], s1[RED_TPB / 32];
  double a = stride == 1 ? DBL_MAX : 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (stride == 1) {
      a = fmin(a, part[i]);
    } else {
      a = fmax(a, part[2 * i]);
      b = fmax(b, part[2 * i + 1]);
    }
  }
  a = stride == 1 ? warp_min(a) : warp_max(a);
  b = warp_max(b);
  if ((threadIdx.x & 31) == 0) {
    s0[threadIdx.x >> 5] = a;
    s1[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < RED_TPB / 32 ? s0[threadIdx.x] : (stride == 1 ? DBL_MAX : 0.0);
    double y = threadIdx.x < RED_TPB / 32 ? s1[threadIdx.x] : 0.0;
    x = stride == 1 ? warp_min(x) : warp_max(x);
    y = warp_max(y);
    if (threadIdx.x == 0) {
      out[0] = x;
      if (stride == 2) out[1] = y;
    }
  }
}

// dependent FMA chains: 8 independent chains per thread
template <typename T_>
__global__ void k_fma_probe(T_* out, int iters, T_ a, T_ b) {
  T_ x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = static_cast<T_>(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = x[i] * a + b;
  }
  T_ s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == static_cast<T_>(-1.2345)) out[0] = s;
}

inline unsigned grid_for(long long n) { return static_cast<unsigned>((n + TPB - 1) / TPB); }

#include "adjoint_kernels.inc"
#include "adjoint_team.inc"

// objective of the differentiation workload: J = sum over the outer radial faces of
// Phi_f^2 / A_f (the integral of <B_r>^2 over r_out); one block, deterministic
__global__ void __launch_bounds__(256) k_outer_br2(const DevTables T, const double* __restrict__ phi,
                                                   double* __restrict__ out, double* __restrict__ gphi) {
  __shared__ double sm[8];
  double acc = 0.0;
  const int nr = T.nr;
  const double s2 = T.qpow[nr] * T.qpow[nr];
  for (int c = threadIdx.x; c < T.ncol; c += blockDim.x) {
    const long long f = static_cast<long long>(c) * (nr + 1) + nr;
    const double A = T.A0[6 * c + 4] * s2;
    acc += phi[f] * phi[f] / A;
    if (gphi) gphi[f] = 2.0 * phi[f] / A;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sm[w];
    out[0] = s;
  }
}

}  // namespace

int reduction_blocks(long long n) {
  long long b = (n + RED_TPB - 1) / RED_TPB;
  if (b > 1024) b = 1024;
  if (b < 1) b = 1;
  return static_cast<int>(b);
}

template <int P, typename R>
cudaError_t upload_reference_constants(const Tables& T) {
  using Dm = Dim<P>;
  RefConst<P, R> h{};
  for (int i = 0; i < 3 * Dm::NNZ; ++i) {
    h.Dval[i] = static_cast<R>(T.Dval[i]);
    h.Drow[i] = static_cast<unsigned char>(T.Drow[i]);
  }
  for (int i = 0; i < 3 * (Dm::N + 1); ++i) h.Dptr[i] = static_cast<unsigned short>(T.Dptr[i]);
  for (int i = 0; i < Dm::NQT * Dm::NFN; ++i) h.psiFc[i] = static_cast<R>(T.psiFc[i]);
  for (int i = 0; i < 6 * Dm::NFN; ++i) h.fnode[i] = static_cast<unsigned char>(T.fnode[i]);
  for (int i = 0; i < 12 * Dm::NS * Dm::NEN; ++i) h.psiEc[i] = static_cast<R>(T.psiEc[i]);
  for (int i = 0; i < 12 * Dm::NEN; ++i) h.enode[i] = static_cast<unsigned char>(T.enode[i]);
  for (int i = 0; i < Dm::M * Dm::M; ++i) h.R_[i] = static_cast<R>(T.R[i]);
  // values at the compiled pattern of D^alpha; every nonzero of the host's D^alpha
  // must lie in it, and the face / edge node lists must be the compiled ones
  {
    using RP = RefPattern<P>;
    static_assert(RP::NNZ == Dm::NNZ && RP::NFN == Dm::NFN && RP::NEN == Dm::NEN, "pattern sizes");
    bool in_pat[3][Dm::N][Dm::N] = {};
    for (int e = 0; e < 3 * RP::NNZ; ++e) {
      const int al = e / RP::NNZ, i = RP::I[e], j = RP::J[e];
      in_pat[al][i][j] = true;
      h.Dpat[e] = static_cast<R>(T.D[(static_cast<size_t>(al) * Dm::N + i) * Dm::N + j]);
    }
    for (int al = 0; al < 3; ++al)
      for (int j = 0; j < Dm::N; ++j)
        for (int t = T.Dptr[al * (Dm::N + 1) + j]; t < T.Dptr[al * (Dm::N + 1) + j + 1]; ++t)
          if (!in_pat[al][T.Drow[al * Dm::NNZ + t]][j]) return cudaErrorInvalidValue;
    for (int t = 0; t < 6 * Dm::NFN; ++t)
      if (T.fnode[t] != RP::FN[t]) return cudaErrorInvalidValue;
    // the node-team reverse predictor holds each column of D^alpha in AdjCols<P>::CL slots
    for (int al = 0; al < 3; ++al)
      for (int j = 0; j < Dm::N; ++j)
        if (T.Dptr[al * (Dm::N + 1) + j + 1] - T.Dptr[al * (Dm::N + 1) + j] > AdjCols<P>::CL)
          return cudaErrorInvalidValue;
    for (int t = 0; t < 12 * Dm::NEN; ++t)
      if (T.enode[t] != RP::EN[t]) return cudaErrorInvalidValue;
  }
  // row form of D^alpha, padded to RL entries per row with zeros (column = the row)
  for (int al = 0; al < 3; ++al) {
    int fill[Dm::N] = {};
    for (int i = 0; i < Dm::N; ++i)
      for (int sl = 0; sl < Dm::RL; ++sl) {
        h.Eval[(al * Dm::RL + sl) * Dm::N + i] = R(0);
        h.Ecol[(al * Dm::RL + sl) * Dm::N + i] = static_cast<unsigned char>(i);
      }
    for (int j = 0; j < Dm::N; ++j)
      for (int t = T.Dptr[al * (Dm::N + 1) + j]; t < T.Dptr[al * (Dm::N + 1) + j + 1]; ++t) {
        const int i = T.Drow[al * Dm::NNZ + t];
        const int sl = fill[i]++;
        if (sl >= Dm::RL) return cudaErrorInvalidValue;
        h.Eval[(al * Dm::RL + sl) * Dm::N + i] = static_cast<R>(T.Dval[al * Dm::NNZ + t]);
        h.Ecol[(al * Dm::RL + sl) * Dm::N + i] = static_cast<unsigned char>(j);
      }
  }
  return cudaMemcpyToSymbol(RC<P, R>::sym(), &h, sizeof(h));
}

template <int P, typename R>
cudaError_t launch_stage(int stage, const DevTables& T, const DevState& S, double dt, cudaStream_t st) {
  R* Wc = static_cast<R*>(S.Wc);
  R* Bp = static_cast<R*>(S.Bp);
  R* trF = static_cast<R*>(S.trF);
  R* trE = static_cast<R*>(S.trE);
  switch (stage) {
    case ST_WENO:
      k_weno<P, R><<<dim3(grid_for(T.Z), 8), TPB, 0, st>>>(T, S.U, sizeof(R) == 4 ? S.Uhl : nullptr, Wc);
      break;
    case ST_BPERP:
      k_bperp<P, R><<<grid_for(T.F), TPB, 0, st>>>(T, S.U, S.phi, Wc, Bp);
      break;
    case ST_ADER:
      if (T.predictor == GEO_PRED_VAR_TEAM && !T.positivity) {
        constexpr int ZB = Team<P>::ZB;
        const unsigned grid = static_cast<unsigned>((T.Z + ZB - 1) / ZB);
        k_ader_vt<P, R><<<grid, ZB * Dim<P>::N, 0, st>>>(T, S.U, S.phi, Wc, Bp, trF, trE, dt);
      } else if (T.predictor != GEO_PRED_ZONE_THREAD) {
        constexpr int ZB = Team<P>::ZB;
        const unsigned grid = static_cast<unsigned>((T.Z + ZB - 1) / ZB);
        if (T.positivity)
          k_ader_team<P, R, true><<<grid, ZB * Dim<P>::N, 0, st>>>(T, S.U, S.phi, Wc, Bp, trF, trE, dt, nullptr);
        else
          k_ader_team<P, R, false><<<grid, ZB * Dim<P>::N, 0, st>>>(T, S.U, S.phi, Wc, Bp, trF, trE, dt, nullptr);
      } else if (T.positivity) {
        k_ader<P, R, true><<<grid_for(T.Z), TPB, 0, st>>>(T, S.U, S.phi, Wc, Bp, trF, trE, dt);
        k_pos_traces<P, R><<<grid_for(T.Z), TPB, 0, st>>>(T, S.U, trF, trE);
      } else {
        k_ader<P, R, false><<<grid_for(T.Z), TPB, 0, st>>>(T, S.U, S.phi, Wc, Bp, trF, trE, dt);
      }
      break;
    case ST_FACE:
      if (T.riemann == GEO_RIEMANN_HLLD)
        k_face_flux<P, R, true><<<grid_for(T.F), TPB, 0, st>>>(T, trF, S.Ff, dt);
      else
        k_face_flux<P, R, false><<<grid_for(T.F), TPB, 0, st>>>(T, trF, S.Ff, dt);
      break;
    case ST_EDGE:
      k_edge_emf<P, R><<<grid_for(T.E), TPB, 0, st>>>(T, trE, S.Ee, dt);
      break;
    case ST_UPD_U:
      k_update_u<<<grid_for(T.Z), TPB, 0, st>>>(T, S.U, S.Ff, S.Uhl);
      break;
    case ST_UPD_PHI:
      k_update_phi<<<grid_for(T.F), TPB, 0, st>>>(T, S.phi, S.Ee);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

#define GEO_INSTANTIATE(P, R)                                                                       \
  template cudaError_t upload_reference_constants<P, R>(const Tables&);                              \
  template cudaError_t launch_stage<P, R>(int, const DevTables&, const DevState&, double, cudaStream_t);
GEO_INSTANTIATE(2, double)
GEO_INSTANTIATE(3, double)
GEO_INSTANTIATE(4, double)
GEO_INSTANTIATE(2, float)
GEO_INSTANTIATE(3, float)
GEO_INSTANTIATE(4, float)
#undef GEO_INSTANTIATE

// the reverse predictor: the node team, or one thread per zone when the forward
// predictor runs one thread per zone
template <int P>
cudaError_t launch_adj_ader(const DevTables& T, const DevState& S, const AdjState& A, double dt, cudaStream_t st) {
  const double* Wc = static_cast<const double*>(S.Wc);
  const double* Bp = static_cast<const double*>(S.Bp);
  if (T.predictor == GEO_PRED_ZONE_THREAD) {
    k_adj_ader<P><<<grid_for(T.Z), TPB, 0, st>>>(T, S.phi, Wc, Bp, A, dt);
    return cudaGetLastError();
  }
  using L = AdjTeamLayout<P>;
  constexpr int ZB = Team<P>::ZB;
  const unsigned grid = static_cast<unsigned>((T.Z + ZB - 1) / ZB);
  // with the iterates stored by the forward recompute, the team skips its own
  // forward Picard sweep
  auto run = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(L::bytes));
    if (e != cudaSuccess) return e;
    kern<<<grid, ZB * Dim<P>::N, L::bytes, st>>>(T, S.phi, Wc, Bp, A, dt);
    return cudaGetLastError();
  };
  return A.It ? run(k_adj_ader_team<P, true>) : run(k_adj_ader_team<P, false>);
}

template <int P>
cudaError_t launch_ader_store_iterates(const DevTables& T, const DevState& S, double* It, double dt, cudaStream_t st) {
  constexpr int ZB = Team<P>::ZB;
  const unsigned grid = static_cast<unsigned>((T.Z + ZB - 1) / ZB);
  k_ader_team<P, double, false, true><<<grid, ZB * Dim<P>::N, 0, st>>>(
      T, S.U, S.phi, static_cast<const double*>(S.Wc), static_cast<const double*>(S.Bp), static_cast<double*>(S.trF),
      static_cast<double*>(S.trE), dt, It);
  return cudaGetLastError();
}
template cudaError_t launch_ader_store_iterates<2>(const DevTables&, const DevState&, double*, double, cudaStream_t);
template cudaError_t launch_ader_store_iterates<3>(const DevTables&, const DevState&, double*, double, cudaStream_t);
template cudaError_t launch_ader_store_iterates<4>(const DevTables&, const DevState&, double*, double, cudaStream_t);

template <int P>
cudaError_t launch_adjoint(const DevTables& T, const DevState& S, const AdjState& A, double dt, cudaStream_t st) {
  const double* Wc = static_cast<const double*>(S.Wc);
  const double* Bp = static_cast<const double*>(S.Bp);
  const double* trF = static_cast<const double*>(S.trF);
  const double* trE = static_cast<const double*>(S.trE);
  k_adj_cot<<<grid_for(T.F + T.E), TPB, 0, st>>>(T, A);
  k_adj_face<P><<<grid_for(T.F), TPB, 0, st>>>(T, trF, A, dt);
  k_adj_edge<P><<<grid_for(T.E), TPB, 0, st>>>(T, trE, A, dt);
  cudaError_t e = launch_adj_ader<P>(T, S, A, dt, st);
  if (e != cudaSuccess) return e;
  k_adj_bperp<P><<<grid_for(T.F), TPB, 0, st>>>(T, S.phi, Wc, A);
  k_adj_weno<P><<<grid_for(T.Z), TPB, 0, st>>>(T, A);
  return cudaGetLastError();
}
template <int P>
cudaError_t launch_adjoint_stage(int stage, const DevTables& T, const DevState& S, const AdjState& A, double dt,
                                 cudaStream_t st) {
  const double* Wc = static_cast<const double*>(S.Wc);
  const double* Bp = static_cast<const double*>(S.Bp);
  switch (stage) {
    case ST_WENO: k_adj_weno<P><<<grid_for(T.Z), TPB, 0, st>>>(T, A); break;
    case ST_ADER: return launch_adj_ader<P>(T, S, A, dt, st);
    case ST_FACE: k_adj_face<P><<<grid_for(T.F), TPB, 0, st>>>(T, static_cast<const double*>(S.trF), A, dt); break;
    case ST_EDGE: k_adj_edge<P><<<grid_for(T.E), TPB, 0, st>>>(T, static_cast<const double*>(S.trE), A, dt); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template cudaError_t launch_adjoint_stage<2>(int, const DevTables&, const DevState&, const AdjState&, double,
                                             cudaStream_t);
template cudaError_t launch_adjoint_stage<3>(int, const DevTables&, const DevState&, const AdjState&, double,
                                             cudaStream_t);
template cudaError_t launch_adjoint_stage<4>(int, const DevTables&, const DevState&, const AdjState&, double,
                                             cudaStream_t);
template cudaError_t launch_adjoint<2>(const DevTables&, const DevState&, const AdjState&, double, cudaStream_t);
template cudaError_t launch_adjoint<3>(const DevTables&, const DevState&, const AdjState&, double, cudaStream_t);
template cudaError_t launch_adjoint<4>(const DevTables&, const DevState&, const AdjState&, double, cudaStream_t);

cudaError_t launch_split_u(const DevTables& T, const DevState& S, cudaStream_t st) {
  if (!S.Uhl) return cudaSuccess;
  k_split_u<<<grid_for(T.Z), TPB, 0, st>>>(T, S.U, S.Uhl);
  return cudaGetLastError();
}

cudaError_t launch_outer_br2(const DevTables& T, const double* phi, double* out_dev, double* gphi, cudaStream_t st) {
  k_outer_br2<<<1, 256, 0, st>>>(T, phi, out_dev, gphi);
  return cudaGetLastError();
}

cudaError_t launch_cfl(const DevTables& T, const DevState& S, double cfl, double* out_host, cudaStream_t st) {
  int nb = reduction_blocks(T.Z);
  k_cfl_partial<<<nb, RED_TPB, 0, st>>>(T, S.U, S.red);
  k_fold<<<1, RED_TPB, 0, st>>>(S.red, nb, 1, S.red + 2048);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double v = 0.0;
  e = cudaMemcpyAsync(&v, S.red + 2048, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  *out_host = (v > 0.0) ? cfl * v : v;
  return cudaSuccess;
}

cudaError_t launch_divb(const DevTables& T, const DevState& S, double* out2_host, cudaStream_t st) {
  int nb = reduction_blocks(T.Z);
  k_divb_partial<<<nb, RED_TPB, 0, st>>>(T, S.phi, S.red);
  k_fold<<<1, RED_TPB, 0, st>>>(S.red, nb, 2, S.red + 2048);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(out2_host, S.red + 2048, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

cudaError_t probe_fma(int prec, cudaStream_t st, double* flops_per_s) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 512, blocks = nsm * 4, iters = (prec == 0) ? 4096 : 65536;
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 16);
  if (e != cudaSuccess) return e;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(a, st);
    if (prec == 0)
      k_fma_probe<double><<<blocks, threads, 0, st>>>(static_cast<double*>(buf), iters, 0.999999, 1e-7);
    else
      k_fma_probe<float><<<blocks, threads, 0, st>>>(static_cast<float*>(buf), iters, 0.999999f, 1e-7f);
    cudaEventRecord(b, st);
  }
  e = cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(buf);
  if (e != cudaSuccess) return e;
  double flops = 2.0 * 8.0 * iters * static_cast<double>(threads) * blocks;
  *flops_per_s = flops / (ms * 1e-3);
  return cudaGetLastError();
}

#include "probe_contract.inc"
#include "prism.inc"

}  // namespace geo
