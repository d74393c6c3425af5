// Device helpers shared by the forward kernels (kernels.cu) and the adjoint
// kernels (adjoint_kernels.inc): ideal MHD fluxes in rationalised units (Eq. 2.2),
// the HLL solver, the Rusanov speed, MinMod, the positivity factors, and the
// face/zone index maps.
#pragma once
#include "device.cuh"

namespace geo {
namespace dev {

constexpr int TPB = 128;

template <typename R> __device__ __forceinline__ const BulkTables<R>& bulk(const DevTables& T);
template <> __device__ __forceinline__ const BulkTables<double>& bulk<double>(const DevTables& T) { return T.b64; }
template <> __device__ __forceinline__ const BulkTables<float>& bulk<float>(const DevTables& T) { return T.b32; }

// ----------------------------------------------------------------------------
// ideal MHD (Eq. 2.2 in rationalised units), in the bulk type R
// ----------------------------------------------------------------------------
template <typename R>
struct Prim {
  R rho, vx, vy, vz, p, bx, by, bz;
};

template <typename R>
__device__ __forceinline__ Prim<R> to_prim(const R* u, R g) {
  Prim<R> w;
  w.rho = u[0];
  R ir = R(1) / u[0];
  w.vx = u[1] * ir;
  w.vy = u[2] * ir;
  w.vz = u[3] * ir;
  w.bx = u[5];
  w.by = u[6];
  w.bz = u[7];
  w.p = (g - R(1)) * (u[4] - R(0.5) * w.rho * (w.vx * w.vx + w.vy * w.vy + w.vz * w.vz) -
                      R(0.5) * (w.bx * w.bx + w.by * w.by + w.bz * w.bz));
  return w;
}

// F(U).n for any vector n
template <typename R>
__device__ __forceinline__ void flux_n(const R* u, const Prim<R>& w, R nx, R ny, R nz, R* F) {
  R vn = w.vx * nx + w.vy * ny + w.vz * nz;
  R bn = w.bx * nx + w.by * ny + w.bz * nz;
  R pt = w.p + R(0.5) * (w.bx * w.bx + w.by * w.by + w.bz * w.bz);
  R vb = w.vx * w.bx + w.vy * w.by + w.vz * w.bz;
  F[0] = w.rho * vn;
  F[1] = u[1] * vn + pt * nx - w.bx * bn;
  F[2] = u[2] * vn + pt * ny - w.by * bn;
  F[3] = u[3] * vn + pt * nz - w.bz * bn;
  F[4] = (u[4] + pt) * vn - bn * vb;
  F[5] = w.bx * vn - w.vx * bn;
  F[6] = w.by * vn - w.vy * bn;
  F[7] = w.bz * vn - w.vz * bn;
}

template <typename R>
__device__ __forceinline__ R fast_speed(const Prim<R>& w, R nx, R ny, R nz, R g) {
  R ir = R(1) / w.rho;
  R a2 = g * w.p * ir;
  R b2 = (w.bx * w.bx + w.by * w.by + w.bz * w.bz) * ir;
  R bn = w.bx * nx + w.by * ny + w.bz * nz;
  R bn2 = bn * bn * ir;
  R s = a2 + b2;
  return sqrt(R(0.5) * (s + sqrt(fmax(s * s - R(4) * a2 * bn2, R(0)))));
}

// HLL flux along the unit normal (Davis wave speeds); the weighted flux is
// accumulated in the type A
template <typename R, typename A>
__device__ __forceinline__ void hll_acc(const R* uL, const R* uR, R nx, R ny, R nz, R g, A w, A* acc) {
  Prim<R> a = to_prim(uL, g), b = to_prim(uR, g);
  R vnL = a.vx * nx + a.vy * ny + a.vz * nz;
  R vnR = b.vx * nx + b.vy * ny + b.vz * nz;
  R cL = fast_speed(a, nx, ny, nz, g), cR = fast_speed(b, nx, ny, nz, g);
  R SL = fmin(vnL - cL, vnR - cR);
  R SR = fmax(vnL + cL, vnR + cR);
  R FL[8], FR[8];
  flux_n(uL, a, nx, ny, nz, FL);
  flux_n(uR, b, nx, ny, nz, FR);
  if (SL >= R(0)) {
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[v] += w * static_cast<A>(FL[v]);
  } else if (SR <= R(0)) {
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[v] += w * static_cast<A>(FR[v]);
  } else {
    R id = R(1) / (SR - SL);
#pragma unroll
    for (int v = 0; v < 8; ++v)
      acc[v] += w * static_cast<A>((SR * FL[v] - SL * FR[v] + SL * SR * (uR[v] - uL[v])) * id);
  }
}

// conserved state of a primitive one
template <typename R>
__device__ __forceinline__ void to_cons(const Prim<R>& w, R g, R* u) {
  u[0] = w.rho;
  u[1] = w.rho * w.vx;
  u[2] = w.rho * w.vy;
  u[3] = w.rho * w.vz;
  u[4] = w.p / (g - R(1)) + R(0.5) * w.rho * (w.vx * w.vx + w.vy * w.vy + w.vz * w.vz) +
         R(0.5) * (w.bx * w.bx + w.by * w.by + w.bz * w.bz);
  u[5] = w.bx;
  u[6] = w.by;
  u[7] = w.bz;
}

// HLLD star state (Miyoshi & Kusano 2005) on one side: tangential vectors as
// 3-vectors orthogonal to n; where rho (S - u)(S - S_M) = B_n^2 the tangential
// fields stay unchanged.  Writes U*, its tangential v and B.
template <typename R>
__device__ __forceinline__ void hlld_star(const Prim<R>& w, const R* u, const R* n, R un, R pt, R S, R d, R SM,
                                          R pts, R Bn, R tol, R* Us, R* vts, R* Bts) {
  const R Bn2 = Bn * Bn;
  const R v[3] = {w.vx, w.vy, w.vz}, B[3] = {w.bx, w.by, w.bz};
  const R den = d * (S - SM) - Bn2;
  const bool ok = fabs(den) > tol * (fabs(d * (S - SM)) + Bn2);
  const R fv = ok ? Bn * (SM - un) / den : R(0);
  const R fb = ok ? (d * (S - un) - Bn2) / den : R(1);
  R vs[3], Bs[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R vt = v[a] - un * n[a], Bt = B[a] - Bn * n[a];
    vts[a] = vt - fv * Bt;
    Bts[a] = Bt * fb;
    vs[a] = SM * n[a] + vts[a];
    Bs[a] = Bn * n[a] + Bts[a];
  }
  const R rs = d / (S - SM);
  const R vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
  const R vBs = vs[0] * Bs[0] + vs[1] * Bs[1] + vs[2] * Bs[2];
  Us[0] = rs;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Us[1 + a] = rs * vs[a];
    Us[5 + a] = Bs[a];
  }
  Us[4] = ((S - un) * u[4] - pt * un + pts * SM + Bn * (vB - vBs)) / (S - SM);
}

// HLLD flux along the unit normal (Miyoshi & Kusano 2005): fast waves S_L, S_R
// (Davis speeds as in hll_acc), Alfven waves S*_L, S*_R and the entropy wave S_M,
// total pressure constant in the fan; the normal field is the mean of the two
// sides' (each state keeps its pressure).  Where B_n^2 vanishes the ** states
// equal the * states.  The weighted flux is accumulated in the type A.
template <typename R, typename A>
__device__ __forceinline__ void hlld_acc(const R* uL0, const R* uR0, R nx, R ny, R nz, R g, A w, A* acc) {
  const R tol = sizeof(R) == 4 ? R(1e-6) : R(1e-12);
  const R n[3] = {nx, ny, nz};
  Prim<R> a = to_prim(uL0, g), b = to_prim(uR0, g);
  const R bnL = a.bx * nx + a.by * ny + a.bz * nz, bnR = b.bx * nx + b.by * ny + b.bz * nz;
  const R Bn = R(0.5) * (bnL + bnR);
  a.bx += (Bn - bnL) * nx; a.by += (Bn - bnL) * ny; a.bz += (Bn - bnL) * nz;
  b.bx += (Bn - bnR) * nx; b.by += (Bn - bnR) * ny; b.bz += (Bn - bnR) * nz;
  R uL[8], uR[8];
  to_cons(a, g, uL);
  to_cons(b, g, uR);
  const R unL = a.vx * nx + a.vy * ny + a.vz * nz, unR = b.vx * nx + b.vy * ny + b.vz * nz;
  const R ptL = a.p + R(0.5) * (a.bx * a.bx + a.by * a.by + a.bz * a.bz);
  const R ptR = b.p + R(0.5) * (b.bx * b.bx + b.by * b.by + b.bz * b.bz);
  const R cL = fast_speed(a, nx, ny, nz, g), cR = fast_speed(b, nx, ny, nz, g);
  const R SL = fmin(unL - cL, unR - cR), SR = fmax(unL + cL, unR + cR);
  R F[8];
  if (SL > R(0) || SR <= R(0)) {
    flux_n(uL, a, nx, ny, nz, F);
    if (SR <= R(0)) flux_n(uR, b, nx, ny, nz, F);
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[v] += w * static_cast<A>(F[v]);
    return;
  }
  const R dL = (SL - unL) * a.rho, dR = (SR - unR) * b.rho;
  const R idd = R(1) / (dR - dL);
  const R SM = (dR * unR - dL * unL - ptR + ptL) * idd;
  const R pts = (dR * ptL - dL * ptR + dL * dR * (unR - unL)) * idd;
  R UsL[8], UsR[8], vtL[3], vtR[3], BtL[3], BtR[3];
  hlld_star(a, uL, n, unL, ptL, SL, dL, SM, pts, Bn, tol, UsL, vtL, BtL);
  hlld_star(b, uR, n, unR, ptR, SR, dR, SM, pts, Bn, tol, UsR, vtR, BtR);
  const R sL = sqrt(UsL[0]), sR = sqrt(UsR[0]);
  const R SsL = SM - fabs(Bn) / sL, SsR = SM + fabs(Bn) / sR;
  const bool left = SM > R(0);
  // the side of the fan that holds x/t = 0
  const R* u0 = left ? uL : uR;
  const R* Us = left ? UsL : UsR;
  const R S = left ? SL : SR, Ss = left ? SsL : SsR;
  const bool outer = left ? (SsL > R(0)) : (SsR <= R(0));  // between the fast and the Alfven wave
  if (left) flux_n(uL, a, nx, ny, nz, F);
  else flux_n(uR, b, nx, ny, nz, F);
#pragma unroll
  for (int v = 0; v < 8; ++v) F[v] += S * (Us[v] - u0[v]);
  const bool mag = Bn * Bn > tol * (pts + R(1e-300));
  if (!outer && mag) {
    const R sg = Bn > R(0) ? R(1) : R(-1), iw = R(1) / (sL + sR);
    R vss[3], Bss[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      vss[c] = SM * n[c] + (sL * vtL[c] + sR * vtR[c] + (BtR[c] - BtL[c]) * sg) * iw;
      Bss[c] = Bn * n[c] + (sL * BtR[c] + sR * BtL[c] + sL * sR * (vtR[c] - vtL[c]) * sg) * iw;
    }
    const R rs = Us[0];
    const R vs0 = Us[1] / rs, vs1 = Us[2] / rs, vs2 = Us[3] / rs;
    const R vBs = vs0 * Us[5] + vs1 * Us[6] + vs2 * Us[7];
    const R vBss = vss[0] * Bss[0] + vss[1] * Bss[1] + vss[2] * Bss[2];
    const R side = left ? -(sL) : sR;
    R Uss[8];
    Uss[0] = rs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Uss[1 + c] = rs * vss[c];
      Uss[5 + c] = Bss[c];
    }
    Uss[4] = Us[4] + side * (vBs - vBss) * sg;
#pragma unroll
    for (int v = 0; v < 8; ++v) F[v] += Ss * (Uss[v] - Us[v]);
  }
#pragma unroll
  for (int v = 0; v < 8; ++v) acc[v] += w * static_cast<A>(F[v]);
}

template <typename R>
__device__ __forceinline__ R rusanov_speed(const R* u, R nx, R ny, R nz, R g) {
  Prim<R> w = to_prim(u, g);
  return fabs(w.vx * nx + w.vy * ny + w.vz * nz) + fast_speed(w, nx, ny, nz, g);
}

// the same Rusanov speed from a primitive state whose 1/rho is already formed
template <typename R>
__device__ __forceinline__ R rusanov_speed_ir(R ir, R vx, R vy, R vz, R p, R bx, R by, R bz, R nx, R ny, R nz,
                                              R g) {
  R a2 = g * p * ir;
  R b2 = (bx * bx + by * by + bz * bz) * ir;
  R bn = bx * nx + by * ny + bz * nz;
  R bn2 = bn * bn * ir;
  R s = a2 + b2;
  return fabs(vx * nx + vy * ny + vz * nz) + sqrt(R(0.5) * (s + sqrt(fmax(s * s - R(4) * a2 * bn2, R(0)))));
}

// a[q] for a runtime q in 0..3 of a register array (selects, no local memory)
template <typename T>
__device__ __forceinline__ T sel4(const T (&a)[4], int q) {
  return q == 0 ? a[0] : (q == 1 ? a[1] : (q == 2 ? a[2] : a[3]));
}

template <typename R>
__device__ __forceinline__ R minmod(R a, R b) {
  if (a * b > R(0)) return (a > R(0) ? R(1) : R(-1)) * fmin(fabs(a), fabs(b));
  return R(0);
}

// Positivity scaling (Zhang-Shu type) of point states toward the zone mean: the
// factor theta <= 1 keeps rho >= eps_rho and p >= eps_p at every point, using the
// concavity of p in the conserved variables for the pressure bound.
template <typename R>
__device__ __forceinline__ R pressure_of(const R* u, R g) {
  const R ir = R(1) / u[0];
  return (g - R(1)) * (u[4] - R(0.5) * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * ir -
                       R(0.5) * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]));
}

template <typename R>
__device__ __forceinline__ void pos_rho(const R* s, const R* mean, R eps_r, R& th_r) {
  if (s[0] < eps_r) th_r = fmin(th_r, (mean[0] - eps_r) / (mean[0] - s[0]));
}

template <typename R>
__device__ __forceinline__ void pos_p(const R* s, const R* mean, R th_r, R g, R pb, R eps_p, R& th_p) {
  R s1[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) s1[v] = mean[v] + th_r * (s[v] - mean[v]);
  const R p1 = pressure_of(s1, g);
  if (p1 < eps_p) th_p = fmin(th_p, (pb - eps_p) / (pb - p1));
}

// predictor traces, structure of arrays: value v of point idx at Gauss time m of
// zone z sits at trF_at(z, m, idx, Z) + v * Z (consecutive zones are adjacent)
template <int P>
__device__ __forceinline__ size_t trF_at(long long z, int m, int idx, long long Z) {
  return (static_cast<size_t>((m - 1) * Dim<P>::NQT + idx) * 8) * Z + z;
}
template <int P>
__device__ __forceinline__ size_t trE_at(long long z, int m, int idx, long long Z) {
  return (static_cast<size_t>((m - 1) * 12 * Dim<P>::NS + idx) * 8) * Z + z;
}

__device__ __forceinline__ int side_of_lf(int lf) { return lf == 0 ? 3 : (lf == 1 ? 1 : (lf == 2 ? 0 : 2)); }

template <int P>
__device__ __forceinline__ int foff(int lf) {
  using Dm = Dim<P>;
  return lf < 4 ? lf * Dm::NQS : 4 * Dm::NQS + (lf - 4) * Dm::NQR;
}
template <int P>
__device__ __forceinline__ int nq_of(int lf) {
  return lf < 4 ? Dim<P>::NQS : Dim<P>::NQR;
}

// face f -> L zone / local face, R zone / local face (-1 when on the boundary),
// the column and local face whose tables hold the face geometry, shell index k
struct FaceInfo {
  long long zL, zR;
  int lfL, lfR, cg, lfg, k, se;
  double gsign;  // canonical normal = gsign * outward normal of (cg, lfg)
};

__device__ __forceinline__ FaceInfo face_info(const DevTables& T, long long f) {
  FaceInfo fi;
  int nr = T.nr;
  if (f < T.F_rad) {
    int c = static_cast<int>(f / (nr + 1));
    int k = static_cast<int>(f % (nr + 1));
    fi.zL = (k >= 1) ? static_cast<long long>(c) * nr + k - 1 : -1;
    fi.zR = (k < nr) ? static_cast<long long>(c) * nr + k : -1;
    fi.lfL = 5;
    fi.lfR = 4;
    fi.cg = c;
    fi.lfg = 4;
    fi.gsign = -1.0;
    fi.k = k;
    fi.se = -1;
  } else {
    long long r = f - T.F_rad;
    int se = static_cast<int>(r / nr);
    int k = static_cast<int>(r % nr);
    int cL = T.se_col[2 * se], cR = T.se_col[2 * se + 1];
    fi.zL = static_cast<long long>(cL) * nr + k;
    fi.zR = static_cast<long long>(cR) * nr + k;
    fi.lfL = T.se_lf[2 * se];
    fi.lfR = T.se_lf[2 * se + 1];
    fi.cg = cL;
    fi.lfg = fi.lfL;
    fi.gsign = 1.0;
    fi.k = k;
    fi.se = se;
  }
  return fi;
}


}  // namespace dev
}  // namespace geo
