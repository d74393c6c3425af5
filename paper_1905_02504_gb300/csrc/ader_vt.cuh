// Predictor schedule GEO_PRED_VAR_TEAM: the node team of k_ader_team with the
// derivative contraction and the point evaluations moved to the variable layout.
// Included by kernels.cu inside its anonymous namespace.
//
// Per flux evaluation of a level (Eqs. C.34-C.36, D.29-D.32) the work splits in
// two layouts that meet in shared memory:
//   node phase      thread (zone, node i) evaluates the metric fluxes
//                   F^alpha_v(U_i) of its node (nonlinear in all 8 variables),
//                   stores them as rows [zone][alpha][v][node];
//   variable phase  thread (zone, v, row group g) forms
//                   dF_{v,i} = sum_alpha sum_j D^alpha_ij F^alpha_{v,j}
//                   for the rows i of group g.  The nonzero pattern of D^alpha is
//                   compiled in (refpattern.h), so the F values sit in registers,
//                   the D values are constant-bank operands, and the only shared
//                   traffic is one 16-byte load per needed 4-node chunk of F.
// The final levels are exchanged once more the same way, and each (zone, v,
// group) thread evaluates its share of the face and edge points (face by face,
// edge by edge: the support node lists are compiled in) and writes the traces.
// Groups are balanced by entry (point) count; the group index is the slowest
// part of the thread index, so every warp runs the code of one group.
// Only the unlimited predictor has this schedule: with positivity on, the
// node-team kernel runs.
// (kernels.cu includes <utility> and the generated refpattern.h at file scope)

template <int V> using IC = std::integral_constant<int, V>;

template <int P, typename R>
struct VtLayout {
  using Dm = Dim<P>;
  static constexpr int ZB = Team<P>::ZB, N = Dm::N, CH = Chunk<R>::CH;
  // node stride of one [alpha][v] row (a multiple of the 16-byte chunk), with
  // P = 4 padded so the two variables of an 8-lane FP32 access phase sit in
  // different bank groups
  static constexpr int NP = (P == 4) ? 36 : ((N + 3) / 4) * 4;
  // zone strides padded so that the zones of one warp-wide scalar access fall
  // into distinct banks: (words per zone) = 32 / ZB modulo 32, at least 4
  static constexpr int WPE = sizeof(R) / 4;
  static constexpr int TGT = ((32 / ZB) > 4 ? (32 / ZB) : 4) / WPE;
  static constexpr int MODE = 32 / WPE;
  __host__ __device__ static constexpr int pad(int x) { return x + ((TGT - x % MODE) % MODE + MODE) % MODE; }
  static constexpr int XZ = pad(24 * NP);  // F rows / final levels per zone
  static constexpr int OZ = pad(8 * N);    // flux differences per zone
  static constexpr int G = RefPattern<P>::G;
  static constexpr int NVT = 8 * ZB * G;   // threads of the variable phase
};

template <int P, typename R>
struct VtSmem {
  using L = VtLayout<P, R>;
  using Dm = Dim<P>;
  alignas(16) R XF[L::ZB * L::XZ];
  R XO[L::ZB * L::OZ];
  R in[L::ZB][Dm::NBIN];
  R W[L::ZB][5 * Dm::NC1];
  R Uz[L::ZB][8];
  R fs[L::ZB];
};

// the 16-byte chunk C of F^alpha's row is used by some entry of row group G
template <int P, int A, int G, int C, int CH>
__host__ __device__ constexpr bool vt_needs_chunk() {
  using RP = RefPattern<P>;
  for (int e = RP::EG[A][G]; e < RP::EG[A][G + 1]; ++e)
    if (RP::J[A * RP::NNZ + e] / CH == C) return true;
  return false;
}

template <int P, typename R, int A, int G, int... Cs>
__device__ __forceinline__ void vt_load_row(const R* row, R* Fr, std::integer_sequence<int, Cs...>) {
  constexpr int CH = Chunk<R>::CH;
  auto one = [&](auto c) {
    if constexpr (vt_needs_chunk<P, A, G, decltype(c)::value, CH>()) ld16(row + decltype(c)::value * CH,
                                                                          Fr + decltype(c)::value * CH);
  };
  (one(IC<Cs>{}), ...);
}

// acc[i - RG[G]] += D^A_ij F_j over the entries of row group G
template <int P, typename R, int A, int G, int... Es>
__device__ __forceinline__ void vt_rows(R* acc, const R* Fr, const RefConst<P, R>& K,
                                        std::integer_sequence<int, Es...>) {
  using RP = RefPattern<P>;
  constexpr int E0 = A * RP::NNZ + RP::EG[A][G], R0 = RP::RG[G];
  ((acc[IC<RP::I[E0 + Es] - R0>::value] += K.Dpat[E0 + Es] * Fr[IC<RP::J[E0 + Es]>::value]), ...);
}

template <int P, typename R, int G, int A>
__device__ __forceinline__ void vt_direction(R* acc, const R* rowA, const RefConst<P, R>& K) {
  using RP = RefPattern<P>;
  constexpr int N = Dim<P>::N, CH = Chunk<R>::CH;
  R Fr[((N + CH - 1) / CH) * CH];
  vt_load_row<P, R, A, G>(rowA, Fr, std::make_integer_sequence<int, (N + CH - 1) / CH>{});
  vt_rows<P, R, A, G>(acc, Fr, K, std::make_integer_sequence<int, RP::EG[A][G + 1] - RP::EG[A][G]>{});
}

// variable phase of one flux evaluation for row group G: reads the F rows of
// variable v of zone zl, writes dF_{v,i} for the group's rows
template <int P, typename R, int G>
__device__ __forceinline__ void vt_contract(const R* XFz, R* XOz, int v, const RefConst<P, R>& K) {
  using RP = RefPattern<P>;
  using L = VtLayout<P, R>;
  constexpr int NRG = RP::RG[G + 1] - RP::RG[G];
  R acc[NRG];
#pragma unroll
  for (int r = 0; r < NRG; ++r) acc[r] = R(0);
  vt_direction<P, R, G, 0>(acc, XFz + (0 * 8 + v) * L::NP, K);
  vt_direction<P, R, G, 1>(acc, XFz + (1 * 8 + v) * L::NP, K);
  vt_direction<P, R, G, 2>(acc, XFz + (2 * 8 + v) * L::NP, K);
#pragma unroll
  for (int r = 0; r < NRG; ++r) XOz[v * Dim<P>::N + RP::RG[G] + r] = acc[r];
}

template <int P, typename R, int G = 0>
__device__ __forceinline__ void vt_contract_dispatch(int g, const R* XFz, R* XOz, int v, const RefConst<P, R>& K) {
  if constexpr (G < RefPattern<P>::G) {
    if (g == G) vt_contract<P, R, G>(XFz, XOz, v, K);
    else vt_contract_dispatch<P, R, G + 1>(g, XFz, XOz, v, K);
  }
}

// One out-of-line copy of the variable phase for all groups: the predictor calls
// it from 1 + (M-1) places (level 1, then each level inside the Picard loop), and
// inlining it there multiplied the fully unrolled group code M-fold, beyond what
// the instruction cache holds.
template <int P, typename R>
__device__ __noinline__ void vt_contract_group(int g, const R* XFz, R* XOz, int v) {
  vt_contract_dispatch<P, R>(g, XFz, XOz, v, RC<P, R>::get());
}

// ---- point evaluations.  Work items are (level m, face or edge e), level-major,
// the 6 faces before the 12 edges; an item's points share its support nodes
// (the face's / edge's nodes), so a thread loads those values once (compile-time
// node indices) and loops over the item's points at run time, the basis weights
// coming from constant memory (the same address for the whole warp).  Items go to
// the row groups in contiguous ranges balanced by cost (points x support).
template <int P>
struct VtItems {
  using Dm = Dim<P>;
  using RP = RefPattern<P>;
  static constexpr int NE = 18, NIT = (Dm::M - 1) * NE, G = RP::G;
  __host__ __device__ static constexpr int np(int e) { return e < 4 ? Dm::NQS : (e < 6 ? Dm::NQR : Dm::NS); }
  __host__ __device__ static constexpr int cost(int t) {
    return np(t % NE) * ((t % NE) < 6 ? RP::NFN : RP::NEN);
  }
  __host__ __device__ static constexpr int total() {
    int s = 0;
    for (int t = 0; t < NIT; ++t) s += cost(t);
    return s;
  }
  // first item of group g
  __host__ __device__ static constexpr int start(int g) {
    if (g <= 0) return 0;
    if (g >= G) return NIT;
    int s = 0;
    for (int t = 0; t < NIT; ++t) {
      if (s * G >= total() * g) return t;
      s += cost(t);
    }
    return NIT;
  }
  // first face point of local face lf (faces 0-3: NQS points, 4-5: NQR)
  __host__ __device__ static constexpr int foff(int lf) {
    return lf < 4 ? lf * Dm::NQS : 4 * Dm::NQS + (lf - 4) * Dm::NQR;
  }
};

template <int P, typename R, int S0, int... As>
__device__ __forceinline__ void vt_gather(const R* row, R* Xs, std::integer_sequence<int, As...>) {
  using RP = RefPattern<P>;
  ((Xs[As] = row[IC<S0 < 6 * RP::NFN ? RP::FN[S0 + As] : RP::EN[S0 - 6 * RP::NFN + As]>::value]), ...);
}

// one item T = m * 18 + e of variable v
template <int P, typename R, int T>
__device__ __forceinline__ void vt_item(const R* XFz, int v, const RefConst<P, R>& K, const R* iJF, const R* iJE,
                                        R* trF, R* trE, long long Z, long long z, bool valid) {
  using IT = VtItems<P>;
  using RP = RefPattern<P>;
  using L = VtLayout<P, R>;
  using Dm = Dim<P>;
  constexpr int m = T / IT::NE, e = T % IT::NE;
  const R* row = XFz + (m * 8 + v) * L::NP;
  if constexpr (e < 6) {
    R Xs[RP::NFN];
    vt_gather<P, R, e * RP::NFN>(row, Xs, std::make_integer_sequence<int, RP::NFN>{});
    constexpr int f0 = IT::foff(e);
#pragma unroll 1
    for (int q = 0; q < IT::np(e); ++q) {
      const R* ps = K.psiFc + (f0 + q) * RP::NFN;
      R s = R(0);
#pragma unroll
      for (int a = 0; a < RP::NFN; ++a) s += ps[a] * Xs[a];
      if (valid) trF[(static_cast<size_t>(m * Dm::NQT + f0 + q) * 8 + v) * Z + z] = s * iJF[f0 + q];
    }
  } else {
    constexpr int le = e - 6;
    R Xs[RP::NEN];
    vt_gather<P, R, 6 * RP::NFN + le * RP::NEN>(row, Xs, std::make_integer_sequence<int, RP::NEN>{});
#pragma unroll 1
    for (int q = 0; q < Dm::NS; ++q) {
      const int idx = le * Dm::NS + q;
      const R* ps = K.psiEc + idx * RP::NEN;
      R s = R(0);
#pragma unroll
      for (int a = 0; a < RP::NEN; ++a) s += ps[a] * Xs[a];
      if (valid) trE[(static_cast<size_t>(m * 12 * Dm::NS + idx) * 8 + v) * Z + z] = s * iJE[idx];
    }
  }
}

template <int P, typename R, int T0, int T1>
__device__ __forceinline__ void vt_items(const R* XFz, int v, const RefConst<P, R>& K, const R* iJF, const R* iJE,
                                         R* trF, R* trE, long long Z, long long z, bool valid) {
  if constexpr (T0 < T1) {
    vt_item<P, R, T0>(XFz, v, K, iJF, iJE, trF, trE, Z, z, valid);
    vt_items<P, R, T0 + 1, T1>(XFz, v, K, iJF, iJE, trF, trE, Z, z, valid);
  }
}

template <int P, typename R, int G = 0>
__device__ __forceinline__ void vt_traces_group(int g, const R* XFz, int v, const RefConst<P, R>& K, const R* iJF,
                                                const R* iJE, R* trF, R* trE, long long Z, long long z, bool valid) {
  if constexpr (G < RefPattern<P>::G) {
    using IT = VtItems<P>;
    if (g == G)
      vt_items<P, R, IT::start(G), IT::start(G + 1)>(XFz, v, K, iJF, iJE, trF, trE, Z, z, valid);
    else
      vt_traces_group<P, R, G + 1>(g, XFz, v, K, iJF, iJE, trF, trE, Z, z, valid);
  }
}

// resident blocks per SM (the register budget per thread follows); FP32 at p = 3,
// 196,608 zones: 4 / 5 / 6 blocks 0.851 / 0.770 / 0.719 ms; FP32 at p = 4,
// 1,572,864 zones: 4 / 5 blocks 26.1 / 28.3 ms
template <int P, typename R> struct VtOcc;
template <> struct VtOcc<2, float> { static constexpr int MINB = 8; };
template <> struct VtOcc<3, float> { static constexpr int MINB = 6; };
template <> struct VtOcc<4, float> { static constexpr int MINB = 4; };
template <> struct VtOcc<2, double> { static constexpr int MINB = 4; };
template <> struct VtOcc<3, double> { static constexpr int MINB = 2; };
template <> struct VtOcc<4, double> { static constexpr int MINB = 2; };

template <int P, typename R>
__global__ void __launch_bounds__(Team<P>::ZB * Dim<P>::N, VtOcc<P, R>::MINB)
    k_ader_vt(const DevTables T, double* __restrict__ U, const double* __restrict__ phi, const R* __restrict__ Wc,
              const R* __restrict__ Bp, R* __restrict__ trF, R* __restrict__ trE, double dt) {
  using Dm = Dim<P>;
  using L = VtLayout<P, R>;
  constexpr int N = Dm::N, M = Dm::M, ZB = Team<P>::ZB;
  __shared__ VtSmem<P, R> S;
  const RefConst<P, R>& K = RC<P, R>::get();
  const BulkTables<R>& BT = bulk<R>(T);
  const long long Z = T.Z;
  const int nr = T.nr;
  const int tid = threadIdx.x;
  const long long zbase = static_cast<long long>(blockIdx.x) * ZB;
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
    const R j0 = valid ? BT.J0[static_cast<size_t>(c) * N + i] : R(1);
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int v = 0; v < 8; ++v) Uh[m][v] = j0 * u[v];
  }
  R iJ, g[3], Sa[9];
  team_node_metrics<P, R>(BT, c, i, valid, iJ, g, Sa);
  // ---- variable-phase role of this thread: (group, variable, zone), zone fastest
  const bool vrole = tid < L::NVT;
  const int vg = tid / (8 * ZB), vv = (tid / ZB) % 8, vz = tid % ZB;
  R* XFz = S.XF + zl * L::XZ;
  const R* XFv = S.XF + vz * L::XZ;
  R* XOv = S.XO + vz * L::OZ;
  const R* XOz = S.XO + zl * L::OZ;
  // one flux difference of every node of the block: dF_i = sum D F - F(U_i) . g_i
  auto flux_difference = [&](const R* Um, R* dFm) {
    {
      R u[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) u[v] = Um[v] * iJ;
      Prim<R> w = to_prim(u, gam);
      R Gf[8];
      flux_n(u, w, g[0], g[1], g[2], Gf);
#pragma unroll
      for (int v = 0; v < 8; ++v) dFm[v] = -Gf[v];
#pragma unroll
      for (int al = 0; al < 3; ++al) {
        R Fa[8];
        flux_n(u, w, Sa[3 * al], Sa[3 * al + 1], Sa[3 * al + 2], Fa);
#pragma unroll
        for (int v = 0; v < 8; ++v) XFz[(al * 8 + v) * L::NP + i] = Fa[v];
      }
    }
    __syncthreads();
    if (vrole) vt_contract_group<P, R>(vg, XFv, XOv, vv);
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 8; ++v) dFm[v] += XOz[v * N + i];
  };
  // ---- Picard iterations (Eqs. C.34-C.36); the first iteration's flux
  // difference of level 1 serves every level (all levels equal level 1 there)
  const R fs = S.fs[zl];
  R dF[M][8];
  flux_difference(Uh[0], dF[0]);
#pragma unroll
  for (int m = 1; m < M; ++m)
#pragma unroll
    for (int v = 0; v < 8; ++v) dF[m][v] = dF[0][v];
#pragma unroll 1
  for (int it = 0; it < P; ++it) {
    if (it > 0) {
#pragma unroll
      for (int m = 1; m < M; ++m) flux_difference(Uh[m], dF[m]);
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
    }
  }
  // ---- final levels to the variable layout (the F rows are free after the last
  // flux difference's closing barrier), then the traces
#pragma unroll
  for (int m = 1; m < M; ++m)
#pragma unroll
    for (int v = 0; v < 8; ++v) XFz[((m - 1) * 8 + v) * L::NP + i] = Uh[m][v];
  __syncthreads();
  if (vrole) {
    const long long zv = zbase + vz;
    const bool validv = zv < Z;
    const int cv = validv ? static_cast<int>(zv / nr) : 0;
    vt_traces_group<P, R>(vg, XFv, vv, K, BT.iJF + static_cast<size_t>(cv) * Dm::NQT,
                          BT.iJE + static_cast<size_t>(cv) * 12 * Dm::NS, trF, trE, Z, zv, validv);
  }
}
