// Device-side declarations shared by the kernels and the C-ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace geo {

template <int P> struct Dim;
template <> struct Dim<2> {
  static constexpr int N = 8, M = 2, NC1 = 3, NC = 4, NB = 7, NQR = 4, NQS = 4, NQT = 24, NS = 1,
                       SMAX = 6, NBIN = 3 * NC + NQT + 6, NNZ = 16, NFN = 4, NEN = 2, RL = 2;
};
template <> struct Dim<3> {
  static constexpr int N = 20, M = 3, NC1 = 9, NC = 10, NB = 16, NQR = 4, NQS = 4, NQT = 24, NS = 2,
                       SMAX = 26, NBIN = 3 * NC + NQT + 6, NNZ = 96, NFN = 8, NEN = 3, RL = 8;
};
template <> struct Dim<4> {
  static constexpr int N = 32, M = 4, NC1 = 19, NC = 20, NB = 30, NQR = 9, NQS = 6, NQT = 42, NS = 3,
                       SMAX = 32, NBIN = 3 * NC + NQT + 6, NNZ = 192, NFN = 12, NEN = 4, RL = 8;
};

// Reference-element constants of one order in the bulk arithmetic type R, kept
// in constant memory (every thread of a warp reads the same entry, so the
// constant cache broadcasts).
template <int P, typename R> struct RefConst {
  R Dval[3 * Dim<P>::NNZ];                      // CSC values of D^xi, D^eta, D^zeta
  unsigned char Drow[3 * Dim<P>::NNZ];          // row (node i) of each value
  unsigned short Dptr[3 * (Dim<P>::N + 1)];     // column (node j) pointers
  R Eval[3 * Dim<P>::RL * Dim<P>::N];           // the same matrices by rows, padded to RL
  unsigned char Ecol[3 * Dim<P>::RL * Dim<P>::N];  // entries per row: [alpha][slot][row i]
  R psiFc[Dim<P>::NQT * Dim<P>::NFN];           // face-node basis at the face points
  unsigned char fnode[6 * Dim<P>::NFN];
  R psiEc[12 * Dim<P>::NS * Dim<P>::NEN];       // edge-node basis at the edge points
  unsigned char enode[12 * Dim<P>::NEN];
  R R_[Dim<P>::M * Dim<P>::M];
  R Dpat[3 * Dim<P>::NNZ];                      // D^alpha at the compiled pattern (refpattern.h)
};

// Per-column matrices used by the bulk arithmetic, in its type R.  The FP64
// form points at the FP64 tables; the FP32-bulk form at FP32 copies made once
// at mesh creation (the FP64 masters stay on the device).  GB and TN are stored
// transposed on the device, [ncol][NBIN][3+3N] and [ncol][NC1][N], so that the
// threads of a node team read consecutive entries.
template <typename R> struct BulkTables {
  const R *pinvH, *oct_inv, *Q, *TF, *nF, *wF, *GB, *TN, *J0, *iJ0, *Sm, *gcl, *JF, *JE;
  // edge geometry: unit tangents and face normals at the edge points
  const R *se_t, *se_nang, *se_nradL, *se_nradR, *sv_fn, *sv_t;
  // [ncol] (l_0 / |x_0|)^2 of the column's zones (the same along a self-similar
  // column): the mesh scale of the WENO-AO eps, eps = 1e-12 + weta u_0^2
  const R* weta;
  // [ncol][NQT], [ncol][12 NS]: 1 / (interpolated J) at the face and edge points
  const R *iJF, *iJE;
};

// Read-only tables in device memory (see host_tables.h for the layouts).
struct DevTables {
  int n, nr, ncol, nsv, nse;
  long long Z, F, E, F_rad, E_rad;
  double gamma;
  int positivity;      // 1: scale nodal and point states toward the zone mean (rho, p > 0)
  int predictor;       // GEO_PRED_*: the predictor's execution schedule
  int riemann;         // GEO_RIEMANN_*: the face solver
  int* status;         // [1] bit 0 set by the U update when a zone leaves rho > 0, p > 0 (or is not finite)
  const double* qpow;  // [nr + 2]: q^k
  const double* iA0;   // [ncol][6]: 1 / A0 (reciprocal face areas at shell 0)
  const double* iq2;   // [nr + 2]: q^-2k
  const double *D, *R, *wt, *psiF, *psiE, *wE;
  const int* st_n;
  const int* st_nb;
  const double* pinvH;
  const int* oct_nb;
  const double *oct_inv, *Q, *V0, *l0, *S0, *A0, *TF, *nF, *wF, *WF, *GB, *TN, *J0, *iJ0, *Sm, *gcl, *JF, *JE;
  const int *col_side_se, *col_side_sgn;
  const int *se_v, *se_col, *se_lf, *se_perm, *se_le, *se_rev;
  const double *se_t, *se_dlw, *se_nang, *se_nradL, *se_nradR;
  const int *sv_nc, *sv_col, *sv_le, *sv_fL, *sv_fR, *sv_fse;
  const double *sv_fn, *sv_t, *sv_dlw;
  BulkTables<double> b64;
  BulkTables<float> b32;
};

// Mutable device state and work arrays of one mesh.
// Work arrays marked (R) hold the bulk arithmetic type (double or float).
struct DevState {
  double* U;     // [8][Z]
  double* phi;   // [F]
  void* Wc;      // (R) [8*NC1][Z] WENO-AO Taylor coefficients
  void* Bp;      // (R) [NQmax][F]  nodal normal B per face (canonical orientation)
  void* trF;     // (R) [(M-1)*NQT*8][Z] predictor states at the zone's face points
  void* trE;     // (R) [(M-1)*12*NS*8][Z] predictor states at the zone's edge points
  double* Ff;    // [8][F] time-integrated face fluxes (FP64 accumulation)
  double* Ee;    // [E]   time-integrated edge EMFs (FP64 accumulation)
  double* red;   // reduction scratch
  float* Uhl;    // FP32-bulk only: [16][Z] U split as hi = fl(U), lo = fl(U - hi), for the WENO differences
};

// Work arrays of the adjoint step (FP64): cotangents of every forward quantity.
struct AdjState {
  const double* gUp;    // [8][Z] cotangent of U at t+dt (input)
  const double* gphip;  // [F]    cotangent of phi at t+dt (input)
  double* gU;           // [8][Z] cotangent of U at t (output; accumulated)
  double* gphi;         // [F]    cotangent of phi at t (output)
  double* gFf;          // [8][F]
  double* gEe;          // [E]
  double* gtrF;         // like trF
  double* gtrE;         // like trE
  double* gW;           // [8*NC1][Z]
  double* gBpz;         // [NQT][Z] cotangent of the zone's KKT inputs from the face fields
  double* gphiz;        // [6][Z]   cotangent of the zone's face-mean inputs
  const double* U0;     // [8][Z] checkpoint state (read only, pristine)
  // Picard iterates of the checkpoint's predictor stored by its forward recompute
  // ([P-1][M-1][8][N][Z]), or null: the reverse predictor then recomputes them
  const double* It = nullptr;
};

enum Stage { ST_WENO = 0, ST_BPERP, ST_ADER, ST_FACE, ST_EDGE, ST_UPD_U, ST_UPD_PHI, N_STAGES };

struct Tables;
// copy the order-P reference constants into constant memory in type R (kernels.cu)
template <int P, typename R>
cudaError_t upload_reference_constants(const Tables& T);

// launchers (kernels.cu); return cudaGetLastError() of the launch
template <int P, typename R>
cudaError_t launch_stage(int stage, const DevTables& T, const DevState& S, double dt, cudaStream_t st);
// the FP64 node-team predictor (no positivity) that also stores its Picard
// iterates for the reverse sweep (It: [P-1][M-1][8][N][Z] doubles)
template <int P>
cudaError_t launch_ader_store_iterates(const DevTables& T, const DevState& S, double* It, double dt, cudaStream_t st);
cudaError_t launch_cfl(const DevTables& T, const DevState& S, double cfl, double* out_host,
                       cudaStream_t st);
cudaError_t launch_divb(const DevTables& T, const DevState& S, double* out2_host, cudaStream_t st);
// refresh S.Uhl from S.U (FP32-bulk meshes, after an upload)
cudaError_t launch_split_u(const DevTables& T, const DevState& S, cudaStream_t st);
cudaError_t probe_fma(int prec, cudaStream_t st, double* flops_per_s);
// reverse sweep of one step (FP64); the forward intermediates of the checkpoint
// state are in S (Wc, Bp, trF, trE), the pristine checkpoint in A.U0
template <int P>
cudaError_t launch_adjoint(const DevTables& T, const DevState& S, const AdjState& A, double dt, cudaStream_t st);
// the reverse kernel of one forward stage alone (ST_WENO, ST_ADER, ST_FACE, ST_EDGE)
template <int P>
cudaError_t launch_adjoint_stage(int stage, const DevTables& T, const DevState& S, const AdjState& A, double dt,
                                 cudaStream_t st);
int reduction_blocks(long long n);
cudaError_t launch_outer_br2(const DevTables& T, const double* phi, double* out_dev, double* gphi, cudaStream_t st);

}  // namespace geo
