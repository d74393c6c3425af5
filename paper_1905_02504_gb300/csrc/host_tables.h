// Host-side (FP64) construction of the mesh and of every per-column table the
// device kernels read.  Zones of one radial column are self-similar on
// log-ratioed shells (paper Sec. IV.b step 7, Sec. V.b), so each table is built
// once for the column's zone at shell 0 and rescaled on the device by powers of
// q = (r_out/r_in)^(1/nr).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace geo {

struct Dims {
  int P;     // scheme order
  int N;     // serendipity nodes
  int M;     // time levels
  int NC1;   // Taylor coefficients of degree 1..P-1
  int NC;    // NC1 + 1 (with the mean)
  int NB;    // terms of one divergence-free component
  int NQR;   // points of a radial face
  int NQS;   // points of a side face
  int NQT;   // points of the six faces
  int NS;    // edge points
  int SMAX;  // largest central stencil
  int G;     // ghost shells
  int NDIV;  // divergence constraints
  int NBIN;  // inputs of the divergence-free reconstruction
  int NNZ;   // nonzeros of one derivative matrix D^alpha
  int NFN;   // nodes on one face
  int NEN;   // nodes on one edge
};
Dims dims_for_order(int p);

struct Tables {
  Dims d;
  int n = 0, nr = 0, ncol = 0, nsv = 0, nse = 0;
  int64_t Z = 0, F = 0, E = 0, F_rad = 0, E_rad = 0;
  double r_in = 0, r_out = 0, q = 1;

  // reference element, shared by all zones
  std::vector<double> D;     // [3][N][N]  d psi_j / d xi_a at node i
  std::vector<double> R;     // [M][M]
  std::vector<double> wt;    // [M-1]      Gauss weights of tau_2..tau_M
  std::vector<double> psiF;  // [NQT][N]   basis at the face points (local faces 0..5)
  std::vector<double> psiE;  // [12][NS][N]
  std::vector<double> wE;    // [NS]
  std::vector<int> foff;     // [7]        offsets of the local faces in NQT
  // sparse forms (the serendipity derivative matrices are sparse, and a basis
  // function restricted to a face / edge only involves that face's / edge's nodes)
  std::vector<int> Dptr;     // [3][N+1]   column pointers of D^alpha (CSC)
  std::vector<int> Drow;     // [3][NNZ]
  std::vector<double> Dval;  // [3][NNZ]
  std::vector<int> fnode;    // [6][NFN]   nodes of each local face
  std::vector<double> psiFc; // [NQT][NFN] basis of those nodes at the face points
  std::vector<int> enode;    // [12][NEN]  nodes of each local edge
  std::vector<double> psiEc; // [12*NS][NEN]

  // per column (zone at shell 0)
  std::vector<int> st_n;       // [ncol]
  std::vector<int> st_nb;      // [ncol][SMAX] packed (col << 3) | (dk + 3)
  std::vector<double> pinvH;   // [ncol][NC1][SMAX]
  std::vector<int> oct_nb;     // [ncol][8][3] packed
  std::vector<double> oct_inv; // [ncol][8][3][3]
  std::vector<double> Q;       // [ncol][NC1][NC1]
  std::vector<double> V0, l0, S0;  // [ncol]
  std::vector<double> xc0;     // [ncol][3]
  std::vector<double> A0;      // [ncol][6]
  std::vector<double> TF;      // [ncol][NQT][NC1] Taylor basis at face points
  std::vector<double> nF;      // [ncol][NQT][3]   outward unit normals
  std::vector<double> wF;      // [ncol][NQT]      w_ref |dA| / A (sums to 1 per face)
  std::vector<double> WF;      // [ncol][NQT]      w_ref |dA| at shell 0
  std::vector<double> GB;      // [ncol][3+3N][NBIN]
  std::vector<double> TN;      // [ncol][N][NC1]   Taylor basis at the nodes
  std::vector<double> J0;      // [ncol][N]
  std::vector<double> iJ0;     // [ncol][N]        1 / J0
  std::vector<double> Sm;      // [ncol][3][N][3]  h_eta x h_zeta, h_zeta x h_xi, h_xi x h_eta
  std::vector<double> gcl;     // [ncol][N][3]
  std::vector<double> JF;      // [ncol][NQT]      interpolated J at face points
  std::vector<double> JE;      // [ncol][12][NS]
  std::vector<int> col_side_se;   // [ncol][4] sides s,e,n,w
  std::vector<int> col_side_sgn;  // [ncol][4] +1: canonical direction is counter-clockwise
  std::vector<int> col_verts;     // [ncol][4] v00,v10,v01,v11

  // per sphere edge (angular faces and angular edges)
  std::vector<int> se_v;       // [nse][2]
  std::vector<int> se_col;     // [nse][2]   L, R column
  std::vector<int> se_lf;      // [nse][2]   local face in L, R
  std::vector<int> se_perm;    // [nse][NQS] R-local point of L point q
  std::vector<int> se_le;      // [nse][2][2] local edge: [col][0 bottom (zeta=-1/2), 1 top]
  std::vector<int> se_rev;     // [nse][2]
  std::vector<double> se_t;    // [nse][NS][3]
  std::vector<double> se_dlw;  // [nse][NS]  |dl| w at r_in
  std::vector<double> se_nang; // [nse][NS][3]
  std::vector<double> se_nradL, se_nradR;  // [nse][NS][3]

  // per sphere vertex (radial edges)
  std::vector<int> sv_nc;      // [nsv]
  std::vector<int> sv_col;     // [nsv][4]
  std::vector<int> sv_le;      // [nsv][4]
  std::vector<int> sv_fL, sv_fR;  // [nsv][4]
  std::vector<int> sv_fse;     // [nsv][4]   sphere edge of face j (faces (se, k) around the edge)
  std::vector<double> sv_fn;   // [nsv][4][NS][3]
  std::vector<double> sv_t;    // [nsv][3]
  std::vector<double> sv_dlw;  // [nsv][NS] at shell 0
};

// Builds every table.  Returns an empty string on success, else a message.
std::string build_tables(int n, int nr, double r_in, double r_out, int p, Tables& T);

// Time tables of the ADER-CG predictor (Eqs. 5.15-5.17, 5.24-5.29): wt = Gauss
// weights of the M-1 Gauss times, R = (K11)^-1 M1 ([M][M], row 1 zero).
void time_tables(int M, std::vector<double>& wt, std::vector<double>& R);

// The paper's reference triangular prism (unit edges, centroid at the origin;
// Sec. V.c, Eqs. 5.12-5.14, Fig. 7) at order p = 2, 3, 4: N = 6 / 15 / 26 nodes
// ([N][3]: the 6 vertices, top face zeta = +1/2 first, then p-2 equidistant nodes
// inside each of the 9 edges, then at p = 4 the two triangle-face centroids) and
// D ([3][N][N]): D^alpha_ij = d psi_j / d xi_alpha at node i.  Returns false if
// p is out of range or the Vandermonde matrix is singular.
bool prism_element(int p, std::vector<double>& nodes, std::vector<double>& D);

// Host geometry services for initial data.
void zone_cubature(const Tables& T, int nq, double* pts, double* w);
void edge_quadrature(const Tables& T, int nq, double* pts, double* tw);
void phi_from_circulation(const Tables& T, const double* circ, double* phi);
void zone_centroids(const Tables& T, double* xc, double* vol);
void face_geometry(const Tables& T, double* area, double* nrm);
void radial_face_quadrature(const Tables& T, int nq, double* pts, double* wn);

}  // namespace geo
