// Host-side FP64 mesh and table construction for the device kernels.
//
// Paper references (arXiv 1905.02504):
//   mesh / isoparametric map      Sec. II.a-II.b, Eq. 5.2-5.5
//   Taylor basis, moments, fits   Sec. III, Eqs. 3.1-3.4
//   divergence-free B (KKT)       Sec. IV.b steps 1-9, Eqs. 4.1-4.15
//   ADER matrices, nodal metrics  Sec. V.b-V.d, Eqs. 5.15-5.29, C.34-C.36
// The cubed sphere replaces the paper's icosahedral prisms; the reference
// element is the unit cube [-1/2,1/2]^3 with serendipity nodes (8/20/32).
#include "host_tables.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <set>
#include <tuple>

namespace geo {

using std::array;
using std::vector;
using V3 = array<double, 3>;

// ---------------------------------------------------------------------------
// small dense linear algebra (row major)
// ---------------------------------------------------------------------------
static bool invert_inplace(vector<double>& a, int n) {
  vector<double> inv(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    double best = std::fabs(a[col * n + col]);
    for (int r = col + 1; r < n; ++r) {
      double v = std::fabs(a[r * n + col]);
      if (v > best) { best = v; piv = r; }
    }
    if (best == 0.0) return false;
    if (piv != col) {
      for (int j = 0; j < n; ++j) {
        std::swap(a[col * n + j], a[piv * n + j]);
        std::swap(inv[col * n + j], inv[piv * n + j]);
      }
    }
    double d = 1.0 / a[col * n + col];
    for (int j = 0; j < n; ++j) { a[col * n + j] *= d; inv[col * n + j] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = a[r * n + col];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        a[r * n + j] -= f * a[col * n + j];
        inv[r * n + j] -= f * inv[col * n + j];
      }
    }
  }
  a.swap(inv);
  return true;
}

// Least-squares pseudo-inverse P (k x m) of A (m x k, m >= k, full column rank)
// by Householder QR: P = R^-1 Q^T.
static bool lsq_pinv(const vector<double>& Ain, int m, int k, vector<double>& P) {
  vector<double> A = Ain;                           // m x k
  vector<double> Qt(static_cast<size_t>(m) * m, 0.0);
  for (int i = 0; i < m; ++i) Qt[i * m + i] = 1.0;  // accumulates Q^T
  vector<double> v(m);
  for (int j = 0; j < k; ++j) {
    double nrm = 0.0;
    for (int i = j; i < m; ++i) nrm += A[i * k + j] * A[i * k + j];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) return false;
    double alpha = A[j * k + j] > 0 ? -nrm : nrm;
    for (int i = 0; i < m; ++i) v[i] = 0.0;
    v[j] = A[j * k + j] - alpha;
    for (int i = j + 1; i < m; ++i) v[i] = A[i * k + j];
    double vv = 0.0;
    for (int i = j; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    for (int c = 0; c < k; ++c) {
      double s = 0.0;
      for (int i = j; i < m; ++i) s += v[i] * A[i * k + c];
      s = 2.0 * s / vv;
      for (int i = j; i < m; ++i) A[i * k + c] -= s * v[i];
    }
    for (int c = 0; c < m; ++c) {
      double s = 0.0;
      for (int i = j; i < m; ++i) s += v[i] * Qt[i * m + c];
      s = 2.0 * s / vv;
      for (int i = j; i < m; ++i) Qt[i * m + c] -= s * v[i];
    }
  }
  // solve R P = (Q^T)[0:k, :]
  P.assign(static_cast<size_t>(k) * m, 0.0);
  for (int c = 0; c < m; ++c) {
    for (int i = k - 1; i >= 0; --i) {
      double s = Qt[i * m + c];
      for (int j = i + 1; j < k; ++j) s -= A[i * k + j] * P[j * m + c];
      if (A[i * k + i] == 0.0) return false;
      P[i * m + c] = s / A[i * k + i];
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// quadrature
// ---------------------------------------------------------------------------
// Gauss-Legendre on [-1/2, 1/2] (weights sum to 1), Newton iteration on P_n.
static void gauss_legendre(int n, vector<double>& x, vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    long double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    long double dp = 0;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = z;
      for (int l = 2; l <= n; ++l) {
        long double p2 = ((2 * l - 1) * z * p1 - (l - 1) * p0) / l;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1; }
      dp = n * (z * p1 - p0) / (z * z - 1);
      long double dz = p1 / dp;
      z -= dz;
      if (std::fabs(static_cast<double>(dz)) < 1e-19) break;
    }
    long double p0 = 1, p1 = z;
    for (int l = 2; l <= n; ++l) {
      long double p2 = ((2 * l - 1) * z * p1 - (l - 1) * p0) / l;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) { p1 = z; p0 = 1; }
    dp = n * (z * p1 - p0) / (z * z - 1);
    x[n - 1 - i] = static_cast<double>(0.5L * z);
    w[n - 1 - i] = static_cast<double>(1.0L / ((1 - z * z) * dp * dp));  // 2/(..) halved
  }
}

static void face_rule(int p, bool radial, vector<double>& uv, vector<double>& w) {
  int nu = 2, nv = 2;
  if (p == 4) { nu = 3; nv = radial ? 3 : 2; }
  vector<double> xu, wu, xv, wv;
  gauss_legendre(nu, xu, wu);
  gauss_legendre(nv, xv, wv);
  uv.clear();
  w.clear();
  for (int a = 0; a < nu; ++a)
    for (int b = 0; b < nv; ++b) {
      uv.push_back(xu[a]);
      uv.push_back(xv[b]);
      w.push_back(wu[a] * wv[b]);
    }
}

static void edge_rule(int p, vector<double>& t, vector<double>& w) {
  if (p == 2) { t = {0.0}; w = {1.0}; return; }
  if (p == 3) { gauss_legendre(2, t, w); return; }
  t = {-0.5, 0.0, 0.5};
  w = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0};
}

// ---------------------------------------------------------------------------
// dimensions
// ---------------------------------------------------------------------------
static vector<array<int, 3>> taylor_exps(int dmin, int dmax) {
  vector<array<int, 3>> out;
  for (int d = dmin; d <= dmax; ++d)
    for (int a = d; a >= 0; --a)
      for (int b = d - a; b >= 0; --b) out.push_back({a, b, d - a - b});
  return out;
}

Dims dims_for_order(int p) {
  Dims d{};
  d.P = p;
  d.N = (p == 2) ? 8 : (p == 3 ? 20 : 32);
  d.M = p;
  d.NC1 = static_cast<int>(taylor_exps(1, p - 1).size());
  d.NC = d.NC1 + 1;
  d.NB = d.NC + p * (p + 1) / 2;
  d.NQR = (p == 4) ? 9 : 4;
  d.NQS = (p == 4) ? 6 : 4;
  d.NQT = 2 * d.NQR + 4 * d.NQS;
  d.NS = (p == 2) ? 1 : (p == 3 ? 2 : 3);
  d.SMAX = (p == 2) ? 6 : (p == 3 ? 26 : 32);
  d.G = (p == 4) ? 2 : 1;
  d.NDIV = d.NC1;
  d.NBIN = 3 * d.NC + d.NQT + 6;
  d.NNZ = (p == 2) ? 16 : (p == 3 ? 96 : 192);
  d.NFN = (p == 2) ? 4 : (p == 3 ? 8 : 12);
  d.NEN = p;
  return d;
}

// ---------------------------------------------------------------------------
// reference hexahedron (serendipity, Eq. 5.3 on the unit cube)
// ---------------------------------------------------------------------------
static const int EDGE_AXIS[12] = {0, 0, 0, 0, 1, 1, 1, 1, 2, 2, 2, 2};
// the two fixed coordinates (in axis order, skipping the running axis)
static const double EDGE_FIX[12][2] = {{-.5, -.5}, {.5, -.5}, {-.5, .5}, {.5, .5},
                                       {-.5, -.5}, {.5, -.5}, {-.5, .5}, {.5, .5},
                                       {-.5, -.5}, {.5, -.5}, {-.5, .5}, {.5, .5}};
static const int FACE_AXIS[6] = {0, 0, 1, 1, 2, 2};
static const double FACE_SIDE[6] = {-.5, .5, -.5, .5, -.5, .5};
static const int FACE_U[6] = {1, 1, 0, 0, 0, 0};
static const int FACE_V[6] = {2, 2, 2, 2, 1, 1};

static V3 edge_point(int e, double t) {
  V3 x{};
  int ax = EDGE_AXIS[e];
  int q = 0;
  for (int a = 0; a < 3; ++a) x[a] = (a == ax) ? t : EDGE_FIX[e][q++];
  return x;
}

struct HexEl {
  int p = 0, N = 0;
  vector<array<int, 3>> ex;
  vector<V3> nodes;
  vector<double> coef;  // [mono][N]

  explicit HexEl(int p_) : p(p_) {
    int r = p - 1;
    for (int tot = 0; tot <= 3 * r; ++tot)
      for (int a = 0; a <= r; ++a)
        for (int b = 0; b <= r; ++b)
          for (int c = 0; c <= r; ++c) {
            if (a + b + c != tot) continue;
            int sl = (a >= 2 ? a : 0) + (b >= 2 ? b : 0) + (c >= 2 ? c : 0);
            if (sl <= r) ex.push_back({a, b, c});
          }
    for (int iz = 0; iz < 2; ++iz)
      for (int iy = 0; iy < 2; ++iy)
        for (int ix = 0; ix < 2; ++ix) nodes.push_back({ix - 0.5, iy - 0.5, iz - 0.5});
    for (int e = 0; e < 12; ++e)
      for (int s = 1; s < p - 1; ++s) nodes.push_back(edge_point(e, -0.5 + s / double(p - 1)));
    N = static_cast<int>(nodes.size());
    vector<double> Vm(static_cast<size_t>(N) * N);
    for (int i = 0; i < N; ++i)
      for (int m = 0; m < N; ++m) Vm[i * N + m] = mono(nodes[i].data(), m);
    invert_inplace(Vm, N);  // Vm^-1 [m][j]
    coef = Vm;
  }
  double mono(const double* x, int m) const {
    return std::pow(x[0], ex[m][0]) * std::pow(x[1], ex[m][1]) * std::pow(x[2], ex[m][2]);
  }
  double dmono(const double* x, int m, int ax) const {
    int e = ex[m][ax];
    if (e == 0) return 0.0;
    double v = e;
    for (int a = 0; a < 3; ++a) v *= std::pow(x[a], a == ax ? e - 1 : ex[m][a]);
    return v;
  }
  void basis(const double* x, double* psi) const {
    for (int j = 0; j < N; ++j) psi[j] = 0.0;
    for (int m = 0; m < N; ++m) {
      double v = mono(x, m);
      if (v == 0.0) continue;
      for (int j = 0; j < N; ++j) psi[j] += coef[m * N + j] * v;
    }
  }
  void dbasis(const double* x, int ax, double* d) const {
    for (int j = 0; j < N; ++j) d[j] = 0.0;
    for (int m = 0; m < N; ++m) {
      double v = dmono(x, m, ax);
      if (v == 0.0) continue;
      for (int j = 0; j < N; ++j) d[j] += coef[m * N + j] * v;
    }
  }
};

// ---------------------------------------------------------------------------
// cubed sphere
// ---------------------------------------------------------------------------
static const int FRAME[6][3][3] = {
    {{0, 1, 0}, {0, 0, 1}, {1, 0, 0}},  {{0, 0, 1}, {1, 0, 0}, {0, 1, 0}},
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},  {{0, 0, 1}, {0, 1, 0}, {-1, 0, 0}},
    {{1, 0, 0}, {0, 0, 1}, {0, -1, 0}}, {{0, 1, 0}, {1, 0, 0}, {0, 0, -1}}};

static V3 sphere_point(int f, double al, double be) {
  double ta = std::tan(al), tb = std::tan(be);
  V3 v;
  for (int d = 0; d < 3; ++d) v[d] = ta * FRAME[f][0][d] + tb * FRAME[f][1][d] + FRAME[f][2][d];
  double nn = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (auto& x : v) x /= nn;
  return v;
}

static V3 cross(const V3& a, const V3& b) {
  return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
static double dot(const V3& a, const V3& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm(const V3& a) { return std::sqrt(dot(a, a)); }

struct Builder {
  int n, nr, p;
  double r_in, r_out;
  HexEl el;
  Dims d;
  int ncol;
  vector<int> colf, coli, colj;
  Tables& T;
  vector<vector<int>> sv_cols, sv_edges;

  Builder(int n_, int nr_, double ri, double ro, int p_, Tables& T_)
      : n(n_), nr(nr_), p(p_), r_in(ri), r_out(ro), el(p_), d(dims_for_order(p_)), T(T_) {
    ncol = 6 * n * n;
    colf.resize(ncol);
    coli.resize(ncol);
    colj.resize(ncol);
    for (int c = 0; c < ncol; ++c) {
      colf[c] = c / (n * n);
      colj[c] = (c / n) % n;
      coli[c] = c % n;
    }
  }

  double radius(int k) const { return r_in * std::pow(r_out / r_in, double(k) / nr); }

  // isoparametric nodes X_i of zone (c, k): rho(zeta_i) P(alpha, beta)
  vector<V3> zone_nodes(int c, int k) const {
    vector<V3> X(el.N);
    double dd = 0.5 * M_PI / n;
    double r0 = radius(k), r1 = radius(k + 1);
    for (int i = 0; i < el.N; ++i) {
      const V3& xi = el.nodes[i];
      double al = -0.25 * M_PI + (coli[c] + xi[0] + 0.5) * dd;
      double be = -0.25 * M_PI + (colj[c] + xi[1] + 0.5) * dd;
      V3 P = sphere_point(colf[c], al, be);
      double rho = r0 * (0.5 - xi[2]) + r1 * (0.5 + xi[2]);
      for (int a = 0; a < 3; ++a) X[i][a] = rho * P[a];
    }
    return X;
  }
  V3 map_point(const vector<V3>& X, const V3& xi) const {
    vector<double> psi(el.N);
    el.basis(xi.data(), psi.data());
    V3 x{0, 0, 0};
    for (int i = 0; i < el.N; ++i)
      for (int a = 0; a < 3; ++a) x[a] += psi[i] * X[i][a];
    return x;
  }
  array<V3, 3> map_jac(const vector<V3>& X, const V3& xi) const {
    array<V3, 3> h{};
    vector<double> dps(el.N);
    for (int ax = 0; ax < 3; ++ax) {
      el.dbasis(xi.data(), ax, dps.data());
      h[ax] = {0, 0, 0};
      for (int i = 0; i < el.N; ++i)
        for (int a = 0; a < 3; ++a) h[ax][a] += dps[i] * X[i][a];
    }
    return h;
  }

  // cubature of a zone: points and physical weights
  struct Cub {
    vector<V3> x;
    vector<double> dV;
    double V = 0;
    V3 xc{0, 0, 0};
  };
  vector<V3> cub_ref;
  vector<double> cub_w;
  vector<double> cub_psi, cub_dpsi;  // [g][N], [g][3][N]
  void init_cubature() {
    int na = (p == 2) ? 3 : (p == 3 ? 6 : 11);
    int nrd = (p == 2) ? 2 : (p == 3 ? 3 : 4);
    vector<double> xa, wa, xr, wr;
    gauss_legendre(na, xa, wa);
    gauss_legendre(nrd, xr, wr);
    for (int a = 0; a < na; ++a)
      for (int b = 0; b < na; ++b)
        for (int c = 0; c < nrd; ++c) {
          cub_ref.push_back({xa[a], xa[b], xr[c]});
          cub_w.push_back(wa[a] * wa[b] * wr[c]);
        }
    int G = static_cast<int>(cub_ref.size());
    cub_psi.resize(static_cast<size_t>(G) * el.N);
    cub_dpsi.resize(static_cast<size_t>(G) * 3 * el.N);
    for (int g = 0; g < G; ++g) {
      el.basis(cub_ref[g].data(), &cub_psi[static_cast<size_t>(g) * el.N]);
      for (int ax = 0; ax < 3; ++ax)
        el.dbasis(cub_ref[g].data(), ax, &cub_dpsi[(static_cast<size_t>(g) * 3 + ax) * el.N]);
    }
  }
  Cub cubature(int c, int k) const {
    vector<V3> X = zone_nodes(c, k);
    Cub C;
    int G = static_cast<int>(cub_ref.size());
    C.x.resize(G);
    C.dV.resize(G);
    for (int g = 0; g < G; ++g) {
      V3 x{0, 0, 0};
      array<V3, 3> h{};
      const double* ps = &cub_psi[static_cast<size_t>(g) * el.N];
      for (int i = 0; i < el.N; ++i)
        for (int a = 0; a < 3; ++a) x[a] += ps[i] * X[i][a];
      for (int ax = 0; ax < 3; ++ax) {
        const double* dp = &cub_dpsi[(static_cast<size_t>(g) * 3 + ax) * el.N];
        h[ax] = {0, 0, 0};
        for (int i = 0; i < el.N; ++i)
          for (int a = 0; a < 3; ++a) h[ax][a] += dp[i] * X[i][a];
      }
      double J = dot(cross(h[0], h[1]), h[2]);
      C.x[g] = x;
      C.dV[g] = J * cub_w[g];
      C.V += C.dV[g];
      for (int a = 0; a < 3; ++a) C.xc[a] += C.dV[g] * x[a];
    }
    for (int a = 0; a < 3; ++a) C.xc[a] /= C.V;
    return C;
  }
  static double mono3(const V3& s, const array<int, 3>& e) {
    return std::pow(s[0], e[0]) * std::pow(s[1], e[1]) * std::pow(s[2], e[2]);
  }
  // <((x - xc0)/l0)^e> over the zone C
  vector<double> moments(const Cub& C, const V3& xc0, double l0,
                         const vector<array<int, 3>>& ex) const {
    vector<double> out(ex.size(), 0.0);
    for (size_t g = 0; g < C.x.size(); ++g) {
      V3 s;
      for (int a = 0; a < 3; ++a) s[a] = (C.x[g][a] - xc0[a]) / l0;
      for (size_t m = 0; m < ex.size(); ++m) out[m] += C.dV[g] * mono3(s, ex[m]);
    }
    for (auto& v : out) v /= C.V;
    return out;
  }

  // ---------------------------------------------------------------- topology
  void topology() {
    std::map<array<int, 3>, int> key2id;
    T.col_verts.assign(4 * ncol, 0);
    vector<V3> svdir;
    const int dij[4][2] = {{0, 0}, {1, 0}, {0, 1}, {1, 1}};
    for (int c = 0; c < ncol; ++c) {
      int f = colf[c];
      for (int q = 0; q < 4; ++q) {
        array<int, 3> key;
        int a = 2 * (coli[c] + dij[q][0]) - n, b = 2 * (colj[c] + dij[q][1]) - n;
        for (int dd = 0; dd < 3; ++dd) key[dd] = a * FRAME[f][0][dd] + b * FRAME[f][1][dd] + n * FRAME[f][2][dd];
        auto it = key2id.find(key);
        int id;
        if (it == key2id.end()) {
          id = static_cast<int>(key2id.size());
          key2id[key] = id;
          V3 v{double(key[0]), double(key[1]), double(key[2])};
          double nn = norm(v);
          for (auto& x : v) x /= nn;
          svdir.push_back(v);
        } else {
          id = it->second;
        }
        T.col_verts[4 * c + q] = id;
      }
    }
    T.nsv = static_cast<int>(key2id.size());
    // sides s (v00,v10), e (v10,v11), n (v01,v11), w (v00,v01)
    const int side_pair[4][2] = {{0, 1}, {1, 3}, {2, 3}, {0, 2}};
    const int ccw_pair[4][2] = {{0, 1}, {1, 3}, {3, 2}, {2, 0}};
    std::map<std::pair<int, int>, int> ekey;
    T.col_side_se.assign(4 * ncol, 0);
    T.col_side_sgn.assign(4 * ncol, 0);
    vector<vector<int>> se_cols;
    T.se_v.clear();
    for (int c = 0; c < ncol; ++c)
      for (int s = 0; s < 4; ++s) {
        int va = T.col_verts[4 * c + side_pair[s][0]], vb = T.col_verts[4 * c + side_pair[s][1]];
        auto key = std::make_pair(std::min(va, vb), std::max(va, vb));
        auto it = ekey.find(key);
        int e;
        if (it == ekey.end()) {
          e = static_cast<int>(ekey.size());
          ekey[key] = e;
          T.se_v.push_back(key.first);
          T.se_v.push_back(key.second);
          se_cols.emplace_back();
        } else {
          e = it->second;
        }
        se_cols[e].push_back(c);
        T.col_side_se[4 * c + s] = e;
        int ca = T.col_verts[4 * c + ccw_pair[s][0]];
        T.col_side_sgn[4 * c + s] = (T.se_v[2 * e] == ca) ? 1 : -1;
      }
    T.nse = static_cast<int>(ekey.size());
    T.se_col.assign(2 * T.nse, -1);
    for (int e = 0; e < T.nse; ++e)
      for (int c : se_cols[e]) {
        int s = 0;
        while (T.col_side_se[4 * c + s] != e) ++s;
        T.se_col[2 * e + (T.col_side_sgn[4 * c + s] > 0 ? 0 : 1)] = c;
      }
    sv_cols.assign(T.nsv, {});
    sv_edges.assign(T.nsv, {});
    for (int c = 0; c < ncol; ++c)
      for (int q = 0; q < 4; ++q) sv_cols[T.col_verts[4 * c + q]].push_back(c);
    for (int e = 0; e < T.nse; ++e) {
      sv_edges[T.se_v[2 * e]].push_back(e);
      sv_edges[T.se_v[2 * e + 1]].push_back(e);
    }
    T.sv_t.assign(3 * T.nsv, 0.0);
    for (int v = 0; v < T.nsv; ++v)
      for (int a = 0; a < 3; ++a) T.sv_t[3 * v + a] = svdir[v][a];
  }
  // local face 0..3 -> side (s,e,n,w)
  static int side_of_lf(int lf) { return lf == 0 ? 3 : (lf == 1 ? 1 : (lf == 2 ? 0 : 2)); }
  static int lf_of_side(int s) { return s == 0 ? 2 : (s == 1 ? 1 : (s == 2 ? 3 : 0)); }
  int angular_nb(int c, int lf) const {
    int e = T.col_side_se[4 * c + side_of_lf(lf)];
    return T.se_col[2 * e] == c ? T.se_col[2 * e + 1] : T.se_col[2 * e];
  }
  std::pair<int, int> face_nb(int c, int k, int lf) const {
    if (lf < 4) return {angular_nb(c, lf), k};
    return {c, lf == 4 ? k - 1 : k + 1};
  }
  vector<std::pair<int, int>> central_stencil(int c) const {
    std::set<std::pair<int, int>> st;
    if (p == 2) {
      for (int lf = 0; lf < 6; ++lf) st.insert(face_nb(c, 0, lf));
    } else {
      std::set<int> cols;
      for (int q = 0; q < 4; ++q)
        for (int cc : sv_cols[T.col_verts[4 * c + q]]) cols.insert(cc);
      for (int cc : cols)
        for (int dk = -1; dk <= 1; ++dk) st.insert({cc, dk});
      st.erase({c, 0});
      if (p == 4) {
        st.insert({c, -2});
        st.insert({c, 2});
        for (int lf = 0; lf < 4; ++lf) {
          int c1 = angular_nb(c, lf);
          int se = T.col_side_se[4 * c + side_of_lf(lf)];
          int s1 = 0;
          while (T.col_side_se[4 * c1 + s1] != se) ++s1;
          int se2 = T.col_side_se[4 * c1 + (s1 + 2) % 4];
          int c2 = T.se_col[2 * se2] == c1 ? T.se_col[2 * se2 + 1] : T.se_col[2 * se2];
          st.insert({c2, 0});
        }
      }
    }
    return vector<std::pair<int, int>>(st.begin(), st.end());
  }

  // ---------------------------------------------------------------- per column
  void column_tables(int c, const vector<array<int, 3>>& tay, const vector<array<int, 3>>& tay_all,
                     const vector<vector<array<int, 3>>>& terms) {
    const int N = d.N, NC1 = d.NC1, SMAX = d.SMAX, NQT = d.NQT, NB = d.NB, NBIN = d.NBIN;
    Cub C0 = cubature(c, 0);
    double V0 = C0.V, l0 = std::cbrt(V0);
    V3 xc0 = C0.xc;
    T.V0[c] = V0;
    T.l0[c] = l0;
    for (int a = 0; a < 3; ++a) T.xc0[3 * c + a] = xc0[a];
    vector<double> mean_all = moments(C0, xc0, l0, tay_all);  // degree 1..p
    auto taylor_val = [&](const V3& s, int m) { return mono3(s, tay_all[m]) - mean_all[m]; };
    // ---- WENO central stencil
    auto st = central_stencil(c);
    int ns = static_cast<int>(st.size());
    T.st_n[c] = ns;
    vector<double> A(static_cast<size_t>(ns) * NC1);
    for (int j = 0; j < ns; ++j) {
      T.st_nb[static_cast<size_t>(c) * SMAX + j] = (st[j].first << 3) | (st[j].second + 3);
      Cub Cj = cubature(st[j].first, st[j].second);
      vector<double> mj = moments(Cj, xc0, l0, tay);
      for (int m = 0; m < NC1; ++m) A[j * NC1 + m] = mj[m] - mean_all[m];
    }
    vector<double> P;
    lsq_pinv(A, ns, NC1, P);
    for (int m = 0; m < NC1; ++m)
      for (int j = 0; j < ns; ++j) T.pinvH[(static_cast<size_t>(c) * NC1 + m) * SMAX + j] = P[m * ns + j];
    // ---- octant stencils: o = ox + 2 oy + 4 oz
    for (int o = 0; o < 8; ++o) {
      int sel[3] = {(o & 1) ? 1 : 0, (o & 2) ? 3 : 2, (o & 4) ? 5 : 4};
      vector<double> Ao(9);
      for (int q = 0; q < 3; ++q) {
        auto nb = face_nb(c, 0, sel[q]);
        T.oct_nb[(static_cast<size_t>(c) * 8 + o) * 3 + q] = (nb.first << 3) | (nb.second + 3);
        Cub Cj = cubature(nb.first, nb.second);
        for (int a = 0; a < 3; ++a) Ao[q * 3 + a] = (Cj.xc[a] - xc0[a]) / l0;
      }
      invert_inplace(Ao, 3);
      for (int i = 0; i < 9; ++i) T.oct_inv[(static_cast<size_t>(c) * 8 + o) * 9 + i] = Ao[i];
    }
    // ---- smoothness quadratic form: sum_{1<=|a|<=p-1} <d^a phi_m d^a phi_m'>
    {
      vector<double> Qm(static_cast<size_t>(NC1) * NC1, 0.0);
      auto derivs = taylor_exps(1, p - 1);
      vector<double> dv(NC1);
      for (size_t g = 0; g < C0.x.size(); ++g) {
        V3 s;
        for (int a = 0; a < 3; ++a) s[a] = (C0.x[g][a] - xc0[a]) / l0;
        for (auto& al : derivs) {
          for (int m = 0; m < NC1; ++m) {
            const auto& e = tay[m];
            double coef = 1.0;
            bool zero = false;
            array<int, 3> r{};
            for (int a = 0; a < 3; ++a) {
              if (e[a] < al[a]) { zero = true; break; }
              for (int t = 0; t < al[a]; ++t) coef *= (e[a] - t);
              r[a] = e[a] - al[a];
            }
            dv[m] = zero ? 0.0 : coef * mono3(s, r);
          }
          for (int i = 0; i < NC1; ++i)
            for (int j = 0; j < NC1; ++j) Qm[i * NC1 + j] += C0.dV[g] * dv[i] * dv[j];
        }
      }
      for (int i = 0; i < NC1 * NC1; ++i) T.Q[static_cast<size_t>(c) * NC1 * NC1 + i] = Qm[i] / V0;
    }
    // ---- faces of the zone at shell 0
    vector<V3> X0 = zone_nodes(c, 0);
    vector<V3> fx(NQT), fn(NQT);
    vector<double> fw(NQT), fdA(NQT);
    vector<V3> fref(NQT);
    double Ssum = 0.0;
    for (int lf = 0; lf < 6; ++lf) {
      vector<double> uv, w;
      face_rule(p, lf >= 4, uv, w);
      int nq = static_cast<int>(w.size());
      double A_lf = 0.0;
      for (int q = 0; q < nq; ++q) {
        V3 xi{};
        xi[FACE_U[lf]] = uv[2 * q];
        xi[FACE_V[lf]] = uv[2 * q + 1];
        xi[FACE_AXIS[lf]] = FACE_SIDE[lf];
        auto h = map_jac(X0, xi);
        int a = FACE_AXIS[lf];
        V3 vec = cross(h[(a + 1) % 3], h[(a + 2) % 3]);
        double sg = FACE_SIDE[lf] > 0 ? 1.0 : -1.0;
        double dA = norm(vec);
        int idx = T.foff[lf] + q;
        for (int b = 0; b < 3; ++b) fn[idx][b] = sg * vec[b] / dA;
        fx[idx] = map_point(X0, xi);
        fw[idx] = w[q];
        fdA[idx] = dA;
        fref[idx] = xi;
        A_lf += w[q] * dA;
      }
      T.A0[6 * c + lf] = A_lf;
      Ssum += A_lf;
      for (int q = 0; q < nq; ++q) {
        int idx = T.foff[lf] + q;
        T.wF[static_cast<size_t>(c) * NQT + idx] = fw[idx] * fdA[idx] / A_lf;
        T.WF[static_cast<size_t>(c) * NQT + idx] = fw[idx] * fdA[idx];
        for (int b = 0; b < 3; ++b) T.nF[(static_cast<size_t>(c) * NQT + idx) * 3 + b] = fn[idx][b];
        V3 s;
        for (int a = 0; a < 3; ++a) s[a] = (fx[idx][a] - xc0[a]) / l0;
        for (int m = 0; m < NC1; ++m) T.TF[(static_cast<size_t>(c) * NQT + idx) * NC1 + m] = taylor_val(s, m);
      }
    }
    T.S0[c] = Ssum;
    // ---- nodal metrics (Sec. V.d step 4)
    vector<double> J(N);
    vector<array<V3, 3>> Sn(N);
    for (int i = 0; i < N; ++i) {
      auto h = map_jac(X0, el.nodes[i]);
      J[i] = dot(cross(h[0], h[1]), h[2]);
      Sn[i][0] = cross(h[1], h[2]);
      Sn[i][1] = cross(h[2], h[0]);
      Sn[i][2] = cross(h[0], h[1]);
      T.J0[static_cast<size_t>(c) * N + i] = J[i];
      T.iJ0[static_cast<size_t>(c) * N + i] = 1.0 / J[i];
      for (int al = 0; al < 3; ++al)
        for (int b = 0; b < 3; ++b) T.Sm[((static_cast<size_t>(c) * 3 + al) * N + i) * 3 + b] = Sn[i][al][b];
      V3 s;
      for (int a = 0; a < 3; ++a) s[a] = (X0[i][a] - xc0[a]) / l0;
      for (int m = 0; m < NC1; ++m) T.TN[(static_cast<size_t>(c) * N + i) * NC1 + m] = taylor_val(s, m);
    }
    for (int i = 0; i < N; ++i) {
      V3 g{0, 0, 0};
      for (int al = 0; al < 3; ++al)
        for (int j = 0; j < N; ++j)
          for (int b = 0; b < 3; ++b) g[b] += T.D[(static_cast<size_t>(al) * N + i) * N + j] * Sn[j][al][b];
      for (int b = 0; b < 3; ++b) T.gcl[(static_cast<size_t>(c) * N + i) * 3 + b] = g[b];
    }
    for (int idx = 0; idx < NQT; ++idx) {
      double s = 0.0;
      for (int i = 0; i < N; ++i) s += T.psiF[static_cast<size_t>(idx) * N + i] * J[i];
      T.JF[static_cast<size_t>(c) * NQT + idx] = s;
    }
    for (int le = 0; le < 12; ++le)
      for (int s = 0; s < d.NS; ++s) {
        double v = 0.0;
        for (int i = 0; i < N; ++i) v += T.psiE[(static_cast<size_t>(le) * d.NS + s) * N + i] * J[i];
        T.JE[(static_cast<size_t>(c) * 12 + le) * d.NS + s] = v;
      }
    // ---- divergence-free reconstruction: KKT (Sec. IV.b steps 3-9)
    {
      const int nx = 3 * NB;
      const int ndiv = d.NDIV;
      const int nC = ndiv + 6;
      const int nrow = nx + NQT;
      // term values at face points
      vector<double> means_t(3 * NB, 0.0);
      for (int dc = 0; dc < 3; ++dc) {
        vector<double> mm = moments(C0, xc0, l0, terms[dc]);
        for (int t = 1; t < NB; ++t) means_t[dc * NB + t] = mm[t];
      }
      auto term_val = [&](const V3& s, int dc, int t) {
        if (t == 0) return 1.0;
        return mono3(s, terms[dc][t]) - means_t[dc * NB + t];
      };
      vector<double> Am(static_cast<size_t>(nrow) * nx, 0.0);
      for (int i = 0; i < nx; ++i) Am[static_cast<size_t>(i) * nx + i] = 1.0;
      vector<double> Cm(static_cast<size_t>(nC) * nx, 0.0);
      for (int idx = 0; idx < NQT; ++idx) {
        V3 s;
        for (int a = 0; a < 3; ++a) s[a] = (fx[idx][a] - xc0[a]) / l0;
        int lf = 0;
        while (idx >= T.foff[lf + 1]) ++lf;
        double wq = T.wF[static_cast<size_t>(c) * NQT + idx];
        for (int dc = 0; dc < 3; ++dc)
          for (int t = 0; t < NB; ++t) {
            double v = fn[idx][dc] * term_val(s, dc, t);
            Am[static_cast<size_t>(nx + idx) * nx + dc * NB + t] = v;
            Cm[static_cast<size_t>(ndiv + lf) * nx + dc * NB + t] += wq * v;
          }
      }
      // div constraints: coefficient of monomial mu (degree 1..p-1) of sum_d d_d B^d
      for (int r = 0; r < ndiv; ++r) {
        const auto& mu = tay[r];
        for (int dc = 0; dc < 3; ++dc)
          for (int t = 1; t < NB; ++t) {
            auto e = terms[dc][t];
            if (e[dc] == 0) continue;
            array<int, 3> lo = e;
            lo[dc] -= 1;
            if (lo == mu) Cm[static_cast<size_t>(r) * nx + dc * NB + t] = e[dc];
          }
      }
      const int nk = nx + nC;
      vector<double> K(static_cast<size_t>(nk) * nk, 0.0);
      for (int i = 0; i < nx; ++i)
        for (int j = 0; j < nx; ++j) {
          double s = 0.0;
          for (int r = 0; r < nrow; ++r) s += Am[static_cast<size_t>(r) * nx + i] * Am[static_cast<size_t>(r) * nx + j];
          K[static_cast<size_t>(i) * nk + j] = s;
        }
      for (int r = 0; r < nC; ++r)
        for (int j = 0; j < nx; ++j) {
          K[static_cast<size_t>(nx + r) * nk + j] = Cm[static_cast<size_t>(r) * nx + j];
          K[static_cast<size_t>(j) * nk + nx + r] = Cm[static_cast<size_t>(r) * nx + j];
        }
      invert_inplace(K, nk);
      // G_in (nx x NBIN): x = Kinv11 A^T b + Kinv12 d
      vector<double> Gin(static_cast<size_t>(nx) * NBIN, 0.0);
      for (int i = 0; i < nx; ++i) {
        // columns for the WENO modes of component dc, term t < NC (row dc*NB+t of A = identity)
        for (int dc = 0; dc < 3; ++dc)
          for (int t = 0; t < d.NC; ++t) {
            double s = 0.0;
            for (int j = 0; j < nx; ++j)
              s += K[static_cast<size_t>(i) * nk + j] * Am[static_cast<size_t>(dc * NB + t) * nx + j];
            Gin[static_cast<size_t>(i) * NBIN + dc * d.NC + t] = s;
          }
        for (int idx = 0; idx < NQT; ++idx) {
          double s = 0.0;
          for (int j = 0; j < nx; ++j)
            s += K[static_cast<size_t>(i) * nk + j] * Am[static_cast<size_t>(nx + idx) * nx + j];
          Gin[static_cast<size_t>(i) * NBIN + 3 * d.NC + idx] = s;
        }
        for (int lf = 0; lf < 6; ++lf)
          Gin[static_cast<size_t>(i) * NBIN + 3 * d.NC + NQT + lf] = K[static_cast<size_t>(i) * nk + nx + ndiv + lf];
      }
      // output rows: the three means, then B_d at every node
      for (int dc = 0; dc < 3; ++dc)
        for (int b = 0; b < NBIN; ++b)
          T.GB[(static_cast<size_t>(c) * (3 + 3 * N) + dc) * NBIN + b] = Gin[static_cast<size_t>(dc * NB) * NBIN + b];
      for (int dc = 0; dc < 3; ++dc)
        for (int i = 0; i < N; ++i) {
          V3 s;
          for (int a = 0; a < 3; ++a) s[a] = (X0[i][a] - xc0[a]) / l0;
          vector<double> tv(NB);
          for (int t = 0; t < NB; ++t) tv[t] = term_val(s, dc, t);
          for (int b = 0; b < NBIN; ++b) {
            double acc = 0.0;
            for (int t = 0; t < NB; ++t) acc += tv[t] * Gin[static_cast<size_t>(dc * NB + t) * NBIN + b];
            T.GB[(static_cast<size_t>(c) * (3 + 3 * N) + 3 + dc * N + i) * NBIN + b] = acc;
          }
        }
    }
  }

  // local edge of column c for side s, bottom (zeta=-1/2) or top
  static int local_edge(int s, int top) {
    if (s == 0 || s == 2) return (s == 2 ? 1 : 0) + 2 * top;  // along xi
    return 4 + (s == 1 ? 1 : 0) + 2 * top;                      // along eta
  }

  void sphere_edge_tables() {
    const int NS = d.NS, NQS = d.NQS;
    vector<double> te, we;
    edge_rule(p, te, we);
    for (int e = 0; e < T.nse; ++e) {
      int cols[2] = {T.se_col[2 * e], T.se_col[2 * e + 1]};
      int sides[2];
      for (int q = 0; q < 2; ++q) {
        int s = 0;
        while (T.col_side_se[4 * cols[q] + s] != e) ++s;
        sides[q] = s;
        T.se_lf[2 * e + q] = lf_of_side(s);
        T.se_le[(2 * e + q) * 2 + 0] = local_edge(s, 0);
        T.se_le[(2 * e + q) * 2 + 1] = local_edge(s, 1);
      }
      vector<V3> XL = zone_nodes(cols[0], 0), XR = zone_nodes(cols[1], 0);
      // face point correspondence
      {
        vector<double> uv, w;
        face_rule(p, false, uv, w);
        int lfL = T.se_lf[2 * e], lfR = T.se_lf[2 * e + 1];
        vector<V3> pl(NQS), pr(NQS);
        for (int q = 0; q < NQS; ++q) {
          V3 a{}, b{};
          a[FACE_U[lfL]] = uv[2 * q]; a[FACE_V[lfL]] = uv[2 * q + 1]; a[FACE_AXIS[lfL]] = FACE_SIDE[lfL];
          b[FACE_U[lfR]] = uv[2 * q]; b[FACE_V[lfR]] = uv[2 * q + 1]; b[FACE_AXIS[lfR]] = FACE_SIDE[lfR];
          pl[q] = map_point(XL, a);
          pr[q] = map_point(XR, b);
        }
        for (int q = 0; q < NQS; ++q) {
          int best = 0;
          double bd = 1e300;
          for (int r = 0; r < NQS; ++r) {
            V3 dd{pl[q][0] - pr[r][0], pl[q][1] - pr[r][1], pl[q][2] - pr[r][2]};
            double v = norm(dd);
            if (v < bd) { bd = v; best = r; }
          }
          T.se_perm[static_cast<size_t>(e) * NQS + q] = best;
        }
      }
      // edge geometry at r_in along the canonical direction va -> vb
      int leL = T.se_le[(2 * e) * 2 + 0];
      int ax = EDGE_AXIS[leL];
      V3 dirv;
      for (int a = 0; a < 3; ++a) dirv[a] = T.sv_t[3 * T.se_v[2 * e + 1] + a] - T.sv_t[3 * T.se_v[2 * e] + a];
      {
        auto h = map_jac(XL, edge_point(leL, 0.0));
        T.se_rev[2 * e] = dot(h[ax], dirv) < 0 ? 1 : 0;
        int leR = T.se_le[(2 * e + 1) * 2 + 0];
        auto hr = map_jac(XR, edge_point(leR, 0.0));
        T.se_rev[2 * e + 1] = dot(hr[EDGE_AXIS[leR]], dirv) < 0 ? 1 : 0;
      }
      int revL = T.se_rev[2 * e];
      for (int s = 0; s < NS; ++s) {
        int sl = revL ? NS - 1 - s : s;           // L-local point of canonical point s
        V3 xi = edge_point(leL, te[sl]);
        auto h = map_jac(XL, xi);
        double dl = norm(h[ax]);
        double sg = revL ? -1.0 : 1.0;
        for (int a = 0; a < 3; ++a) T.se_t[(static_cast<size_t>(e) * NS + s) * 3 + a] = sg * h[ax][a] / dl;
        T.se_dlw[static_cast<size_t>(e) * NS + s] = dl * we[sl];
        // canonical normal of the angular face = outward normal of L's side face
        int lfL = T.se_lf[2 * e];
        int fa = FACE_AXIS[lfL];
        V3 vec = cross(h[(fa + 1) % 3], h[(fa + 2) % 3]);
        double fs = FACE_SIDE[lfL] > 0 ? 1.0 : -1.0;
        double nv = norm(vec);
        for (int a = 0; a < 3; ++a) T.se_nang[(static_cast<size_t>(e) * NS + s) * 3 + a] = fs * vec[a] / nv;
        // canonical normal (+r) of the radial faces of L and R at this point:
        // minus the outward normal of local face 4 (zeta=-1/2)
        V3 v4 = cross(h[0], h[1]);
        double n4 = norm(v4);
        for (int a = 0; a < 3; ++a) T.se_nradL[(static_cast<size_t>(e) * NS + s) * 3 + a] = v4[a] / n4;
        int leR = T.se_le[(2 * e + 1) * 2 + 0];
        int sr = T.se_rev[2 * e + 1] ? NS - 1 - s : s;
        auto hr = map_jac(XR, edge_point(leR, te[sr]));
        V3 v4r = cross(hr[0], hr[1]);
        double n4r = norm(v4r);
        for (int a = 0; a < 3; ++a) T.se_nradR[(static_cast<size_t>(e) * NS + s) * 3 + a] = v4r[a] / n4r;
      }
    }
  }

  void sphere_vertex_tables() {
    const int NS = d.NS;
    vector<double> te, we;
    edge_rule(p, te, we);
    for (int v = 0; v < T.nsv; ++v) {
      int nc = static_cast<int>(sv_cols[v].size());
      T.sv_nc[v] = nc;
      for (int j = 0; j < 4; ++j) {
        T.sv_col[4 * v + j] = -1;
        T.sv_le[4 * v + j] = 0;
        T.sv_fL[4 * v + j] = 0;
        T.sv_fR[4 * v + j] = 0;
      }
      for (int j = 0; j < nc; ++j) {
        int c = sv_cols[v][j];
        int corner = 0;
        while (T.col_verts[4 * c + corner] != v) ++corner;
        T.sv_col[4 * v + j] = c;
        T.sv_le[4 * v + j] = 8 + (corner % 2) + 2 * (corner / 2);
      }
      // radial edge geometry from the first column (direction +zeta = +r)
      {
        int c = sv_cols[v][0];
        vector<V3> X = zone_nodes(c, 0);
        int le = T.sv_le[4 * v];
        for (int s = 0; s < NS; ++s) {
          auto h = map_jac(X, edge_point(le, te[s]));
          T.sv_dlw[static_cast<size_t>(v) * NS + s] = norm(h[2]) * we[s];
          // radial edge: x = rho(zeta) P_v, so the tangent is the vertex direction
          if (s == 0)
            for (int a = 0; a < 3; ++a) T.sv_t[3 * v + a] = h[2][a] / norm(h[2]);
        }
      }
      int nf = static_cast<int>(sv_edges[v].size());
      for (int j = 0; j < nf; ++j) {
        int e = sv_edges[v][j];
        int cL = T.se_col[2 * e], cR = T.se_col[2 * e + 1];
        int iL = -1, iR = -1;
        for (int q = 0; q < nc; ++q) {
          if (sv_cols[v][q] == cL) iL = q;
          if (sv_cols[v][q] == cR) iR = q;
        }
        T.sv_fL[4 * v + j] = iL;
        T.sv_fR[4 * v + j] = iR;
        T.sv_fse[4 * v + j] = e;
        vector<V3> X = zone_nodes(cL, 0);
        int le = T.sv_le[4 * v + iL];
        int lfL = T.se_lf[2 * e];
        int fa = FACE_AXIS[lfL];
        double fs = FACE_SIDE[lfL] > 0 ? 1.0 : -1.0;
        for (int s = 0; s < NS; ++s) {
          auto h = map_jac(X, edge_point(le, te[s]));
          V3 vec = cross(h[(fa + 1) % 3], h[(fa + 2) % 3]);
          double nv = norm(vec);
          for (int a = 0; a < 3; ++a)
            T.sv_fn[((static_cast<size_t>(v) * 4 + j) * NS + s) * 3 + a] = fs * vec[a] / nv;
        }
      }
    }
  }

  // CSC lists of D^alpha and the face / edge supports of the point evaluations
  std::string sparse_forms() {
    const int N = d.N, NS = d.NS, NQT = d.NQT;
    double dmax = 0.0;
    for (double v : T.D) dmax = std::max(dmax, std::fabs(v));
    const double tol = 1e-13 * dmax;
    T.Dptr.assign(3 * (N + 1), 0);
    T.Drow.clear();
    T.Dval.clear();
    for (int a = 0; a < 3; ++a) {
      int cnt = 0;
      for (int j = 0; j < N; ++j) {
        T.Dptr[a * (N + 1) + j] = cnt;
        for (int i = 0; i < N; ++i) {
          double v = T.D[(static_cast<size_t>(a) * N + i) * N + j];
          if (std::fabs(v) > tol) {
            T.Drow.push_back(i);
            T.Dval.push_back(v);
            ++cnt;
          }
        }
      }
      T.Dptr[a * (N + 1) + N] = cnt;
      if (cnt != d.NNZ) return "internal: unexpected sparsity of the derivative matrices";
    }
    T.fnode.assign(6 * d.NFN, 0);
    T.psiFc.assign(static_cast<size_t>(NQT) * d.NFN, 0.0);
    for (int lf = 0; lf < 6; ++lf) {
      int cnt = 0;
      for (int i = 0; i < N; ++i)
        if (el.nodes[i][FACE_AXIS[lf]] == FACE_SIDE[lf]) {
          if (cnt >= d.NFN) return "internal: face node count";
          T.fnode[lf * d.NFN + cnt++] = i;
        }
      if (cnt != d.NFN) return "internal: face node count";
      for (int q = T.foff[lf]; q < T.foff[lf + 1]; ++q)
        for (int i = 0; i < N; ++i) {
          double v = T.psiF[static_cast<size_t>(q) * N + i];
          int a = -1;
          for (int t = 0; t < d.NFN; ++t)
            if (T.fnode[lf * d.NFN + t] == i) a = t;
          if (a < 0) {
            if (std::fabs(v) > 1e-12) return "internal: basis not supported on the face nodes";
          } else {
            T.psiFc[static_cast<size_t>(q) * d.NFN + a] = v;
          }
        }
    }
    T.enode.assign(12 * d.NEN, 0);
    T.psiEc.assign(static_cast<size_t>(12) * NS * d.NEN, 0.0);
    for (int le = 0; le < 12; ++le) {
      int ax = EDGE_AXIS[le];
      int cnt = 0;
      for (int i = 0; i < N; ++i) {
        bool on = true;
        int qq = 0;
        for (int a = 0; a < 3; ++a) {
          if (a == ax) continue;
          if (el.nodes[i][a] != EDGE_FIX[le][qq]) on = false;
          ++qq;
        }
        if (on) {
          if (cnt >= d.NEN) return "internal: edge node count";
          T.enode[le * d.NEN + cnt++] = i;
        }
      }
      if (cnt != d.NEN) return "internal: edge node count";
      for (int s = 0; s < NS; ++s)
        for (int i = 0; i < N; ++i) {
          double v = T.psiE[(static_cast<size_t>(le) * NS + s) * N + i];
          int a = -1;
          for (int t = 0; t < d.NEN; ++t)
            if (T.enode[le * d.NEN + t] == i) a = t;
          if (a < 0) {
            if (std::fabs(v) > 1e-12) return "internal: basis not supported on the edge nodes";
          } else {
            T.psiEc[(static_cast<size_t>(le) * NS + s) * d.NEN + a] = v;
          }
        }
    }
    return "";
  }

  std::string build() {
    T.d = d;
    T.n = n;
    T.nr = nr;
    T.ncol = ncol;
    T.r_in = r_in;
    T.r_out = r_out;
    T.q = std::pow(r_out / r_in, 1.0 / nr);
    const int N = d.N, M = d.M, NS = d.NS, NQT = d.NQT;
    // reference element tables
    T.D.assign(static_cast<size_t>(3) * N * N, 0.0);
    for (int ax = 0; ax < 3; ++ax)
      for (int i = 0; i < N; ++i) el.dbasis(el.nodes[i].data(), ax, &T.D[(static_cast<size_t>(ax) * N + i) * N]);
    // time: tau_1 = 0 and Gauss points; R = (K11)^-1 M1.
    time_tables(M, T.wt, T.R);
    T.foff.assign(7, 0);
    for (int lf = 0; lf < 6; ++lf) T.foff[lf + 1] = T.foff[lf] + (lf >= 4 ? d.NQR : d.NQS);
    T.psiF.assign(static_cast<size_t>(NQT) * N, 0.0);
    for (int lf = 0; lf < 6; ++lf) {
      vector<double> uv, w;
      face_rule(p, lf >= 4, uv, w);
      for (size_t q = 0; q < w.size(); ++q) {
        V3 xi{};
        xi[FACE_U[lf]] = uv[2 * q];
        xi[FACE_V[lf]] = uv[2 * q + 1];
        xi[FACE_AXIS[lf]] = FACE_SIDE[lf];
        el.basis(xi.data(), &T.psiF[(static_cast<size_t>(T.foff[lf]) + q) * N]);
      }
    }
    {
      vector<double> te, we;
      edge_rule(p, te, we);
      T.wE = we;
      T.psiE.assign(static_cast<size_t>(12) * NS * N, 0.0);
      for (int le = 0; le < 12; ++le)
        for (int s = 0; s < NS; ++s) {
          V3 xi = edge_point(le, te[s]);
          el.basis(xi.data(), &T.psiE[(static_cast<size_t>(le) * NS + s) * N]);
        }
    }
    {
      std::string msg = sparse_forms();
      if (!msg.empty()) return msg;
    }
    topology();
    T.Z = static_cast<int64_t>(ncol) * nr;
    T.F_rad = static_cast<int64_t>(ncol) * (nr + 1);
    T.F = T.F_rad + static_cast<int64_t>(T.nse) * nr;
    T.E_rad = static_cast<int64_t>(T.nsv) * nr;
    T.E = T.E_rad + static_cast<int64_t>(T.nse) * (nr + 1);
    init_cubature();
    const size_t nc = ncol;
    T.st_n.assign(nc, 0);
    T.st_nb.assign(nc * d.SMAX, 3);
    T.pinvH.assign(nc * d.NC1 * d.SMAX, 0.0);
    T.oct_nb.assign(nc * 24, 0);
    T.oct_inv.assign(nc * 72, 0.0);
    T.Q.assign(nc * d.NC1 * d.NC1, 0.0);
    T.V0.assign(nc, 0.0);
    T.l0.assign(nc, 0.0);
    T.S0.assign(nc, 0.0);
    T.xc0.assign(nc * 3, 0.0);
    T.A0.assign(nc * 6, 0.0);
    T.TF.assign(nc * NQT * d.NC1, 0.0);
    T.nF.assign(nc * NQT * 3, 0.0);
    T.wF.assign(nc * NQT, 0.0);
    T.WF.assign(nc * NQT, 0.0);
    T.GB.assign(nc * (3 + 3 * N) * d.NBIN, 0.0);
    T.TN.assign(nc * N * d.NC1, 0.0);
    T.J0.assign(nc * N, 0.0);
    T.iJ0.assign(nc * N, 0.0);
    T.Sm.assign(nc * 9 * N, 0.0);
    T.gcl.assign(nc * N * 3, 0.0);
    T.JF.assign(nc * NQT, 0.0);
    T.JE.assign(nc * 12 * NS, 0.0);
    auto tay = taylor_exps(1, p - 1);
    auto tay_all = taylor_exps(1, p);
    vector<vector<array<int, 3>>> terms(3);
    for (int dc = 0; dc < 3; ++dc) {
      terms[dc] = taylor_exps(0, p - 1);
      for (auto& e : taylor_exps(p, p))
        if (e[dc] >= 1) terms[dc].push_back(e);
      if (static_cast<int>(terms[dc].size()) != d.NB) return "internal: divergence-free term count";
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int c = 0; c < ncol; ++c) column_tables(c, tay, tay_all, terms);
    T.se_perm.assign(static_cast<size_t>(T.nse) * d.NQS, 0);
    T.se_lf.assign(2 * T.nse, 0);
    T.se_le.assign(4 * T.nse, 0);
    T.se_rev.assign(2 * T.nse, 0);
    T.se_t.assign(static_cast<size_t>(T.nse) * NS * 3, 0.0);
    T.se_dlw.assign(static_cast<size_t>(T.nse) * NS, 0.0);
    T.se_nang.assign(static_cast<size_t>(T.nse) * NS * 3, 0.0);
    T.se_nradL.assign(static_cast<size_t>(T.nse) * NS * 3, 0.0);
    T.se_nradR.assign(static_cast<size_t>(T.nse) * NS * 3, 0.0);
    sphere_edge_tables();
    T.sv_nc.assign(T.nsv, 0);
    T.sv_col.assign(4 * T.nsv, -1);
    T.sv_le.assign(4 * T.nsv, 0);
    T.sv_fL.assign(4 * T.nsv, 0);
    T.sv_fR.assign(4 * T.nsv, 0);
    T.sv_fse.assign(4 * T.nsv, 0);
    T.sv_fn.assign(static_cast<size_t>(T.nsv) * 4 * NS * 3, 0.0);
    T.sv_dlw.assign(static_cast<size_t>(T.nsv) * NS, 0.0);
    sphere_vertex_tables();
    return "";
  }
};

// ---------------------------------------------------------------------------
// the paper's reference triangular prism (Sec. V.c)
// ---------------------------------------------------------------------------
// monomials xi^a eta^b zeta^c of the order-p prism space (Eqs. 5.12-5.14)
static const int PRISM_EXP2[6][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {0, 1, 1}};
static const int PRISM_EXP3[15][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2},
                                      {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}, {2, 0, 1}, {0, 2, 1}, {1, 0, 2},
                                      {0, 1, 2}};
static const int PRISM_EXP4[26][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2},
                                      {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {3, 0, 0}, {0, 3, 0}, {0, 0, 3}, {2, 1, 0},
                                      {2, 0, 1}, {1, 2, 0}, {0, 2, 1}, {1, 0, 2}, {0, 1, 2}, {1, 1, 1}, {1, 0, 3},
                                      {0, 1, 3}, {3, 0, 1}, {0, 3, 1}, {2, 1, 1}, {1, 2, 1}};

static double ipow(double x, int e) {
  double r = 1.0;
  for (int k = 0; k < e; ++k) r *= x;
  return r;
}

bool prism_element(int p, vector<double>& nodes, vector<double>& D) {
  if (p < 2 || p > 4) return false;
  const int N = p == 2 ? 6 : (p == 3 ? 15 : 26);
  const int(*ex)[3] = p == 2 ? PRISM_EXP2 : (p == 3 ? PRISM_EXP3 : PRISM_EXP4);
  const double s3 = std::sqrt(3.0);
  const double tri[3][2] = {{-0.5, -0.5 / s3}, {0.5, -0.5 / s3}, {0.0, 1.0 / s3}};
  nodes.clear();
  for (double z : {0.5, -0.5})
    for (int v = 0; v < 3; ++v) nodes.insert(nodes.end(), {tri[v][0], tri[v][1], z});
  // edges: the three sides of the top face, of the bottom face, then the three
  // edges along zeta; p-2 equidistant interior nodes each
  for (int e = 0; e < 9; ++e)
    for (int k = 1; k <= p - 2; ++k) {
      const double t = static_cast<double>(k) / (p - 1);
      if (e < 6) {
        const int a = e % 3, b = (e + 1) % 3;
        const double z = e < 3 ? 0.5 : -0.5;
        nodes.insert(nodes.end(), {(1 - t) * tri[a][0] + t * tri[b][0], (1 - t) * tri[a][1] + t * tri[b][1], z});
      } else {
        nodes.insert(nodes.end(), {tri[e - 6][0], tri[e - 6][1], 0.5 - t});
      }
    }
  if (p == 4) nodes.insert(nodes.end(), {0.0, 0.0, 0.5, 0.0, 0.0, -0.5});
  if (static_cast<int>(nodes.size()) != 3 * N) return false;
  // Lagrange basis (Eq. 5.3): C = V^-1 with V_im = monomial m at node i
  vector<double> V(static_cast<size_t>(N) * N);
  for (int i = 0; i < N; ++i)
    for (int m = 0; m < N; ++m)
      V[i * N + m] = ipow(nodes[3 * i], ex[m][0]) * ipow(nodes[3 * i + 1], ex[m][1]) * ipow(nodes[3 * i + 2], ex[m][2]);
  if (!invert_inplace(V, N)) return false;
  D.assign(static_cast<size_t>(3) * N * N, 0.0);
  for (int ax = 0; ax < 3; ++ax)
    for (int i = 0; i < N; ++i)
      for (int m = 0; m < N; ++m) {
        const int e = ex[m][ax];
        if (e == 0) continue;
        int f[3] = {ex[m][0], ex[m][1], ex[m][2]};
        f[ax] -= 1;
        const double dm =
            e * ipow(nodes[3 * i], f[0]) * ipow(nodes[3 * i + 1], f[1]) * ipow(nodes[3 * i + 2], f[2]);
        for (int j = 0; j < N; ++j) D[(static_cast<size_t>(ax) * N + i) * N + j] += dm * V[m * N + j];
      }
  // entries that vanish exactly (basis functions constant along a direction at a
  // node) come out of the inverse at rounding level; set them to zero so that the
  // predictor skips them (580 of 2028 entries are nonzero at p = 4)
  double dmax = 0.0;
  for (double x : D) dmax = std::fmax(dmax, std::fabs(x));
  for (double& x : D)
    if (std::fabs(x) <= 1e-12 * dmax) x = 0.0;
  return true;
}

// Time tables of the ADER-CG predictor (Eqs. 5.15-5.17, 5.24-5.29): tau_1 = 0
// and the M-1 Gauss points in [0, 1]; wt = their Gauss weights; R = (K11)^-1 M1
// ([M][M], row 1 zero), with K11_bm = int phi_b phi_m' and M1_bm = int phi_b phi_m.
void time_tables(int M, vector<double>& wt, vector<double>& R) {
  vector<double> xg, wg;
  gauss_legendre(M - 1, xg, wg);
  vector<double> tau(M);
  tau[0] = 0.0;
  for (int m = 1; m < M; ++m) tau[m] = 0.5 + xg[m - 1];
  wt = wg;
  auto phi = [&](int m, double t) {
    double v = 1.0;
    for (int l = 0; l < M; ++l)
      if (l != m) v *= (t - tau[l]) / (tau[m] - tau[l]);
    return v;
  };
  auto dphi = [&](int m, double t) {
    double s = 0.0;
    for (int l = 0; l < M; ++l) {
      if (l == m) continue;
      double v = 1.0 / (tau[m] - tau[l]);
      for (int j = 0; j < M; ++j)
        if (j != m && j != l) v *= (t - tau[j]) / (tau[m] - tau[j]);
      s += v;
    }
    return s;
  };
  vector<double> xq, wq;
  gauss_legendre(M + 1, xq, wq);
  int nb = M - 1;
  vector<double> K11(static_cast<size_t>(nb) * nb, 0.0), Mm(static_cast<size_t>(nb) * M, 0.0);
  for (size_t g = 0; g < xq.size(); ++g) {
    double t = 0.5 + xq[g];
    for (int b = 1; b < M; ++b) {
      for (int m = 1; m < M; ++m) K11[(b - 1) * nb + (m - 1)] += wq[g] * phi(b, t) * dphi(m, t);
      for (int m = 0; m < M; ++m) Mm[(b - 1) * M + m] += wq[g] * phi(b, t) * phi(m, t);
    }
  }
  invert_inplace(K11, nb);
  R.assign(static_cast<size_t>(M) * M, 0.0);
  for (int b = 0; b < nb; ++b)
    for (int m = 0; m < M; ++m) {
      double s = 0.0;
      for (int j = 0; j < nb; ++j) s += K11[b * nb + j] * Mm[j * M + m];
      R[(b + 1) * M + m] = s;
    }
}

std::string build_tables(int n, int nr, double r_in, double r_out, int p, Tables& T) {
  if (p < 2 || p > 4) return "order must be 2, 3 or 4";
  if (n < 2) return "subdiv must be >= 2";
  if (nr < 2 || (p == 4 && nr < 3)) return "nr too small for this order";
  if (!(r_in > 0.0) || !(r_out > r_in)) return "need 0 < r_in < r_out";
  Builder b(n, nr, r_in, r_out, p, T);
  return b.build();
}

// ---------------------------------------------------------------------------
// geometry services for initial data
// ---------------------------------------------------------------------------
void zone_cubature(const Tables& T, int nq, double* pts, double* w) {
  Tables tmp;  // the builder only needs the topology-free map here
  Builder b(T.n, T.nr, T.r_in, T.r_out, T.d.P, tmp);
  vector<double> x, wx;
  gauss_legendre(nq, x, wx);
  int G = nq * nq * nq;
  vector<V3> ref;
  vector<double> rw;
  for (int a = 0; a < nq; ++a)
    for (int bb = 0; bb < nq; ++bb)
      for (int c = 0; c < nq; ++c) {
        ref.push_back({x[a], x[bb], x[c]});
        rw.push_back(wx[a] * wx[bb] * wx[c]);
      }
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t z = 0; z < T.Z; ++z) {
    int c = static_cast<int>(z / T.nr), k = static_cast<int>(z % T.nr);
    vector<V3> X = b.zone_nodes(c, k);
    for (int g = 0; g < G; ++g) {
      V3 xx = b.map_point(X, ref[g]);
      auto h = b.map_jac(X, ref[g]);
      double J = dot(cross(h[0], h[1]), h[2]);
      for (int a = 0; a < 3; ++a) pts[(z * G + g) * 3 + a] = xx[a];
      w[z * G + g] = J * rw[g];
    }
  }
}

void edge_quadrature(const Tables& T, int nq, double* pts, double* tw) {
  Tables tmp;
  Builder b(T.n, T.nr, T.r_in, T.r_out, T.d.P, tmp);
  vector<double> x, wx;
  gauss_legendre(nq, x, wx);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t e = 0; e < T.E; ++e) {
    int c, k, le;
    bool rev;
    if (e < T.E_rad) {
      int sv = static_cast<int>(e / T.nr);
      k = static_cast<int>(e % T.nr);
      c = T.sv_col[4 * sv];
      le = T.sv_le[4 * sv];
      rev = false;
    } else {
      int64_t r = e - T.E_rad;
      int se = static_cast<int>(r / (T.nr + 1));
      int kk = static_cast<int>(r % (T.nr + 1));
      c = T.se_col[2 * se];
      rev = T.se_rev[2 * se] != 0;
      if (kk < T.nr) { k = kk; le = T.se_le[(2 * se) * 2 + 0]; }
      else { k = kk - 1; le = T.se_le[(2 * se) * 2 + 1]; }
    }
    vector<V3> X = b.zone_nodes(c, k);
    int ax = EDGE_AXIS[le];
    for (int s = 0; s < nq; ++s) {
      int sl = rev ? nq - 1 - s : s;
      V3 xi = edge_point(le, x[sl]);
      V3 xx = b.map_point(X, xi);
      auto h = b.map_jac(X, xi);
      double sg = rev ? -1.0 : 1.0;
      for (int a = 0; a < 3; ++a) {
        pts[(e * nq + s) * 3 + a] = xx[a];
        tw[(e * nq + s) * 3 + a] = sg * h[ax][a] * wx[sl];
      }
    }
  }
}

void phi_from_circulation(const Tables& T, const double* circ, double* phi) {
  const int nr = T.nr;
  for (int c = 0; c < T.ncol; ++c)
    for (int k = 0; k <= nr; ++k) {
      double s = 0.0;
      for (int q = 0; q < 4; ++q) {
        int se = T.col_side_se[4 * c + q];
        s += T.col_side_sgn[4 * c + q] * circ[T.E_rad + static_cast<int64_t>(se) * (nr + 1) + k];
      }
      phi[static_cast<int64_t>(c) * (nr + 1) + k] = s;
    }
  for (int se = 0; se < T.nse; ++se) {
    int va = T.se_v[2 * se], vb = T.se_v[2 * se + 1];
    for (int k = 0; k < nr; ++k) {
      int64_t base = T.E_rad + static_cast<int64_t>(se) * (nr + 1);
      phi[T.F_rad + static_cast<int64_t>(se) * nr + k] =
          circ[base + k] + circ[static_cast<int64_t>(vb) * nr + k] - circ[base + k + 1] -
          circ[static_cast<int64_t>(va) * nr + k];
    }
  }
}

void zone_centroids(const Tables& T, double* xc, double* vol) {
  for (int c = 0; c < T.ncol; ++c)
    for (int k = 0; k < T.nr; ++k) {
      double s = std::pow(T.q, k);
      int64_t z = static_cast<int64_t>(c) * T.nr + k;
      for (int a = 0; a < 3; ++a) xc[3 * z + a] = T.xc0[3 * c + a] * s;
      vol[z] = T.V0[c] * s * s * s;
    }
}

void radial_face_quadrature(const Tables& T, int nq, double* pts, double* wn) {
  Tables tmp;
  Builder b(T.n, T.nr, T.r_in, T.r_out, T.d.P, tmp);
  vector<double> x, wx;
  gauss_legendre(nq, x, wx);
  const int G = nq * nq;
#pragma omp parallel for schedule(dynamic, 16)
  for (int c = 0; c < T.ncol; ++c)
    for (int k = 0; k <= T.nr; ++k) {
      // the inner face (zeta = -1/2) of shell k; the outer face of the last shell
      const int kz = k < T.nr ? k : T.nr - 1;
      const double zeta = k < T.nr ? -0.5 : 0.5;
      vector<V3> X = b.zone_nodes(c, kz);
      const int64_t f = static_cast<int64_t>(c) * (T.nr + 1) + k;
      for (int a = 0; a < nq; ++a)
        for (int bb = 0; bb < nq; ++bb) {
          const V3 xi{x[a], x[bb], zeta};
          const V3 xx = b.map_point(X, xi);
          const auto h = b.map_jac(X, xi);
          const V3 n = cross(h[0], h[1]);  // (h_xi x h_eta): along +r on these faces
          const int64_t g = f * G + a * nq + bb;
          for (int d = 0; d < 3; ++d) {
            pts[g * 3 + d] = xx[d];
            wn[g * 3 + d] = n[d] * wx[a] * wx[bb];
          }
        }
    }
}

void face_geometry(const Tables& T, double* area, double* nrm) {
  const int NQT = T.d.NQT;
  auto fill = [&](int64_t f, int c, int lf, int k, double sign) {
    const double s2 = std::pow(T.q, 2 * k);
    double n[3] = {0.0, 0.0, 0.0};
    for (int q = T.foff[lf]; q < T.foff[lf + 1]; ++q) {
      const size_t idx = static_cast<size_t>(c) * NQT + q;
      for (int a = 0; a < 3; ++a) n[a] += T.WF[idx] * T.nF[3 * idx + a];
    }
    area[f] = T.A0[6 * c + lf] * s2;
    for (int a = 0; a < 3; ++a) nrm[3 * f + a] = sign * n[a] * s2;
  };
  // radial faces: the inner face (local face 4) of shell k, canonical normal +r
  for (int c = 0; c < T.ncol; ++c)
    for (int k = 0; k <= T.nr; ++k) fill(static_cast<int64_t>(c) * (T.nr + 1) + k, c, 4, k, -1.0);
  // angular faces: outward normal of the L column's local face
  for (int se = 0; se < T.nse; ++se)
    for (int k = 0; k < T.nr; ++k)
      fill(T.F_rad + static_cast<int64_t>(se) * T.nr + k, T.se_col[2 * se], T.se_lf[2 * se], k, 1.0);
}

}  // namespace geo
