"""Reference-element bases of the ADER-CG predictor (Sec. V.b-V.c, App. B-D).

Spatial basis.  The paper's reference element is a triangular prism with
serendipity nodes (Eqs. 5.12-5.14, Fig. 7).  The build meshes the sphere with a
cubed sphere, so its reference element is the unit cube [-1/2,1/2]^3 with the
hexahedral serendipity spaces of the same orders: all monomials of superlinear
degree <= p-1 (8 / 20 / 32 functions for p = 2 / 3 / 4).  Nodes: the 8 vertices
plus p-2 equidistant nodes inside each of the 12 edges ("the edges are
bisected/trisected in equidistant fashion", Fig. 7).  The Lagrange basis
satisfies psi_j(x_i) = delta_ij (Eq. 5.3) and is found by inverting the
Vandermonde matrix (the "computer algebra" step of Sec. V.d, step 1).

Temporal basis.  M = p levels at tau_1 = 0 and the Gauss points (Eqs. 5.15-5.17),
Lagrange property Eq. 5.18.

R matrix.  With nodal collocation in space (App. C, Eq. C.34) the Galerkin
projection in time (Eqs. 5.24-5.29) reduces to
    U_k = U_1 + sum_m R_km (S_m - dF_m),  k = 2..M   (Eqs. C.35-C.36, D.30-D.32)
with R = (K_tau^11)^-1 M^1.  where K_tau_bm = int phi_b phi_m' and
M_bm = int phi_b phi_m over tau in [0,1], b = 2..M.  Row 1 of R is zero.

Local numbering of the hexahedron (used by both mesh and predictor):
  vertices  v = ix + 2*iy + 4*iz,  coordinate (ix-1/2, iy-1/2, iz-1/2)
  faces     0: xi=-1/2, 1: xi=+1/2, 2: eta=-1/2, 3: eta=+1/2, 4: zeta=-1/2, 5: zeta=+1/2
  edges     0-3 along xi   at (eta,zeta) = (-,-),(+,-),(-,+),(+,+)
            4-7 along eta  at (xi,zeta)  = (-,-),(+,-),(-,+),(+,+)
            8-11 along zeta at (xi,eta)  = (-,-),(+,-),(-,+),(+,+)

Pinned by: tests/test_oracle_refelem.py -- delta property, reproduction of every
monomial of the space, the printed R matrices (Eqs. B.9, C.18, D.28), the printed
prism bases (Eqs. B.10-B.15, C.19-C.33 via the same generator), the nodal
flux-difference row of Eq. B.16, and K_tau^0 = [1..1] (Eq. 5.29).
"""
import itertools

import numpy as np

from . import quadrature


# ----------------------------------------------------------------------------
# generic Lagrange basis from nodes and a monomial list (Eq. 5.3)
# ----------------------------------------------------------------------------

def monomials(points, exps):
    """points (n, d), exps (m, d) -> (n, m) matrix of monomial values."""
    points = np.asarray(points, dtype=np.float64)
    exps = np.asarray(exps, dtype=np.int64)
    out = np.ones((points.shape[0], exps.shape[0]))
    for d in range(points.shape[1]):
        out *= points[:, d:d + 1] ** exps[None, :, d]
    return out


def monomial_derivative(points, exps, axis):
    """d/dx_axis of each monomial at points -> (n, m)."""
    exps = np.asarray(exps, dtype=np.int64)
    lowered = exps.copy()
    fac = exps[:, axis].astype(np.float64)
    lowered[:, axis] = np.maximum(exps[:, axis] - 1, 0)
    return monomials(points, lowered) * fac[None, :]


def lagrange_coefficients(nodes, exps):
    """Coefficient matrix C (m, n): psi_j(x) = sum_m C[m, j] * x^exps[m]."""
    V = monomials(nodes, exps)
    return np.linalg.inv(V)


# ----------------------------------------------------------------------------
# hexahedral serendipity element
# ----------------------------------------------------------------------------

def hex_exponents(p):
    """Monomials of superlinear degree <= p-1 (serendipity space of the order-p scheme)."""
    r = p - 1
    out = []
    for total in range(0, 3 * r + 1):
        for a, b, c in itertools.product(range(r + 1), repeat=3):
            if a + b + c != total:
                continue
            sl = sum(e for e in (a, b, c) if e >= 2)
            if sl <= r:
                out.append((a, b, c))
    return np.array(out, dtype=np.int64)


VERTS = np.array([[ix - 0.5, iy - 0.5, iz - 0.5]
                  for iz in (0, 1) for iy in (0, 1) for ix in (0, 1)])

# edge e runs along EDGE_AXIS[e]; EDGE_FIXED[e] holds the two fixed coordinates
EDGE_AXIS = np.array([0, 0, 0, 0, 1, 1, 1, 1, 2, 2, 2, 2])
EDGE_FIXED = np.array([
    # along xi: (eta, zeta)
    [np.nan, -0.5, -0.5], [np.nan, 0.5, -0.5], [np.nan, -0.5, 0.5], [np.nan, 0.5, 0.5],
    # along eta: (xi, zeta)
    [-0.5, np.nan, -0.5], [0.5, np.nan, -0.5], [-0.5, np.nan, 0.5], [0.5, np.nan, 0.5],
    # along zeta: (xi, eta)
    [-0.5, -0.5, np.nan], [0.5, -0.5, np.nan], [-0.5, 0.5, np.nan], [0.5, 0.5, np.nan],
])

FACE_AXIS = np.array([0, 0, 1, 1, 2, 2])
FACE_SIDE = np.array([-0.5, 0.5, -0.5, 0.5, -0.5, 0.5])
# in-face parameter axes (u, v): side faces use (angular, radial)
FACE_PARAMS = {0: (1, 2), 1: (1, 2), 2: (0, 2), 3: (0, 2), 4: (0, 1), 5: (0, 1)}


def edge_points(e, t):
    """Reference coordinates of parameter values t (array) on local edge e."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    pts = np.tile(EDGE_FIXED[e], (t.size, 1))
    pts[:, EDGE_AXIS[e]] = t
    return pts


def face_points(f, uv):
    """Reference coordinates of in-face parameters uv (n, 2) on local face f."""
    uv = np.atleast_2d(uv)
    pts = np.zeros((uv.shape[0], 3))
    a, b = FACE_PARAMS[f]
    pts[:, a] = uv[:, 0]
    pts[:, b] = uv[:, 1]
    pts[:, FACE_AXIS[f]] = FACE_SIDE[f]
    return pts


def hex_nodes(p):
    """Serendipity nodes: 8 vertices, then p-2 equidistant nodes per edge (edge order)."""
    nodes = [v for v in VERTS]
    if p >= 3:
        ts = np.linspace(-0.5, 0.5, p)[1:-1]
        for e in range(12):
            nodes.extend(edge_points(e, ts))
    return np.array(nodes)


class HexElement:
    """Nodal serendipity element of order p on [-1/2,1/2]^3."""

    def __init__(self, p):
        self.p = p
        self.exps = hex_exponents(p)
        self.nodes = hex_nodes(p)
        self.N = self.nodes.shape[0]
        assert self.N == self.exps.shape[0]
        self.coef = lagrange_coefficients(self.nodes, self.exps)
        # D[axis][i, j] = d psi_j / d axis at node i   (the rows of Eq. C.34)
        self.D = np.stack([self.dbasis(self.nodes, a) for a in range(3)])

    def basis(self, pts):
        """psi_j at pts -> (n, N)."""
        return monomials(pts, self.exps) @ self.coef

    def dbasis(self, pts, axis):
        return monomial_derivative(pts, self.exps, axis) @ self.coef


# ----------------------------------------------------------------------------
# temporal basis and the R matrix
# ----------------------------------------------------------------------------

def time_nodes(p):
    return quadrature.time_gauss(p)[0]


def lagrange_1d(nodes):
    """Coefficients (in powers of tau) of the 1D Lagrange polynomials on nodes."""
    nodes = np.asarray(nodes, dtype=np.float64)
    V = np.vander(nodes, increasing=True)
    return np.linalg.inv(V)            # column j: coefficients of phi_j


def r_matrix(p):
    """R = (K_tau^11)^-1 M^1. (Eqs. 5.26-5.29 in time only); first row zero."""
    tau = time_nodes(p)
    M = len(tau)
    C = lagrange_1d(tau)
    xg, wg = quadrature.gauss_legendre(M + 1)
    tg = 0.5 + xg
    powers = np.vander(tg, M, increasing=True)                 # (ng, M)
    dpowers = np.zeros_like(powers)
    for k in range(1, M):
        dpowers[:, k] = k * tg ** (k - 1)
    phi = powers @ C                                            # (ng, M)
    dphi = dpowers @ C
    Kt = np.einsum("g,gb,gm->bm", wg, phi, dphi)
    Mm = np.einsum("g,gb,gm->bm", wg, phi, phi)
    R = np.zeros((M, M))
    R[1:, :] = np.linalg.solve(Kt[1:, 1:], Mm[1:, :])
    K0 = -np.linalg.solve(Kt[1:, 1:], Kt[1:, :1])
    return R, K0


# ----------------------------------------------------------------------------
# the paper's prism element (used only as a pin of the generic generator)
# ----------------------------------------------------------------------------

def prism_exponents(p):
    """Monomials of Eqs. 5.12 (p=2), 5.13 (p=3) and 5.14 (p=4)."""
    if p == 2:
        return np.array([(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1)])
    if p == 3:
        return np.array([(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0),
                         (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1), (2, 0, 1),
                         (0, 2, 1), (1, 0, 2), (0, 1, 2)])
    if p == 4:
        return np.array([(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0),
                         (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1), (3, 0, 0), (0, 3, 0),
                         (0, 0, 3), (2, 1, 0), (2, 0, 1), (1, 2, 0), (0, 2, 1), (1, 0, 2),
                         (0, 1, 2), (1, 1, 1), (1, 0, 3), (0, 1, 3), (3, 0, 1), (0, 3, 1),
                         (2, 1, 1), (1, 2, 1)])
    raise ValueError(p)
