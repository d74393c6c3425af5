"""The paper's reference triangular prism and its isoparametric frustum zones
(Sec. II.b, Sec. V.c, Eqs. 5.12-5.14, Fig. 7, App. B-D) -- oracle (test
infrastructure only).

Reference element: the equilateral triangular prism with unit edges and its
centroid at the origin; triangle vertices (-1/2, -1/(2 sqrt3)), (1/2, -1/(2 sqrt3)),
(0, 1/sqrt3), zeta in [-1/2, 1/2].  Serendipity nodes (Fig. 7): the 6 vertices,
p-2 equidistant nodes inside each of the 9 edges, and at p = 4 the centroids of
the two triangular faces (6 / 15 / 26 nodes).  The Lagrange basis on the
monomials of Eqs. 5.12-5.14 comes from the generic generator of refelem.py
(Eq. 5.3), and D^alpha_ij = d psi_j / d xi_alpha at node i.

Frustum zone: the isoparametric map x(xi) = sum_i psi_i(xi) x_i with nodes x_i
on the spherical frustum between radii r0 and r1 over the spherical triangle
(a, b, c): radius linear in zeta, lateral position by the node rule of
geodesic.py (vertices, arc-equidistant edge points, normalised centroid).  The
zone object offers what oracle/ader.py's predictor reads (el, p, map_jacobian),
so the paper's ADER-CG predictor runs unchanged on the paper's own element.

Pinned by tests/test_oracle_prism.py: the node sets equal the printed ones
(Eqs. B/C.2-C.16 and D.2-D.27), the frustum map's volume equals the one of
geodesic.py computed through a different factorisation (triangle basis times
linear radius), and the predictor on the prism reproduces advected polynomials
of degree <= p-1 exactly on an affine zone and preserves a uniform state on a
curved frustum.
"""
import numpy as np

from . import refelem
from .geodesic import _slerp, triangle_rule

S3 = np.sqrt(3.0)
TRI = np.array([[-0.5, -0.5 / S3], [0.5, -0.5 / S3], [0.0, 1.0 / S3]])   # reference triangle vertices
# the 9 edges: three in each triangular face, three along zeta
EDGES = [((0, 1), 0.5), ((1, 2), 0.5), ((2, 0), 0.5), ((0, 1), -0.5), ((1, 2), -0.5), ((2, 0), -0.5),
         (0, None), (1, None), (2, None)]


def prism_nodes(p):
    """Serendipity nodes of the order-p reference prism (Fig. 7): vertices
    (top face zeta = +1/2 first), p-2 equidistant nodes inside each edge, and for
    p = 4 the triangle-face centroids.  The order of the list is this module's;
    the paper's numbering differs."""
    out = [(x, y, 0.5) for x, y in TRI] + [(x, y, -0.5) for x, y in TRI]
    t = np.linspace(0.0, 1.0, p)[1:-1]
    for e, z in EDGES:
        for s in t:
            if z is None:          # along zeta at vertex e
                out.append((TRI[e][0], TRI[e][1], 0.5 - s))
            else:
                i, j = e
                q = (1.0 - s) * TRI[i] + s * TRI[j]
                out.append((q[0], q[1], z))
    if p == 4:
        out += [(0.0, 0.0, 0.5), (0.0, 0.0, -0.5)]
    return np.array(out)


class PrismElement:
    def __init__(self, p):
        self.p = p
        self.nodes = prism_nodes(p)
        self.exps = refelem.prism_exponents(p)
        self.N = len(self.nodes)
        assert self.N == len(self.exps)
        self.C = refelem.lagrange_coefficients(self.nodes, self.exps)
        self.D = np.stack([self.dbasis(self.nodes, a) for a in range(3)])

    def basis(self, pts):
        return refelem.monomials(pts, self.exps) @ self.C

    def dbasis(self, pts, axis):
        return refelem.monomial_derivative(pts, self.exps, axis) @ self.C


def barycentric(pts):
    """Barycentric coordinates (l1, l2, l3) of reference-triangle points (n, 2)."""
    T = np.array([TRI[1] - TRI[0], TRI[2] - TRI[0]]).T
    l23 = np.linalg.solve(T, (np.asarray(pts)[:, :2] - TRI[0]).T).T
    return np.column_stack([1.0 - l23.sum(1), l23])


def sphere_point(a, b, c, lam):
    """Unit-sphere position of barycentric lam over the spherical triangle (a, b, c):
    a vertex, an arc-equidistant point of an edge, or the normalised combination."""
    V = (a, b, c)
    on = [k for k in range(3) if lam[k] > 1e-12]
    if len(on) == 1:
        return V[on[0]]
    if len(on) == 2:
        i, j = on
        return _slerp(V[i], V[j], lam[j] / (lam[i] + lam[j]))
    q = lam[0] * a + lam[1] * b + lam[2] * c
    return q / np.linalg.norm(q)


class FrustumZone:
    """The order-p prism mapped onto the frustum r in [r0, r1] over (a, b, c); or,
    with `X` given, onto arbitrary node positions (an affine zone)."""

    def __init__(self, p, a=None, b=None, c=None, r0=None, r1=None, X=None):
        self.p = p
        self.el = PrismElement(p)
        if X is None:
            lam = barycentric(self.el.nodes)
            X = np.array([(r0 + (r1 - r0) * (z + 0.5)) * sphere_point(a, b, c, l)
                          for l, z in zip(lam, self.el.nodes[:, 2])])
        self.X = X[None]

    def map_jacobian(self, X, pts):
        """dx/dxi_alpha at pts: (zones, points, alpha, 3)."""
        return np.stack([np.einsum("nj,zjd->znd", self.el.dbasis(pts, a), X) for a in range(3)], axis=2)

    def volume(self, nq=6):
        """Integral of det(dx/dxi) over the reference prism: a rule on the unit
        right triangle mapped affinely onto the reference triangle (area sqrt3/4)
        times Gauss-Legendre in zeta."""
        tp, tw = triangle_rule(nq)
        xy = TRI[0] + tp[:, :1] * (TRI[1] - TRI[0]) + tp[:, 1:2] * (TRI[2] - TRI[0])
        g, w = np.polynomial.legendre.leggauss(nq)
        vol = 0.0
        for zq, wz in zip(0.5 * g, 0.5 * w):
            pts = np.column_stack([xy, np.full(len(xy), zq)])
            h = self.map_jacobian(self.X, pts)[0]
            det = np.einsum("nd,nd->n", np.cross(h[:, 0], h[:, 1]), h[:, 2])
            vol += wz * (tw * np.abs(det)).sum() * (S3 / 2.0)
        return vol
