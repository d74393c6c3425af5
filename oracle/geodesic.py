"""Spherical icosahedral geodesic mesh (Sec. II.a, Figs. 1-2) and its isoparametric
frustum zones (Sec. II.b, Figs. 3-4) -- oracle (test infrastructure only).

The paper meshes the sphere by projecting an icosahedron onto it (level 0: 20
great triangles) and bisecting every spherical triangle's edges along great
circles (level L: 20 * 4^L triangles); the surface mesh is then extruded in the
radial direction with logarithmically ratioed shells, giving triangular-prism
frustum zones.  Zones are mapped isoparametrically from a reference triangular
prism: polynomial of degree p-1 across the triangle (nodes at the vertices, at
equidistant points of the edges -- equidistant along the great-circle arc -- and,
for p = 4, at the centroid of the triangle), linear in the radial direction.

Here the reference triangle is parametrised by two barycentric coordinates
(x, y) on the unit right triangle and the radial coordinate by zeta in [0, 1];
the paper's equilateral reference prism with unit edges differs from this by an
affine map, which changes no physical quantity computed below.

This module holds the mesh and its geometry only.  The build's scheme runs on
the cubed-sphere mesh (oracle/mesh.py); the stage kernels of the scheme on the
prism zones are not built.

Pinned by tests/test_oracle_geodesic.py: the mean central angle of an edge at
levels 0, 1 and 4 against the values the paper prints (63.4, 33.9 and 4.33
degrees), the vertex / edge / triangle counts with Euler's formula and the twelve
five-valent vertices, the spherical excess of all triangles summing to 4 pi, the
largest radial deviation of the quadratic and cubic mappings of the paper's
5-degree polar triangle against the paper's "one part in 1e6 / 1e7", and the
total volume of the mapped frustums converging to the shell volume at the
mapping's order.
"""
import itertools

import numpy as np


# ----------------------------------------------------------------------------
# surface mesh (Sec. II.a)
# ----------------------------------------------------------------------------

def icosahedron():
    """12 unit vertices and the 20 triangles, each oriented counter-clockwise
    seen from outside.  The triangles are the vertex triples that are mutually
    nearest neighbours (edge = the smallest vertex distance)."""
    g = (1.0 + 5.0 ** 0.5) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v += [(0.0, s1, s2 * g), (s1, s2 * g, 0.0), (s2 * g, 0.0, s1)]
    v = np.array(v)
    v /= np.linalg.norm(v, axis=1)[:, None]
    d = np.linalg.norm(v[:, None] - v[None], axis=2)
    edge = d[d > 1e-12].min()
    tris = []
    for t in itertools.combinations(range(12), 3):
        if all(abs(d[a, b] - edge) < 1e-9 for a, b in itertools.combinations(t, 2)):
            tris.append(_outward(v, t))
    return v, np.array(tris)


def _outward(v, t):
    a, b, c = t
    n = np.cross(v[b] - v[a], v[c] - v[a])
    return (a, b, c) if n @ (v[a] + v[b] + v[c]) > 0 else (a, c, b)


def subdivide(v, tris):
    """One level of bisection: the midpoint of every edge is pushed onto the
    sphere (the great-circle midpoint) and each triangle splits into four."""
    verts = list(v)
    mid = {}

    def m(a, b):
        k = (min(a, b), max(a, b))
        if k not in mid:
            x = verts[a] + verts[b]
            verts.append(x / np.linalg.norm(x))
            mid[k] = len(verts) - 1
        return mid[k]

    out = []
    for a, b, c in tris:
        ab, bc, ca = m(a, b), m(b, c), m(c, a)
        out += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
    return np.array(verts), np.array(out)


def geodesic_sphere(level):
    """Unit vertices (V, 3) and triangles (20 4^level, 3) of the level-`level` mesh."""
    v, t = icosahedron()
    for _ in range(level):
        v, t = subdivide(v, t)
    return v, t


def edges_of(tris):
    """Sorted unique vertex pairs of the triangles' sides."""
    e = set()
    for a, b, c in tris:
        for x, y in ((a, b), (b, c), (c, a)):
            e.add((min(x, y), max(x, y)))
    return np.array(sorted(e))


def central_angles(v, edges):
    """Angle at the sphere's centre subtended by each edge (radians)."""
    c = np.clip((v[edges[:, 0]] * v[edges[:, 1]]).sum(1), -1.0, 1.0)
    return np.arccos(c)


def spherical_area(a, b, c):
    """Area of the spherical triangle with unit vertices a, b, c (rows): its
    spherical excess, tan(E/2) = |a.(b x c)| / (1 + a.b + b.c + c.a)
    (Van Oosterom & Strackee 1983)."""
    num = np.abs(np.einsum("ij,ij->i", a, np.cross(b, c)))
    den = 1.0 + np.einsum("ij,ij->i", a, b) + np.einsum("ij,ij->i", b, c) + np.einsum("ij,ij->i", c, a)
    return 2.0 * np.arctan2(num, den)


def shell_radii(r_in, r_out, nr):
    """Logarithmically ratioed shell boundaries r_k = r_in (r_out / r_in)^(k / nr)."""
    return r_in * (r_out / r_in) ** (np.arange(nr + 1) / nr)


# ----------------------------------------------------------------------------
# isoparametric frustums (Sec. II.b)
# ----------------------------------------------------------------------------

def triangle_lattice(k):
    """Barycentric nodes (x, y) of the degree-k Lagrange triangle, ordered by
    (i, j) with x = i/k, y = j/k."""
    return np.array([(i / k, j / k) for i in range(k + 1) for j in range(k + 1 - i)])


def _slerp(a, b, t):
    w = np.arccos(np.clip(a @ b, -1.0, 1.0))
    return (np.sin((1.0 - t) * w) * a + np.sin(t * w) * b) / np.sin(w)


def mapping_nodes(a, b, c, p):
    """Unit-sphere nodes of the degree p-1 lateral mapping of the spherical
    triangle (a, b, c) at the lattice of triangle_lattice(p-1): vertices, points
    equidistant along the great-circle arcs of the edges, and the normalised
    centroid for the interior node of p = 4."""
    k = p - 1
    out = []
    for x, y in triangle_lattice(k):
        z = 1.0 - x - y
        on_edge = min(x, y, z) < 1e-12
        if max(x, y, z) > 1.0 - 1e-12:
            q = a * z + b * x + c * y
        elif on_edge:
            if z < 1e-12:
                q = _slerp(b, c, y / (x + y))
            elif x < 1e-12:
                q = _slerp(a, c, y / (y + z))
            else:
                q = _slerp(a, b, x / (x + z))
        else:
            q = a * z + b * x + c * y
            q = q / np.linalg.norm(q)
        out.append(q)
    return np.array(out)


def _tri_exponents(k):
    return [(i, j) for i in range(k + 1) for j in range(k + 1 - i)]


def triangle_basis(k, pts):
    """Values and (x, y) derivatives of the degree-k Lagrange basis on the
    lattice nodes at points pts (n, 2): three arrays (n, nodes)."""
    ex = _tri_exponents(k)
    nodes = triangle_lattice(k)
    V = np.array([[x ** i * y ** j for i, j in ex] for x, y in nodes])
    C = np.linalg.inv(V)
    x, y = pts[:, 0:1], pts[:, 1:2]
    P = np.concatenate([x ** i * y ** j for i, j in ex], axis=1)
    Px = np.concatenate([(i * x ** max(i - 1, 0)) * y ** j for i, j in ex], axis=1)
    Py = np.concatenate([x ** i * (j * y ** max(j - 1, 0)) for i, j in ex], axis=1)
    return P @ C, Px @ C, Py @ C


def lateral_map(a, b, c, p, pts):
    """S(x, y) = sum_i psi_i(x, y) s_i, the mapped unit-sphere surface, and its
    two tangent vectors, at points pts (n, 2)."""
    s = mapping_nodes(a, b, c, p)
    L, Lx, Ly = triangle_basis(p - 1, pts)
    return L @ s, Lx @ s, Ly @ s


def triangle_rule(n):
    """A quadrature rule on the unit right triangle exact for polynomials of
    degree 2n - 2 in each variable: the Duffy collapse of an n x n Gauss-Legendre
    tensor rule (x = u, y = (1 - u) w, Jacobian 1 - u)."""
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    pts, wts = [], []
    for ui, wu in zip(g, w):
        for vi, wv in zip(g, w):
            pts.append((ui, (1.0 - ui) * vi))
            wts.append(wu * wv * (1.0 - ui))
    return np.array(pts), np.array(wts)


def frustum_volume(a, b, c, r0, r1, p, nq=6):
    """Volume of the mapped frustum x(x, y, zeta) = r(zeta) S(x, y),
    r(zeta) = r0 + (r1 - r0) zeta: the integral of det[dx/dx, dx/dy, dx/dzeta]
    over the reference prism by a triangle rule times Gauss-Legendre in zeta."""
    pts, wts = triangle_rule(nq)
    S, Sx, Sy = lateral_map(a, b, c, p, pts)
    g, w = np.polynomial.legendre.leggauss(nq)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    vol = 0.0
    trip = np.einsum("ij,ij->i", np.cross(Sx, Sy), S)   # (S_x x S_y) . S
    for zq, wz in zip(g, w):
        r = r0 + (r1 - r0) * zq
        # det[r S_x, r S_y, (r1 - r0) S] = r^2 (r1 - r0) (S_x x S_y) . S
        vol += wz * (r * r * (r1 - r0)) * (wts * trip).sum()
    return abs(vol)


def radial_deviation(a, b, c, p, n=201):
    """Largest | |S(x, y)| - 1 | of the lateral mapping over a lattice of the
    reference triangle (the quantity of the paper's Fig. 4)."""
    s = np.linspace(0.0, 1.0, n)
    pts = np.array([(x, y) for x in s for y in s if x + y <= 1.0 + 1e-12])
    S, _, _ = lateral_map(a, b, c, p, pts)
    return np.abs(np.linalg.norm(S, axis=1) - 1.0).max()


def mesh_volume(level, r_in, r_out, nr, p):
    """Sum of the mapped frustum volumes of the extruded level-`level` mesh."""
    v, t = geodesic_sphere(level)
    r = shell_radii(r_in, r_out, nr)
    total = 0.0
    for tri in t:
        a, b, c = v[tri[0]], v[tri[1]], v[tri[2]]
        for k in range(nr):
            total += frustum_volume(a, b, c, r[k], r[k + 1], p)
    return total
