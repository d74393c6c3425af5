"""Pins of the icosahedral geodesic mesh and its isoparametric frustums
(oracle/geodesic.py) against what the paper prints (Sec. II.a-II.b) and what
geometry fixes."""
import numpy as np
import pytest

from oracle import geodesic as G


def test_level_counts_euler_and_valences():
    for L in range(4):
        v, t = G.geodesic_sphere(L)
        e = G.edges_of(t)
        assert (len(v), len(e), len(t)) == (10 * 4 ** L + 2, 30 * 4 ** L, 20 * 4 ** L)
        assert len(v) - len(e) + len(t) == 2
        val = np.bincount(e.ravel(), minlength=len(v))
        assert (val == 5).sum() == 12 and ((val == 5) | (val == 6)).all()
        assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)


def test_central_angles_match_the_printed_values():
    """Level 0: (pi/2) - atan(1/2) = 63.4 degrees for every edge; level 1: 33.9
    degrees and level 4: 4.33 degrees on average (Sec. II.a); each level about
    halves the angle (the finest accuracy mesh, 0.54 degrees, is level 7)."""
    printed = {0: (63.4, 0.05), 1: (33.9, 0.05), 4: (4.33, 0.005)}
    for L, (deg, tol) in printed.items():
        v, t = G.geodesic_sphere(L)
        a = np.degrees(G.central_angles(v, G.edges_of(t)))
        assert abs(a.mean() - deg) < tol, (L, a.mean())
    v, t = G.geodesic_sphere(0)
    a = G.central_angles(v, G.edges_of(t))
    assert np.allclose(a, np.pi / 2 - np.arctan(0.5), atol=1e-14)


def test_triangles_tile_the_sphere():
    """Consistent outward orientation, and the spherical excesses sum to 4 pi."""
    for L in range(4):
        v, t = G.geodesic_sphere(L)
        a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
        n = np.cross(b - a, c - a)
        assert (np.einsum("ij,ij->i", n, a + b + c) > 0).all()
        assert abs(G.spherical_area(a, b, c).sum() - 4 * np.pi) < 1e-12
        # every edge is shared by exactly two triangles, traversed in opposite directions
        half = {}
        for x, y, z in t:
            for p, q in ((x, y), (y, z), (z, x)):
                assert (p, q) not in half
                half[(p, q)] = 1
        assert all((q, p) in half for (p, q) in half)


def _polar_triangle(deg):
    th = np.radians(deg)
    return [np.array([np.sin(th) * np.cos(2 * np.pi * k / 3), np.sin(th) * np.sin(2 * np.pi * k / 3), np.cos(th)])
            for k in range(3)]


def test_mapping_of_the_polar_triangle():
    """Sec. II.b, Fig. 4: a spherical equilateral triangle at the pole with its
    vertices 5 degrees from the centroid; the quadratic and cubic mappings keep the
    radius to about one part in 1e6 and 1e7.  Halving the triangle shrinks the
    deviation at least at the mapping's order p (h^2 linear, h^4 cubic; the
    quadratic interpolant of the sphere gains one order, h^4, by symmetry)."""
    tri = _polar_triangle(5.0)
    d = {p: G.radial_deviation(*tri, p) for p in (2, 3, 4)}
    assert 1e-6 <= d[3] < 1e-5
    assert 1e-7 <= d[4] < 1e-6
    assert d[2] > 1e-3
    half = _polar_triangle(2.5)
    for p in (2, 3, 4):
        rate = np.log2(d[p] / G.radial_deviation(*half, p))
        assert rate > p - 0.1 and rate < 4.1, (p, rate)


def test_mapped_nodes_lie_on_the_sphere_and_reproduce_the_vertices():
    tri = _polar_triangle(5.0)
    for p in (2, 3, 4):
        s = G.mapping_nodes(*tri, p)
        assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-15)
        S, _, _ = G.lateral_map(*tri, p, np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]))
        assert np.allclose(S, np.array(tri), atol=1e-15)


def test_triangle_rule_is_exact():
    pts, w = G.triangle_rule(4)
    for i in range(6):
        for j in range(6 - i):
            # int_T x^i y^j = i! j! / (i + j + 2)!
            from math import factorial
            exact = factorial(i) * factorial(j) / factorial(i + j + 2)
            assert abs((w * pts[:, 0] ** i * pts[:, 1] ** j).sum() - exact) < 1e-15


@pytest.mark.parametrize("p", [2, 3, 4])
def test_frustum_volumes_converge_to_the_shell(p):
    """The mapped frustums of levels 1-3 (one shell, r in [1, 2]) sum to the shell
    volume 4 pi (r_out^3 - r_in^3) / 3 with an error that falls at least at the
    mapping's order p (the quadratic mapping's volume error falls at order 4)."""
    exact = 4.0 / 3.0 * np.pi * (2.0 ** 3 - 1.0)
    err = [abs(G.mesh_volume(L, 1.0, 2.0, 1, p) - exact) / exact for L in (1, 2, 3)]
    rates = [np.log2(err[i] / err[i + 1]) for i in range(2)]
    assert min(rates) > p - 0.3, (p, err, rates)


def test_flat_frustum_volume_closed_form():
    """With the linear mapping the frustum is the region between two similar flat
    triangles at radii r0 and r1 along rays through the origin: its volume is the
    cone-volume difference (r1^3 - r0^3) / 3 * (a . (b x c)) / 2 (the tetrahedron
    with apex at the origin, scaled)."""
    a, b, c = _polar_triangle(20.0)
    vol = G.frustum_volume(a, b, c, 1.5, 2.5, 2)
    exact = (2.5 ** 3 - 1.5 ** 3) * abs(a @ np.cross(b, c)) / 6.0
    assert abs(vol - exact) < 1e-14 * exact
