"""Pins of the oracle's cubed-sphere mesh and isoparametric geometry (Sec. II, Eq. 5.2-5.5)."""
import numpy as np
import pytest

from oracle import mesh as M
from oracle import refelem


@pytest.fixture(scope="module", params=[2, 3, 4])
def small(request):
    p = request.param
    m = M.Mesh(3, 2, 1.0, 2.0, p)
    c = np.repeat(np.arange(m.ncol), m.nr)
    k = np.tile(np.arange(m.nr), m.ncol)
    return m, m.zone_geometry(c, k)


def test_topology_counts(small):
    m, _ = small
    n = m.n
    assert m.nsv == 6 * n * n + 2 and m.nse == 12 * n * n
    assert m.nsv - m.nse + m.ncol == 2                      # Euler characteristic of the sphere
    # every sphere vertex touches 3 (cube corners) or 4 columns
    counts = np.array([len(c) for c in m.sv_cols])
    assert set(counts) == {3, 4} and (counts == 3).sum() == 8
    assert m.F == 6 * n * n * (m.nr + 1) + 12 * n * n * m.nr


def test_face_closure_per_zone(small):
    """sum over the six faces of sum_q w_q n_q |dA_q| = 0 (exact face quadrature)."""
    m, g = small
    tot = np.zeros((m.Z, 3))
    for lf in range(6):
        fg = m.face_geometry(g["X"], lf)
        tot += np.einsum("q,zq,zqd->zd", fg["w"], fg["dA"], fg["n"])
    scale = g["V"] ** (2.0 / 3.0)
    assert (np.linalg.norm(tot, axis=1) / scale).max() < 1e-14


def test_discrete_div_of_curl_is_zero(small):
    m, _ = small
    a = np.random.default_rng(3).standard_normal(m.E)
    phi = (m.face_edge_sign * a[m.face_edges]).sum(1)
    div = (m.zone_face_sign * phi[m.zone_face]).sum(1)
    assert np.abs(div).max() < 1e-14 * np.abs(a).max() * 8


def test_shared_faces_coincide(small):
    """Both zones of an interior face map the same surface (conforming mesh)."""
    m, g = small
    fgeo = [m.face_geometry(g["X"], lf) for lf in range(6)]
    for f in range(m.F):
        zL, lfL = m.face_L[f]
        zR, lfR = m.face_R[f]
        if zL < 0 or zR < 0:
            continue
        xL, xR = fgeo[lfL]["x"][zL], fgeo[lfR]["x"][zR]
        d = np.linalg.norm(xL[:, None] - xR[None], axis=-1).min(1)
        assert d.max() < 1e-12
        # outward normals of the two sides are opposite at matching points
        j = np.linalg.norm(xL[:, None] - xR[None], axis=-1).argmin(1)
        assert np.abs(fgeo[lfL]["n"][zL] + fgeo[lfR]["n"][zR][j]).max() < 1e-12


def test_positive_jacobian_and_outward_normals(small):
    m, g = small
    assert (g["J"] > 0).all()
    for lf in range(6):
        fg = m.face_geometry(g["X"], lf)
        out = fg["x"] - g["xc"][:, None, :]
        assert ((out * fg["n"]).sum(-1) > 0).all()


@pytest.mark.parametrize("p,rate", [(2, 1.8), (3, 3.5), (4, 3.5)])
def test_volume_converges(p, rate):
    errs = []
    for n in (4, 8):
        m = M.Mesh(n, 1, 1.0, 2.0, p)
        g = m.zone_geometry(np.arange(m.ncol), np.zeros(m.ncol, int))
        errs.append(abs(g["V"].sum() / (4.0 / 3.0 * np.pi * 7.0) - 1.0))
    assert np.log2(errs[0] / errs[1]) > rate


def test_sphericity_improves_with_map_order():
    """Fig. 4 analogue: the radius deviation of the mapped outer surface shrinks with
    map order and with resolution at the interpolation rates h^2 (linear), h^3
    (quadratic), h^4 (cubic).  (The paper's 1e-6 / 1e-7 refer to its triangular
    element; on 5 degree quads the quadratic / cubic maps give ~2e-5 / ~4e-6.)"""
    rng = np.random.default_rng(0)
    pts = rng.uniform(-0.5, 0.5, (400, 3))
    pts[:, 2] = 0.5
    dev = {}
    for n in (18, 36):                                        # 5 and 2.5 degree columns
        for p in (2, 3, 4):
            m = M.Mesh(n, 1, 1.0, 2.0, p)
            c = np.arange(0, m.ncol, 37)
            X = m.zone_nodes(c, np.zeros(c.size, int))
            x = m.map_points(X, pts)
            dev[n, p] = (np.abs(np.linalg.norm(x, axis=-1) - 2.0) / 2.0).max()
    assert dev[18, 2] > dev[18, 3] > dev[18, 4]
    assert dev[18, 3] < 3e-5 and dev[18, 4] < 6e-6
    assert dev[18, 2] / dev[36, 2] > 3.5
    assert dev[18, 3] / dev[36, 3] > 7.0
    assert dev[18, 4] / dev[36, 4] > 12.0


def test_cube_vertex_keys_match_at_seams():
    m = M.Mesh(4, 1, 1.0, 2.0, 2)
    for v in range(m.nsv):
        cols = m.sv_cols[v]
        pos = []
        for c in cols:
            X = m.zone_nodes(c, 0)[0]
            q = list(m.col_verts[c]).index(v)
            pos.append(X[[0, 1, 2, 3][q]])
        pos = np.array(pos)
        assert np.abs(pos - pos[0]).max() < 1e-14
