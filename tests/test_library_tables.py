"""Host tables of the library (no GPU) pinned directly to what the paper prints:
the predictor's time-coupling matrix R (Eqs. B.9, C.18, D.28)."""
import numpy as np
import pytest

from test_oracle_refelem import load_r_matrices


@pytest.mark.parametrize("p", [2, 3, 4])
def test_library_time_matrix_is_the_printed_R(p):
    from paper_1905_02504_gb300 import geomhd
    R = geomhd.geo_time_matrix(p)
    printed = load_r_matrices()[p]
    assert np.abs(R - printed).max() < 1e-14


@pytest.mark.parametrize("n,nr,p", [(4, 4, 2), (4, 4, 3), (3, 5, 4)])
def test_library_geometry_matches_oracle_on_cpu(n, nr, p):
    """The library's host tables (geo_host_geometry, the tables geo_mesh_create
    uploads) give the oracle's zone volumes and centroids and face areas and
    area-weighted normals (isoparametric zones, Sec. II.b), and every zone's six
    signed area vectors close."""
    from oracle.step import Oracle
    from paper_1905_02504_gb300 import geomhd
    o = Oracle(n, nr, 1.0, 2.0, p)
    om = o.mesh
    xc, vol, area, nrm = geomhd.geo_host_geometry(n, nr, 1.0, 2.0, p, om.Z, om.F)
    c = np.repeat(np.arange(om.ncol), om.nr)
    k = np.tile(np.arange(om.nr), om.ncol)
    g = om.zone_geometry(c, k)
    assert np.abs(vol - g["V"]).max() <= 1e-13 * g["V"].max()
    assert np.abs(xc - g["xc"]).max() <= 1e-13
    ref_a = np.empty(om.F)
    ref_n = np.empty((om.F, 3))
    for f in range(om.F):
        zL, lfL = om.face_L[f]
        zR, lfR = om.face_R[f]
        z0, lf0, sgn = (zL, lfL, 1.0) if zL >= 0 else (zR, lfR, -1.0)
        fg = o.dfb.fgeo[lf0]
        ref_a[f] = o.dfb.area[z0, lf0]
        ref_n[f] = sgn * (fg["w"][:, None] * fg["dA"][z0][:, None] * fg["n"][z0]).sum(0)
    assert np.abs(area - ref_a).max() <= 1e-13 * ref_a.max()
    assert np.abs(nrm - ref_n).max() <= 1e-13 * ref_a.max()
    close = (om.zone_face_sign[..., None] * nrm[om.zone_face]).sum(1)
    assert np.abs(close).max() <= 1e-14 * ref_a.max()
