"""Cubed-sphere geodesic mesh with log-ratioed radial shells and isoparametric
hexahedral zones (Sec. II.a-II.b, Sec. V.a) -- oracle version.

Readings of the paper taken here (the paper meshes with spherical icosahedra;
the build's mesh is a cubed sphere):
  * Angular mesh: equiangular gnomonic cube, every grid line a great circle
    (Fig. 2: "two great circles ... form a coordinate system"); n x n columns per
    cube face, n = 2^k reached by great-circle bisection.
  * Radial shells: r_k = r_in (r_out/r_in)^(k/nr) for any integer k, the
    logarithmically ratioed spacing the paper recommends (Sec. V.b); ghost shells
    (k < 0, k >= nr) continue the same law.
  * Isoparametric map (Eq. 5.2): x(xi) = sum_i X_i psi_i(xi) with the order-p
    serendipity basis; node X_i = rho(zeta_i) * P(alpha(xi_i), beta(eta_i)), P the
    equiangular point on the unit sphere, rho linear in zeta (radial variation
    always linear, Sec. II.b).  Angular map degree is p-1 (linear/quadratic/cubic).
  * Jacobian J = (h_xi x h_eta) . h_zeta, h = dx/dxi (Eqs. 5.4-5.5).
  * Cubature: tensor Gauss-Legendre, n_ang x n_ang x n_rad points with
    (n_ang, n_rad) = (3,2), (6,3), (11,4) for p = 2, 3, 4: exact for J times the
    moments of degree <= p used below.
  * Zone moments about the centroid, scaled by l_0 = V^(1/3) (Eqs. 3.2-3.3; the
    paper leaves l_0 open).

Canonical enumeration (the C-ABI uses the same numbering):
  columns   c = (f*n + j)*n + i, cube face f, angular indices i (alpha), j (beta)
  zones     z = c*nr + k
  sphere vertices: first appearance scanning columns, corners (v00, v10, v01, v11),
            key = integer lattice point of the cube surface
  sphere edges:    first appearance scanning columns, sides (s, e, n, w); canonical
            direction from the lower to the higher sphere-vertex id
  faces     radial (c, k), k = 0..nr at r_k: c*(nr+1)+k, normal +r, L=(c,k-1), R=(c,k)
            angular (se, k): F_rad + se*nr + k, normal along t x r (t = edge
            direction), L = the column on the -normal side
  edges     radial (sv, k) from r_k to r_k+1: sv*nr + k, direction +r
            angular (se, k) at r_k: E_rad + se*(nr+1) + k, direction of se
Face/edge orientation: Phi_f is the flux through the face along its canonical
normal; face boundary traversed counter-clockwise about the normal; an edge
enters with sign +1 when its direction agrees (Eqs. 2.5-2.6).

Pinned by: tests/test_oracle_mesh.py -- closure sum_faces sum_q n dA = 0 per zone,
total volume converging to 4/3 pi (r_out^3 - r_in^3), sphericity deviation
shrinking with map order (Fig. 4 analogue), Euler characteristic of the sphere
grid, face/edge incidence giving d(curl) = 0, vertex keys matching at seams.
"""
import numpy as np

from . import quadrature, refelem

# cube face frames (e_a, e_b, e_n), right handed: e_a x e_b = e_n
_X = np.array([1, 0, 0])
_Y = np.array([0, 1, 0])
_Z = np.array([0, 0, 1])
FRAMES = np.array([
    [_Y, _Z, _X],
    [_Z, _X, _Y],
    [_X, _Y, _Z],
    [_Z, _Y, -_X],
    [_X, _Z, -_Y],
    [_Y, _X, -_Z],
], dtype=np.int64)

CUBATURE = {2: (3, 2), 3: (6, 3), 4: (11, 4)}


def taylor_exponents(dmax, dmin=1):
    """Monomials of degree dmin..dmax ordered by degree, then by descending
    exponent of x, then of y (x, y, z | xx, xy, xz, yy, yz, zz | ...)."""
    out = []
    for d in range(dmin, dmax + 1):
        for a in range(d, -1, -1):
            for b in range(d - a, -1, -1):
                out.append((a, b, d - a - b))
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def sphere_point(f, alpha, beta):
    ea, eb, en = FRAMES[f].astype(np.float64)
    ta = np.tan(alpha)[..., None]
    tb = np.tan(beta)[..., None]
    v = ta * ea + tb * eb + en
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


class Mesh:
    def __init__(self, n, nr, r_in, r_out, p):
        self.n, self.nr, self.r_in, self.r_out, self.p = n, nr, float(r_in), float(r_out), p
        self.el = refelem.HexElement(p)
        self.N = self.el.N
        self.ncol = 6 * n * n
        self.Z = self.ncol * nr
        cols = np.arange(self.ncol)
        self.col_f = cols // (n * n)
        self.col_j = (cols // n) % n
        self.col_i = cols % n
        self._build_topology()
        self._build_faces_edges()

    # ------------------------------------------------------------------ radii
    def radius(self, k):
        return self.r_in * (self.r_out / self.r_in) ** (np.asarray(k, dtype=np.float64) / self.nr)

    # -------------------------------------------------------------- topology
    def _build_topology(self):
        n = self.n
        key_to_id = {}
        self.col_verts = np.zeros((self.ncol, 4), dtype=np.int64)
        sv_pos = []
        for c in range(self.ncol):
            f, i, j = self.col_f[c], self.col_i[c], self.col_j[c]
            ea, eb, en = FRAMES[f]
            for q, (di, dj) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
                key = tuple((2 * (i + di) - n) * ea + (2 * (j + dj) - n) * eb + n * en)
                if key not in key_to_id:
                    key_to_id[key] = len(key_to_id)
                    sv_pos.append(np.array(key, dtype=np.float64))
                self.col_verts[c, q] = key_to_id[key]
        self.nsv = len(key_to_id)
        self.sv_dir = np.array(sv_pos)
        self.sv_dir /= np.linalg.norm(self.sv_dir, axis=1, keepdims=True)
        # sides s (v00->v10), e (v10->v11), n (v01->v11), w (v00->v01): local order
        side_pairs = ((0, 1), (1, 3), (2, 3), (0, 2))
        ekey = {}
        self.col_edges = np.zeros((self.ncol, 4), dtype=np.int64)
        se_verts, se_cols = [], []
        for c in range(self.ncol):
            for s, (a, b) in enumerate(side_pairs):
                va, vb = self.col_verts[c, a], self.col_verts[c, b]
                key = (min(va, vb), max(va, vb))
                if key not in ekey:
                    ekey[key] = len(ekey)
                    se_verts.append(key)
                    se_cols.append([])
                e = ekey[key]
                se_cols[e].append(c)
                self.col_edges[c, s] = e
        self.nse = len(ekey)
        self.se_verts = np.array(se_verts, dtype=np.int64)
        assert all(len(x) == 2 for x in se_cols)
        # counter-clockwise direction of each side about +r: s: v00->v10, e: v10->v11,
        # n: v11->v01, w: v01->v00.  ccw_sign[c, s] = +1 if the canonical direction of
        # the sphere edge agrees with it.
        ccw = ((0, 1), (1, 3), (3, 2), (2, 0))
        self.col_ccw_sign = np.zeros((self.ncol, 4), dtype=np.int64)
        for c in range(self.ncol):
            for s, (a, b) in enumerate(ccw):
                va = self.col_verts[c, a]
                e = self.col_edges[c, s]
                self.col_ccw_sign[c, s] = 1 if self.se_verts[e, 0] == va else -1
        # L column of an angular face: the one whose ccw direction equals the
        # canonical direction (its outward normal t_ccw x r is the canonical normal)
        self.se_L = np.full(self.nse, -1, dtype=np.int64)
        self.se_R = np.full(self.nse, -1, dtype=np.int64)
        for e in range(self.nse):
            for c in se_cols[e]:
                s = list(self.col_edges[c]).index(e)
                if self.col_ccw_sign[c, s] > 0:
                    self.se_L[e] = c
                else:
                    self.se_R[e] = c
        assert (self.se_L >= 0).all() and (self.se_R >= 0).all()
        # sphere edges incident to each sphere vertex
        self.sv_edges = [[] for _ in range(self.nsv)]
        for e in range(self.nse):
            for v in self.se_verts[e]:
                self.sv_edges[v].append(e)
        self.sv_cols = [[] for _ in range(self.nsv)]
        for c in range(self.ncol):
            for v in self.col_verts[c]:
                self.sv_cols[v].append(c)

    # --------------------------------------------------------- isoparametric map
    def zone_nodes(self, c, k):
        """Map nodes X_i of zones (c, k) -> (nz, N, 3)."""
        c = np.atleast_1d(c)
        k = np.atleast_1d(k)
        n = self.n
        d = 0.5 * np.pi / n
        xi = self.el.nodes
        a = -0.25 * np.pi + (self.col_i[c][:, None] + xi[None, :, 0] + 0.5) * d
        b = -0.25 * np.pi + (self.col_j[c][:, None] + xi[None, :, 1] + 0.5) * d
        out = np.zeros((c.size, self.N, 3))
        for f in range(6):
            m = self.col_f[c] == f
            if m.any():
                out[m] = sphere_point(f, a[m], b[m])
        r0 = self.radius(k)[:, None]
        r1 = self.radius(k + 1)[:, None]
        rho = r0 * (0.5 - xi[None, :, 2]) + r1 * (0.5 + xi[None, :, 2])
        return out * rho[..., None]

    def map_points(self, X, pts):
        """x(pts) for zones with nodes X (nz, N, 3), pts (np, 3) -> (nz, np, 3)."""
        return np.einsum("pn,znd->zpd", self.el.basis(pts), X)

    def map_jacobian(self, X, pts):
        """h[a] = dx/dxi_a at pts -> (nz, np, 3(a), 3(component))."""
        return np.stack([np.einsum("pn,znd->zpd", self.el.dbasis(pts, a), X)
                         for a in range(3)], axis=2)

    # ---------------------------------------------------------- zone geometry
    def cubature(self):
        na, nrd = CUBATURE[self.p]
        xa, wa = quadrature.gauss_legendre(na)
        xr, wr = quadrature.gauss_legendre(nrd)
        pts = np.array([[x, y, z] for x in xa for y in xa for z in xr])
        wts = np.array([wx * wy * wz for wx in wa for wy in wa for wz in wr])
        return pts, wts

    def zone_geometry(self, c, k):
        """Volume, centroid, l_0, cubature points/weights (physical) of zones (c,k)."""
        X = self.zone_nodes(c, k)
        pts, wts = self.cubature()
        xg = self.map_points(X, pts)
        h = self.map_jacobian(X, pts)
        J = np.einsum("zpd,zpd->zp", np.cross(h[:, :, 0], h[:, :, 1]), h[:, :, 2])
        dV = J * wts[None, :]
        V = dV.sum(axis=1)
        xc = np.einsum("zp,zpd->zd", dV, xg) / V[:, None]
        l0 = V ** (1.0 / 3.0)
        return dict(X=X, V=V, xc=xc, l0=l0, xg=xg, dV=dV, J=J)

    def scaled_moments(self, geo_of, xc0, l00, exps):
        """<((x - xc0)/l00)^e> over the zones described by geo_of -> (nz, ne)."""
        s = (geo_of["xg"] - xc0[:, None, :]) / l00[:, None, None]
        # integer powers by repeated products: pw[d][k] = s_d^k
        pw = []
        for d in range(3):
            pw.append([np.ones(s.shape[:2])])
            for _ in range(int(exps[:, d].max())):
                pw[d].append(pw[d][-1] * s[..., d])
        vals = np.empty((s.shape[0], len(exps), s.shape[1]))
        for j, (a, b, c) in enumerate(exps):
            vals[:, j] = pw[0][a] * pw[1][b] * pw[2][c]
        return (vals @ geo_of["dV"][:, :, None])[..., 0] / geo_of["V"][:, None]

    # ------------------------------------------------------ faces and edges
    def face_geometry(self, X, lf):
        """Quadrature data of local face lf for zones with nodes X: reference
        points, reference weights, physical points, outward unit normals, |dA|."""
        rule_pts, rule_w = quadrature.face_rule(self.p, radial_face=(lf >= 4))
        ref = refelem.face_points(lf, rule_pts)
        x = self.map_points(X, ref)
        h = self.map_jacobian(X, ref)
        a = refelem.FACE_AXIS[lf]
        vec = np.cross(h[:, :, (a + 1) % 3], h[:, :, (a + 2) % 3]) * np.sign(refelem.FACE_SIDE[lf])
        dA = np.linalg.norm(vec, axis=-1)
        return dict(ref=ref, w=rule_w, x=x, n=vec / dA[..., None], dA=dA)

    def edge_geometry(self, X, le):
        """Edge-rule data of local edge le (parameter increasing)."""
        t, w = quadrature.edge_rule(self.p)
        ref = refelem.edge_points(le, t)
        x = self.map_points(X, ref)
        h = self.map_jacobian(X, ref)[:, :, refelem.EDGE_AXIS[le]]
        dl = np.linalg.norm(h, axis=-1)
        return dict(ref=ref, w=w, x=x, t=h / dl[..., None], dl=dl)

    def _build_faces_edges(self):
        nr = self.nr
        self.F_rad = self.ncol * (nr + 1)
        self.F = self.F_rad + self.nse * nr
        self.E_rad = self.nsv * nr
        self.E = self.E_rad + self.nse * (nr + 1)
        Z = self.Z
        # zone -> faces (local order 0..5) and outward signs
        side_of_lf = {0: 3, 1: 1, 2: 0, 3: 2}      # local face -> side index (s,e,n,w)
        self.zone_face = np.zeros((Z, 6), dtype=np.int64)
        self.zone_face_sign = np.zeros((Z, 6), dtype=np.int64)
        for c in range(self.ncol):
            for k in range(nr):
                z = c * nr + k
                for lf in range(4):
                    s = side_of_lf[lf]
                    se = self.col_edges[c, s]
                    self.zone_face[z, lf] = self.F_rad + se * nr + k
                    self.zone_face_sign[z, lf] = self.col_ccw_sign[c, s]
                self.zone_face[z, 4] = c * (nr + 1) + k
                self.zone_face_sign[z, 4] = -1
                self.zone_face[z, 5] = c * (nr + 1) + k + 1
                self.zone_face_sign[z, 5] = 1
        # face -> (L zone, local face in L, R zone, local face in R); -1 = boundary
        self.face_L = np.full((self.F, 2), -1, dtype=np.int64)
        self.face_R = np.full((self.F, 2), -1, dtype=np.int64)
        for z in range(Z):
            for lf in range(6):
                f = self.zone_face[z, lf]
                tgt = self.face_L if self.zone_face_sign[z, lf] > 0 else self.face_R
                assert tgt[f, 0] < 0
                tgt[f] = (z, lf)
        # face -> 4 edges with circulation signs (counter-clockwise about the normal)
        self.face_edges = np.zeros((self.F, 4), dtype=np.int64)
        self.face_edge_sign = np.zeros((self.F, 4), dtype=np.int64)
        ccw_sides = (0, 1, 2, 3)
        for c in range(self.ncol):
            for k in range(nr + 1):
                f = c * (nr + 1) + k
                for q, s in enumerate(ccw_sides):
                    se = self.col_edges[c, s]
                    self.face_edges[f, q] = self.E_rad + se * (nr + 1) + k
                    self.face_edge_sign[f, q] = self.col_ccw_sign[c, s]
        for se in range(self.nse):
            va, vb = self.se_verts[se]
            for k in range(nr):
                f = self.F_rad + se * nr + k
                self.face_edges[f] = (self.E_rad + se * (nr + 1) + k, vb * nr + k,
                                      self.E_rad + se * (nr + 1) + k + 1, va * nr + k)
                self.face_edge_sign[f] = (1, 1, -1, -1)

    # ---------------------------------------------------------- edge stencils
    def edge_zones(self, e):
        """Zones around edge e with their local edge index, and the faces between
        them as (face, index of L zone in the list, index of R zone in the list)."""
        nr = self.nr
        lf_of_side = {0: 2, 1: 1, 2: 3, 3: 0}   # side (s,e,n,w) -> local face
        if e < self.E_rad:
            sv, k = divmod(e, nr)
            zones = []
            for c in self.sv_cols[sv]:
                corner = list(self.col_verts[c]).index(sv)      # v00,v10,v01,v11
                ix, iy = corner % 2, corner // 2
                zones.append((c * nr + k, 8 + ix + 2 * iy))
            faces = []
            for se in self.sv_edges[sv]:
                f = self.F_rad + se * nr + k
                faces.append(f)
        else:
            se, kk = divmod(e - self.E_rad, nr + 1)
            zones = []
            for c in (self.se_L[se], self.se_R[se]):
                s = list(self.col_edges[c]).index(se)
                for k in (kk - 1, kk):
                    if k < 0 or k >= nr:
                        continue
                    top = 1 if k == kk - 1 else 0       # edge at zeta=+1/2 of zone k=kk-1
                    if s in (0, 2):                     # along xi, eta = -/+
                        le = 0 + (1 if s == 2 else 0) + 2 * top
                    else:                               # along eta, xi = +/-
                        le = 4 + (1 if s == 1 else 0) + 2 * top
                    zones.append((c * nr + k, le))
            faces = []
            for k in (kk - 1, kk):
                if 0 <= k < nr:
                    faces.append(self.F_rad + se * nr + k)
            if 1 <= kk <= nr - 1:
                for c in (self.se_L[se], self.se_R[se]):
                    faces.append(c * (nr + 1) + kk)
        zlist = [z for z, _ in zones]
        flist = []
        for f in faces:
            L, R = self.face_L[f, 0], self.face_R[f, 0]
            flist.append((f, zlist.index(L), zlist.index(R)))
        return zones, flist
