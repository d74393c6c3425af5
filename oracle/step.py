"""The full one-step update (Sec. VI), CFL time step and div B diagnostic -- oracle.

Step (Sec. VI, steps 2-5), for zone averages U (Z, 8) and primal face fluxes
Phi (F,):
  1. WENO-AO of all eight conserved variables (weno.py).
  2. Divergence-free reconstruction of B; the zone-centred B is overwritten with
     its constant terms (divfree.py, Sec. IV.b step 10).
  3. ADER-CG predictor (ader.py).
  4. Corrector:
     * face flux  F_f = dt sum_{m>=2} w_m sum_q w_q |dA_q| HLL(U_L, U_R; n_q)
       (or HLLD, riemann="hlld": the higher-fidelity face solver of the paper's
       introduction)
       at every face quadrature point and Gauss time (the space and time
       integrals switch places, Sec. V.d step 10);
     * edge EMF   E_e = dt sum_{m>=2} w_m sum_s w_s |dl_s| (E.t)_s with the
       multidimensional solver of physics.edge_emf at every edge point;
     * U_z <- U_z - (1/V_z) sum_f s_zf F_f      (finite-volume update, Eq. 2.2)
       Phi_f <- Phi_f - sum_e s_fe E_e           (Yee/CT update, Eqs. 2.5-2.6; the
       time integral already carries dt, reading the doubled dt of Eqs. 2.5-2.6
       as a misprint).
Boundaries (Sec. VII, "continuative outflow"): at r_in and r_out the missing
state of a face point equals the interior one; a boundary edge has the two
interior zones and the face between them (mirrored ghosts add equal halves).
CFL (Sec. VII.b): dt = cfl min_z d_z / (|v_z| + c_f,max), d_z = 6 V_z / S_z (the
in-sphere diameter of a tangential polyhedron), c_f,max^2 = gamma p/rho + B^2/rho.

Pinned by: tests/test_oracle_step.py -- free-stream preservation of a uniform state
on the curved mesh, discrete div B at rounding every step, conservation of mass
and energy up to the boundary-flux ledger, and the design order of accuracy on
the exact advected entropy wave; the CFL step of a uniform state against the
closed-form in-sphere diameter 6V/S of the exact spherical frustum (gnomonic
solid angle, great-circle side sectors), which the mapped zones approach at the
map's order; divB on hand-built fields with known per-zone divergence.
"""
import numpy as np

from . import positivity, quadrature
from .ader import AderPredictor
from .divfree import DivFreeB
from .mesh import Mesh
from .physics import edge_emf, hll, hlld, primitives, rusanov_speed, fast_speed
from .weno import WenoAO


class Oracle:
    def __init__(self, n, nr, r_in, r_out, p, gamma=5.0 / 3.0, positivity=False, riemann="hll"):
        self.gamma = gamma
        self.positivity = positivity
        assert riemann in ("hll", "hlld")
        self.riemann = hlld if riemann == "hlld" else hll
        m = self.mesh = Mesh(n, nr, r_in, r_out, p)
        self.weno = WenoAO(m)
        self.dfb = DivFreeB(m, self.weno)
        self.ader = AderPredictor(m, self.dfb.X, gamma)
        self.V = self.weno.geo0["V"]
        self.tau, self.wt = quadrature.time_gauss(p)
        self._build_face_tables()
        self._build_edge_tables()

    # --------------------------------------------------------------- tables
    def _build_face_tables(self):
        m = self.mesh
        self.face_ref = [self.dfb.fgeo[lf]["ref"] for lf in range(6)]

    def _build_edge_tables(self):
        m = self.mesh
        el = m.el
        t, w = quadrature.edge_rule(m.p)
        self.edge_w = w
        groups = {}
        X = self.dfb.X
        for e in range(m.E):
            zones, faces = m.edge_zones(e)
            z0, le0 = zones[0]
            g0 = m.edge_geometry(X[z0:z0 + 1], le0)
            x0 = g0["x"][0]
            tv = g0["t"][0]
            dl = g0["dl"][0]
            # canonical direction: +r for radial edges, va -> vb for angular ones
            if e < m.E_rad:
                rev = False
            else:
                se = (e - m.E_rad) // (m.nr + 1)
                va, vb = m.se_verts[se]
                rev = np.dot(tv[0], m.sv_dir[vb] - m.sv_dir[va]) < 0.0
            if rev:
                x0, tv, dl = x0[::-1], -tv[::-1], dl[::-1]
            slots = []
            for z, le in zones:
                gz = m.edge_geometry(X[z:z + 1], le)
                xz = gz["x"][0]
                d = np.linalg.norm(x0[:, None, :] - xz[None, :, :], axis=-1)
                pr = d.argmin(1)
                assert d[np.arange(len(pr)), pr].max() < 1e-9
                zrev = np.dot(gz["t"][0][pr[0]], tv[0]) < 0.0
                slots.append((z, le, pr, zrev))
            fl = []
            for f, iL, iR in faces:
                zL, lfL = m.face_L[f]
                zz, le, pr, _ = slots[iL]
                ref = refelem.edge_points(le, t)[pr]
                h = m.map_jacobian(X[zL:zL + 1], ref)[0]
                a = refelem.FACE_AXIS[lfL]
                vec = np.cross(h[:, (a + 1) % 3], h[:, (a + 2) % 3]) * np.sign(refelem.FACE_SIDE[lfL])
                nrm = vec / np.linalg.norm(vec, axis=-1, keepdims=True)
                fl.append((iL, iR, nrm))
            key = (len(zones), len(faces))
            groups.setdefault(key, []).append((e, slots, fl, x0, tv, dl))
        self.edge_groups = groups

    # ---------------------------------------------------------------- initial
    def initial_state(self, problem):
        """Zone averages by the zone cubature and Phi from the circulation of the
        vector potential along each edge (8-point Gauss per edge, Sec. VIII)."""
        m = self.mesh
        g0 = self.weno.geo0
        U = problem.zone_averages(g0["xg"], g0["dV"])
        X = self.dfb.X
        xq, wq = quadrature.gauss_legendre(8)
        circ = np.zeros(m.E)
        for (kz, kf), items in self.edge_groups.items():
            for e, slots, fl, x0, tv, dl in items:
                z, le, pr, zrev = slots[0]
                ref = refelem.edge_points(le, xq)
                x = m.map_points(X[z:z + 1], ref)[0]
                h = m.map_jacobian(X[z:z + 1], ref)[0][:, refelem.EDGE_AXIS[le]]
                tw = (-1.0 if zrev else 1.0) * h * wq[:, None]
                circ[e] = problem.edge_circulation(x[None], tw[None])[0]
        phi = (m.face_edge_sign * circ[m.face_edges]).sum(1)
        if getattr(problem, "has_radial_flux", lambda: False)():
            # fields given by their flux (the r^-2 radial field of the shock tubes,
            # Sec. VIII.c): the face rule over each radial face, normal along +r;
            # face (c, k) is the inner face of zone (c, k), the last the outer face
            # of the last shell
            fin, fout = self.dfb.fgeo[4], self.dfb.fgeo[5]
            z = np.arange(m.Z)
            c, k = z // m.nr, z % m.nr
            wn = -fin["n"] * (fin["w"][None, :] * fin["dA"])[..., None]
            phi[c * (m.nr + 1) + k] += problem.radial_face_flux(fin["x"], wn)
            last = z[k == m.nr - 1]
            wn = fout["n"][last] * (fout["w"][None, :] * fout["dA"][last])[..., None]
            phi[c[last] * (m.nr + 1) + m.nr] += problem.radial_face_flux(fout["x"][last], wn)
        return U, phi

    # ------------------------------------------------------------------ step
    def step(self, U, phi, dt, return_stages=False):
        m = self.mesh
        p = m.p
        g = self.gamma
        coeffs = self.weno.reconstruct(U)
        Bcoef, Bmean, bperp = self.dfb.reconstruct(coeffs, U, phi, return_bperp=True)
        U1 = U.copy()
        U1[:, 5:8] = Bmean
        X = self.dfb.X
        Unodes = np.empty(X.shape[:2] + (8,))
        Unodes[..., :5] = self.weno.evaluate(coeffs, U1, X)[..., :5]
        Unodes[..., 5:8] = self.dfb.evaluate(Bcoef, X)
        if self.positivity:
            Unodes, _ = positivity.limit(Unodes, U1, g)
        Uh = self.ader.predict(Unodes, dt)
        # ---- face fluxes
        traces = [self.ader.point_values(Uh, self.face_ref[lf]) for lf in range(6)]
        t, w = quadrature.edge_rule(p)
        edge_traces = [self.ader.point_values(Uh, refelem.edge_points(le, t)) for le in range(12)]
        if self.positivity:
            # one scaling per zone over every predicted face / edge point and Gauss time
            parts = [tr[:, 1:].reshape(m.Z, -1, 8) for tr in traces + edge_traces]
            sizes = [x.shape[1] for x in parts]
            lim, _ = positivity.limit(np.concatenate(parts, axis=1), U1, g)
            out, off = [], 0
            for tr, sz in zip(traces + edge_traces, sizes):
                new = tr.copy()
                new[:, 1:] = lim[:, off:off + sz].reshape(tr[:, 1:].shape)
                out.append(new)
                off += sz
            traces, edge_traces = out[:6], out[6:]
        Fface = np.zeros((m.F, 8))
        fg = self.dfb.fgeo
        for f in range(m.F):
            zL, lfL = m.face_L[f]
            zR, lfR = m.face_R[f]
            if zL >= 0:
                geo, z0, lf0, sgn = fg[lfL], zL, lfL, 1.0
            else:
                geo, z0, lf0, sgn = fg[lfR], zR, lfR, -1.0
            n = sgn * geo["n"][z0]
            W = geo["w"] * geo["dA"][z0]
            for mi in range(1, m.p):
                sL = traces[lfL][zL, mi] if zL >= 0 else None
                if zR >= 0:
                    sR = traces[lfR][zR, mi]
                    if zL >= 0:
                        sR = sR[self.dfb.face_perm[f]]
                else:
                    sR = sL
                if sL is None:
                    sL = sR
                Fq = self.riemann(sL, sR, n, g)
                Fface[f] += dt * self.wt[mi - 1] * (W[:, None] * Fq).sum(0)
        # ---- edge EMFs
        Eedge = np.zeros(m.E)
        for (kz, kf), items in self.edge_groups.items():
            for e, slots, fl, x0, tv, dl in items:
                acc = 0.0
                for mi in range(1, m.p):
                    for s in range(len(w)):
                        st = np.stack([edge_traces[le][z, mi, pr[s]] for z, le, pr, _ in slots])
                        faces = [(iL, iR, nrm[s]) for iL, iR, nrm in fl]
                        Es = edge_emf(st, faces, tv[s], g)
                        acc += self.wt[mi - 1] * w[s] * dl[s] * Es
                Eedge[e] = dt * acc
        # ---- update
        Unew = U1 - (m.zone_face_sign[..., None] * Fface[m.zone_face]).sum(1) / self.V[:, None]
        phinew = phi - (m.face_edge_sign * Eedge[m.face_edges]).sum(1)
        if return_stages:
            return Unew, phinew, dict(coeffs=coeffs, Bcoef=Bcoef, Bmean=Bmean, bperp=bperp,
                                      Uh=Uh, Fface=Fface, Eedge=Eedge)
        return Unew, phinew

    # ------------------------------------------------------------- diagnostics
    def cfl_dt(self, U, cfl):
        return cfl_time_step(U, self.V, self.dfb.area.sum(1), self.gamma, cfl)

    def divB(self, phi):
        m = self.mesh
        div = (m.zone_face_sign * phi[m.zone_face]).sum(1)
        scale = np.abs(phi[m.zone_face]).sum(1)
        return np.abs(div).max(), (np.abs(div) / np.maximum(scale, 1e-300)).max()


def cfl_time_step(U, V, S, gamma, cfl):
    """dt = cfl min_z d_z / (|v_z| + c_f,max,z) with d_z = 6 V_z / S_z, the in-sphere
    diameter of a tangential polyhedron of volume V_z and surface S_z (Sec. VII.b),
    and c_f,max^2 = gamma p / rho + B^2 / rho."""
    rho, v, p, B = primitives(U, gamma)
    cf = np.sqrt(gamma * p / rho + (B * B).sum(-1) / rho)
    d = 6.0 * V / S
    return cfl * np.min(d / (np.linalg.norm(v, axis=-1) + cf))


from . import refelem  # noqa: E402  (used in table construction above)
