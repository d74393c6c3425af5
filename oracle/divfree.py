"""Divergence-free reconstruction of the magnetic field on isoparametric zones
(Sec. IV.a-IV.b, Eqs. 4.1-4.15) -- oracle.

Per zone, in the zone's Taylor basis s = (x - x_0)/l_0:
  * Ansatz (Eqs. 4.1, 4.4, 4.7 generalised to every order): component B^d is the
    complete Taylor basis of degree <= p-1 (with the constant) plus every degree-p
    monomial that contains s_d, each minus its zone mean; 7/16/30 terms for
    p = 2/3/4 (p = 3 reproduces Eq. 4.1 exactly).
  * Nodal normal fields at each face point (Eq. 4.11):
      Bperp_i = <Bperp> + MinMod(n_i.B_L(x_i) - <Bperp>, n_i.B_R(x_i) - <Bperp>)
    with B_L, B_R the WENO-AO polynomials of the zone magnetic field of the two
    zones, then the mean-consistency shift (Eq. 4.12) so that Eq. 4.13 holds with
    w_i = (reference weight x surface Jacobian)/A_j (these w_i sum to one).
    <Bperp> = Phi_f / A_f, Phi_f the primal face flux.  MinMod(a,b) =
    sign(a) min(|a|,|b|) if ab > 0 else 0.  At a domain boundary face the missing
    side takes the interior polynomial (MinMod(a,a) = a).
  * Constraints (exact): every coefficient of div B of degree 1..p-1 vanishes (Eq.
    4.10 minus the constant one, which is implied by the face constraints), and the
    six face integrals match <Bperp> (Eq. 4.14).
  * Least-squares rows, unit weights (Steps 5-6 of Sec. IV.b): coefficients of
    degree <= p-1 equal the WENO-AO coefficients of the zone field, degree-p
    coefficients equal zero (Eqs. 4.3, 4.6, 4.9), and the nodal rows of Eq. 4.15.
  * KKT system [[A^T A, C^T], [C, 0]] solved densely per zone (Step 7 without the
    radial-column amortisation, which only the GPU path uses).
  * Step 10: the zone-centred B becomes the constant terms of the solution.

Pinned by: tests/test_oracle_divfree_ader.py -- for B = curl A with a polynomial A of
degree <= p the reconstruction has div B = 0 identically and reproduces a linear
field exactly; Eq. 4.13 holds to rounding; the face constraints hold; the mean
equals the face-consistent value.
"""
import numpy as np

from . import refelem
from .mesh import taylor_exponents


def minmod(a, b):
    from . import physics
    if physics.BRANCHES is not None:
        s = np.abs(a) + np.abs(b) + 1e-300
        physics.record("minmod", np.stack([a * b / (s * s), (np.abs(b) - np.abs(a)) / s]))
    return np.where(a * b > 0.0, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)


def component_terms(p, d):
    """Exponents of the ansatz of component d (constant first)."""
    base = taylor_exponents(p - 1, 0)
    top = taylor_exponents(p, p)
    extra = top[top[:, d] >= 1]
    return np.concatenate([base, extra])


def poly_values(s, exps, means):
    """phi_t(s) = s^e - mean_t (constant term: 1) -> (..., nt)."""
    v = np.ones(s.shape[:-1] + (len(exps),))
    for d in range(3):
        v *= s[..., d:d + 1] ** exps[:, d]
    return v - means


class DivFreeB:
    def __init__(self, mesh, weno):
        m = self.mesh = mesh
        p = m.p
        self.weno = weno
        g0 = weno.geo0
        Z = m.Z
        self.terms = [component_terms(p, d) for d in range(3)]
        self.nb = len(self.terms[0])
        nb = self.nb
        self.means = []
        for d in range(3):
            mm = m.scaled_moments(g0, g0["xc"], g0["l0"], self.terms[d])
            mm[:, 0] = 0.0                                  # constant term is 1
            self.means.append(mm)
        self.nc = len(taylor_exponents(p - 1, 0))
        X = g0.get("X")
        if X is None:
            zc = np.repeat(np.arange(m.ncol), m.nr)
            zk = np.tile(np.arange(m.nr), m.ncol)
            X = m.zone_nodes(zc, zk)
        self.X = X
        # zone-local face data
        self.fgeo = [m.face_geometry(X, lf) for lf in range(6)]
        self.nq = [len(fg["w"]) for fg in self.fgeo]
        self.area = np.stack([np.einsum("q,zq->z", fg["w"], fg["dA"]) for fg in self.fgeo], 1)
        # point correspondence across every face: R-local index of L point q
        self.face_perm = self._face_perm()
        # ---- constraint matrix C and least-squares matrix A per zone
        s_l0 = g0["l0"]
        div_rows = taylor_exponents(p - 1, 1)
        nC = len(div_rows) + 6
        nx = 3 * nb
        C = np.zeros((Z, nC, nx))
        for r, mu in enumerate(div_rows):
            for d in range(3):
                for t, e in enumerate(self.terms[d]):
                    if e[d] == 0:
                        continue
                    lowered = e.copy()
                    lowered[d] -= 1
                    if np.array_equal(lowered, mu):
                        C[:, r, d * nb + t] = e[d] / s_l0
        nodal_blocks = []
        for lf in range(6):
            fg = self.fgeo[lf]
            s = (fg["x"] - g0["xc"][:, None, :]) / s_l0[:, None, None]
            wq = fg["w"][None, :] * fg["dA"] / self.area[:, lf:lf + 1]
            blk = np.zeros((Z, len(fg["w"]), nx))
            for d in range(3):
                phi = poly_values(s, self.terms[d], self.means[d][:, None, :])
                blk[:, :, d * nb:(d + 1) * nb] = fg["n"][..., d:d + 1] * phi
            nodal_blocks.append(blk)
            C[:, len(div_rows) + lf, :] = np.einsum("zq,zqx->zx", wq, blk)
        A = np.concatenate([np.broadcast_to(np.eye(nx), (Z, nx, nx))] + nodal_blocks, axis=1)
        self.A = A
        self.C = C
        K = np.zeros((Z, nx + nC, nx + nC))
        K[:, :nx, :nx] = np.einsum("zrx,zry->zxy", A, A)
        K[:, :nx, nx:] = np.transpose(C, (0, 2, 1))
        K[:, nx:, :nx] = C
        self.K = K
        self.n_div = len(div_rows)

    def _face_perm(self):
        m = self.mesh
        perm = {}
        for f in range(m.F):
            zL, lfL = m.face_L[f]
            zR, lfR = m.face_R[f]
            if zL < 0 or zR < 0:
                continue
            xL = self.fgeo[lfL]["x"][zL]
            xR = self.fgeo[lfR]["x"][zR]
            d = np.linalg.norm(xL[:, None, :] - xR[None, :, :], axis=-1)
            pr = d.argmin(axis=1)
            assert d[np.arange(len(pr)), pr].max() < 1e-9 and len(set(pr)) == len(pr)
            perm[f] = pr
        return perm

    def face_bperp(self, weno_coeffs, U, phi):
        """Nodal normal fields per face (Eqs. 4.11-4.12), canonical orientation, in
        the L zone's point order (R's when the face has no L zone)."""
        m = self.mesh
        out = {}
        Bvals = []
        for lf in range(6):
            vals = self.weno.evaluate(weno_coeffs, U, self.fgeo[lf]["x"])[..., 5:8]
            Bvals.append(vals)                               # (Z, nq, 3)
        for f in range(m.F):
            zL, lfL = m.face_L[f]
            zR, lfR = m.face_R[f]
            if zL >= 0:
                fg, z0, lf0, sgn = self.fgeo[lfL], zL, lfL, 1.0
            else:
                fg, z0, lf0, sgn = self.fgeo[lfR], zR, lfR, -1.0
            n = sgn * fg["n"][z0]
            w = fg["w"] * fg["dA"][z0] / self.area[z0, lf0]
            mean = phi[f] / self.area[z0, lf0]
            bL = (n * Bvals[lfL][zL]).sum(-1) if zL >= 0 else None
            if zR >= 0:
                BR = Bvals[lfR][zR]
                if zL >= 0:
                    BR = BR[self.face_perm[f]]
                bR = (n * BR).sum(-1)
            else:
                bR = None
            if bL is None:
                bL = bR
            if bR is None:
                bR = bL
            b = mean + minmod(bL - mean, bR - mean)
            b = b + (mean - (w * b).sum())
            out[f] = b
        return out

    def reconstruct(self, weno_coeffs, U, phi, return_bperp=False):
        """Divergence-free coefficients (Z, 3, nb) and the new zone-mean B (Z, 3)."""
        m = self.mesh
        Z = m.Z
        nb = self.nb
        nx = 3 * nb
        bperp = self.face_bperp(weno_coeffs, U, phi)
        b = np.zeros((Z, self.A.shape[1]))
        d = np.zeros((Z, self.C.shape[1]))
        for dcomp in range(3):
            b[:, dcomp * nb] = U[:, 5 + dcomp]
            b[:, dcomp * nb + 1:dcomp * nb + self.nc] = weno_coeffs[:, 5 + dcomp, :]
        for z in range(Z):
            row = nx
            for lf in range(6):
                f = m.zone_face[z, lf]
                sgn = m.zone_face_sign[z, lf]
                vals = bperp[f]
                if sgn < 0 and m.face_L[f, 0] >= 0:
                    # z is R: its point q' holds the L point q with perm[q] = q'
                    loc = np.empty_like(vals)
                    loc[self.face_perm[f]] = vals
                    vals = loc
                nq = self.nq[lf]
                b[z, row:row + nq] = sgn * vals
                row += nq
                d[z, self.n_div + lf] = sgn * phi[f] / self.area[z, lf]
        rhs = np.concatenate([np.einsum("zrx,zr->zx", self.A, b), d], axis=1)
        sol = np.linalg.solve(self.K, rhs[..., None])[..., 0]
        coef = sol[:, :nx].reshape(Z, 3, nb)
        if return_bperp:
            return coef, coef[:, :, 0].copy(), bperp
        return coef, coef[:, :, 0].copy()

    def evaluate(self, coef, pts):
        """B at physical points pts (Z, np, 3) -> (Z, np, 3)."""
        g0 = self.weno.geo0
        s = (pts - g0["xc"][:, None, :]) / g0["l0"][:, None, None]
        out = np.zeros(pts.shape)
        for d in range(3):
            phi = poly_values(s, self.terms[d], self.means[d][:, None, :])
            out[..., d] = np.einsum("zpt,zt->zp", phi, coef[:, d, :])
        return out
