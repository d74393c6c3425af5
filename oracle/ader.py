"""ADER-CG predictor on isoparametrically mapped zones (Sec. V, Eqs. 5.20-5.29,
App. C Eqs. C.34-C.36, App. D Eqs. D.29-D.32) -- oracle.

Per zone, with the order-p serendipity nodes x_i (i = 1..N) and M = p time levels:
  1. Metric terms at the nodes (Sec. V.d step 4): J_i = (h_xi x h_eta).h_zeta,
     S^xi = h_eta x h_zeta, S^eta = h_zeta x h_xi, S^zeta = h_xi x h_eta
     (computed for every zone; no self-similarity shortcut).
  2. Initialisation (steps 5-6): U_hat_{1,i} = J_i U(x_i) from the WENO-AO
     polynomial (fluid) and the divergence-free polynomial (B); all levels start
     from level 1.
  3. Nodal fluxes (Eq. 5.23 with the zone's own metrics): F_hat_{m,j} =
     dt S^xi_j . F(U_hat_{m,j}/J_j), likewise G_hat, H_hat.
  4. Flux difference at node i (Eq. C.34):
       dF_{m,i} = sum_j D^xi_ij F_hat_{m,j} + D^eta_ij G_hat_{m,j} + D^zeta_ij H_hat_{m,j}
                  - dt F(U_hat_{m,i}/J_i) . g_i,     g_i = sum_alpha sum_j D^alpha_ij S^alpha_j
     The last term is the discrete geometric-conservation residual of the nodal
     metrics; the paper does not discuss it, the build subtracts it so that a
     uniform state is preserved to rounding on curved zones (it is O(truncation)
     for smooth data).  Source terms are zero for ideal MHD.
  5. Picard update (Eqs. C.35-C.36): U_hat_{k,i} = U_hat_{1,i} - sum_m R_km dF_{m,i},
     k = 2..M, repeated p times (step 9: 2/3/4 iterations).
Outputs: the space-time nodal solution.  Point values (face and edge points at
the Gauss times tau_2..tau_M) are U(x, tau_m) = sum_i U_hat_{m,i} psi_i(x) /
sum_i J_i psi_i(x): the nodal interpolant of J U divided by the interpolant of J
(so a uniform state stays exactly uniform).

Pinned by: tests/test_oracle_divfree_ader.py -- uniform state preserved to rounding on the
curved mesh; on an affinely mapped zone, linear advection of a polynomial of
degree <= p-1 is reproduced exactly in space-time after p iterations; the nodal
flux-difference row matches Eq. B.16 on the paper's prism.
"""
import numpy as np

from . import refelem
from .physics import flux_dir


class AderPredictor:
    def __init__(self, mesh, X, gamma):
        self.mesh = mesh
        self.gamma = gamma
        el = self.el = mesh.el
        self.p = mesh.p
        self.M = mesh.p
        self.R, _ = refelem.r_matrix(mesh.p)
        self.X = X
        h = mesh.map_jacobian(X, el.nodes)                     # (Z, N, 3, 3)
        hx, hy, hz = h[:, :, 0], h[:, :, 1], h[:, :, 2]
        self.J = np.einsum("znd,znd->zn", np.cross(hx, hy), hz)
        self.S = np.stack([np.cross(hy, hz), np.cross(hz, hx), np.cross(hx, hy)], axis=1)
        self.gcl = sum(np.einsum("ij,zjd->zid", el.D[a], self.S[:, a]) for a in range(3))

    def flux_difference(self, Uh, dt):
        """dF_i of Eq. C.34 (with the geometric-conservation term) for one level."""
        Up = Uh / self.J[..., None]
        g = self.gamma
        out = np.zeros_like(Uh)
        for a in range(3):
            Fa = dt * flux_dir(Up, self.S[:, a], g)
            out += np.einsum("ij,zjv->ziv", self.el.D[a], Fa)
        out -= dt * flux_dir(Up, self.gcl, g)
        return out

    def predict(self, Unodes, dt):
        """Unodes: reconstructed conserved values at the nodes (Z, N, 8) ->
        space-time nodal U_hat (Z, M, N, 8)."""
        U1 = self.J[..., None] * Unodes
        levels = [U1] + [U1.copy() for _ in range(self.M - 1)]
        dF1 = self.flux_difference(U1, dt)
        for _ in range(self.p):
            dF = [dF1] + [self.flux_difference(levels[m], dt) for m in range(1, self.M)]
            new = []
            for k in range(1, self.M):
                acc = U1.copy()
                for m in range(self.M):
                    acc = acc - self.R[k, m] * dF[m]
                new.append(acc)
            levels = [U1] + new
        return np.stack(levels, axis=1)

    def point_values(self, Uh, ref_pts):
        """States at reference points for every level -> (Z, M, np, 8)."""
        psi = self.el.basis(ref_pts)                            # (np, N)
        num = np.einsum("pn,zmnv->zmpv", psi, Uh)
        den = psi @ self.J.T                                    # (np, Z)
        return num / den.T[:, None, :, None]
