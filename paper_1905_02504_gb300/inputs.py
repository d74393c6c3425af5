"""Seeded synthetic initial data shared by the CUDA path's harness and the oracle.

This module holds no arithmetic of the method: it only defines the analytic
initial conditions of the synthetic workloads (primitive fields and a vector
potential), a counter-based random generator, and averaging helpers that take
points and weights from whichever mesh implementation asks (each side integrates
with its own geometry).

Workloads (rationalised units, gamma = 5/3 unless stated):
  smooth  rho = 1 + 0.1 sin(2 pi (x+y+z)/sqrt3), p = 1, v = (0.5, 0.5, 0.5),
          A = 0.1 (sin 2 pi z, sin 2 pi x, sin 2 pi y)  ->  B = curl A
  entropy rho = 1 + 0.1 sin(2 pi (x+y+z)/sqrt3), p = 1, v = v0, uniform B0
          (an exact solution: rho(x - v0 t)); A = B0 x r / 2
  blast   rho = 1, v = 0, p = 100 inside |x - (0,0,1.5)| < 0.1, else 0.1,
          B = (0, 0, 10/sqrt(4 pi)), A = B x r / 2
  lowbeta rho = 1, v = 0, p_out = 0.1, p_in = 1000 p_out, same sphere,
          B = (1,1,0) sqrt(2 p_out / 0.01)/sqrt2 (plasma beta 0.01 outside)
Spherical shock tubes (paper Sec. VIII.c; theta the polar angle from +z, fields
in rationalised units, i.e. the paper's Gaussian values divided by sqrt(4 pi)):
  sod      r in [2, 3]: (rho, p) = (1, 1) for r <= 2.5, (0.125, 0.1) outside,
           v = 0, B = 0, gamma = 1.4 (the standard Sod value; the paper gives none)
  briowu   r in [4, 6], r_m = 4.5: (rho, p) = (1, 1) inside, (0.125, 0.1) outside,
           v = 0, B_phi = +1 / -1, B_r = 0.75 sin(theta) (4.5/r)^2, gamma = 2
  ryujones r in [3, 6], r_m = 4.5: (rho, p, v_r) = (1, 20, 10) inside,
           (1, 1, -10) outside, B_phi = 5/sqrt(4 pi) on both sides,
           B_r = 5/sqrt(4 pi) sin(theta) (4.5/r)^2, gamma = 5/3
  The toroidal field comes from A = A_r r_hat,
    A_r = (B_phiL/2) r cos(theta) [1 - tanh((r - r_m)/delta)]
        + (B_phiR/2) r cos(theta) [1 + tanh((r - r_m)/delta)],
  whose curl is the tanh-tapered B_phi sin(theta) (delta ~ half a radial zone);
  the fluid jumps are sharp.  The radial field has net flux through every sphere,
  so it has no single-valued vector potential on the shell: its face fluxes are
  integrated directly over the radial faces (radial_face_flux).
Optional multiplicative density noise rho *= (1 + amp u), u in [-1, 1) drawn by
splitmix64(seed ^ zone_id) (seed 1905).
"""
import numpy as np

GAMMA = 5.0 / 3.0
SEED = 1905
_MASK = (1 << 64) - 1


def splitmix64(x):
    """splitmix64 finaliser of a uint64 array (Steele, Lea & Flood 2014)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(ids, seed=SEED):
    """Counter-based uniform numbers in [-1, 1) for integer ids."""
    z = splitmix64(np.asarray(ids, dtype=np.uint64) ^ np.uint64(seed))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


# radial extent of each workload's shell
DOMAINS = {"sod": (2.0, 3.0), "briowu": (4.0, 6.0), "ryujones": (3.0, 6.0)}
SHOCK_TUBES = {
    # name: (gamma, r_m, (rho, p, v_r) inside, (rho, p, v_r) outside, B_phiL, B_phiR, B_r0)
    "sod": (1.4, 2.5, (1.0, 1.0, 0.0), (0.125, 0.1, 0.0), 0.0, 0.0, 0.0),
    "briowu": (2.0, 4.5, (1.0, 1.0, 0.0), (0.125, 0.1, 0.0), 1.0, -1.0, 0.75),
    "ryujones": (5.0 / 3.0, 4.5, (1.0, 20.0, 10.0), (1.0, 1.0, -10.0), 5.0 / np.sqrt(4.0 * np.pi),
                 5.0 / np.sqrt(4.0 * np.pi), 5.0 / np.sqrt(4.0 * np.pi)),
}


def domain(name):
    """(r_in, r_out) of a workload: the shock tubes' own shells, else [1, 2]."""
    return DOMAINS.get(name, (1.0, 2.0))


class Problem:
    def __init__(self, name, gamma=None, noise=0.0, v0=(0.5, 0.5, 0.5), B0=(0.0, 0.0, 0.0), delta=0.01):
        self.name = name
        if gamma is None:
            gamma = SHOCK_TUBES[name][0] if name in SHOCK_TUBES else GAMMA
        self.gamma = gamma
        self.noise = noise
        self.delta = delta
        self.v0 = np.asarray(v0, dtype=np.float64)
        self.B0 = np.asarray(B0, dtype=np.float64)
        if name == "blast":
            self.B0 = np.array([0.0, 0.0, 10.0 / np.sqrt(4.0 * np.pi)])
        elif name == "lowbeta":
            self.B0 = np.array([1.0, 1.0, 0.0]) * np.sqrt(2.0 * 0.1 / 0.01) / np.sqrt(2.0)

    # ------------------------------------------------------- shock tubes
    def _tube(self, x):
        """r, cos(theta), sin(theta), r_hat, phi_hat and the inside mask."""
        r = np.sqrt((x * x).sum(-1))
        rc = np.sqrt(x[..., 0] ** 2 + x[..., 1] ** 2)
        ct, st = x[..., 2] / r, rc / r
        rhat = x / r[..., None]
        phat = np.zeros(x.shape)
        safe = np.maximum(rc, 1e-300)
        phat[..., 0] = -x[..., 1] / safe
        phat[..., 1] = x[..., 0] / safe
        return r, ct, st, rhat, phat, r <= SHOCK_TUBES[self.name][1]

    def _tanh_weights(self, r):
        t = np.tanh((r - SHOCK_TUBES[self.name][1]) / self.delta)
        return 0.5 * (1.0 - t), 0.5 * (1.0 + t)

    def has_radial_flux(self):
        return self.name in SHOCK_TUBES and SHOCK_TUBES[self.name][6] != 0.0

    def radial_field(self, x):
        """B_r0 sin(theta) (4.5 / r)^2 along r_hat (divergence-free for r > 0)."""
        r, ct, st, rhat, _, _ = self._tube(x)
        return (SHOCK_TUBES[self.name][6] * st * (4.5 / r) ** 2)[..., None] * rhat

    def radial_face_flux(self, pts, wn):
        """pts (F, Q, 3) face points, wn (F, Q, 3) weight x area element along the
        face normal -> the flux of the radial field through each face (F,)."""
        return (self.radial_field(pts) * wn).sum(-1).sum(-1)

    # ---------------------------------------------------------------- fields
    def primitive(self, x):
        X, Y, Zc = x[..., 0], x[..., 1], x[..., 2]
        if self.name in ("smooth", "entropy"):
            rho = 1.0 + 0.1 * np.sin(2.0 * np.pi * (X + Y + Zc) / np.sqrt(3.0))
            p = np.ones_like(X)
            v = np.broadcast_to(self.v0, x.shape).copy()
        elif self.name in ("blast", "lowbeta"):
            rho = np.ones_like(X)
            r2 = X * X + Y * Y + (Zc - 1.5) ** 2
            pin = 100.0
            p = np.where(r2 < 0.01, pin, 0.1)
            v = np.zeros(x.shape)
        elif self.name in SHOCK_TUBES:
            _, _, _, rhat, _, inside = self._tube(x)
            L, R = SHOCK_TUBES[self.name][2], SHOCK_TUBES[self.name][3]
            rho = np.where(inside, L[0], R[0])
            p = np.where(inside, L[1], R[1])
            v = np.where(inside, L[2], R[2])[..., None] * rhat
        elif self.name == "uniform":
            rho = np.full(X.shape, 1.3)
            p = np.full(X.shape, 0.7)
            v = np.broadcast_to(self.v0, x.shape).copy()
        else:
            raise ValueError(self.name)
        return rho, v, p

    def vector_potential(self, x):
        if self.name == "smooth":
            A = np.empty(x.shape)
            A[..., 0] = 0.1 * np.sin(2.0 * np.pi * x[..., 2])
            A[..., 1] = 0.1 * np.sin(2.0 * np.pi * x[..., 0])
            A[..., 2] = 0.1 * np.sin(2.0 * np.pi * x[..., 1])
            return A
        if self.name in SHOCK_TUBES:
            r, ct, _, rhat, _, _ = self._tube(x)
            wL, wR = self._tanh_weights(r)
            _, _, _, _, bL, bR, _ = SHOCK_TUBES[self.name]
            return ((bL * wL + bR * wR) * r * ct)[..., None] * rhat
        return 0.5 * np.cross(np.broadcast_to(self.B0, x.shape), x)

    def magnetic(self, x):
        if self.name == "smooth":
            k = 2.0 * np.pi
            B = np.empty(x.shape)
            B[..., 0] = 0.1 * k * np.cos(k * x[..., 1])
            B[..., 1] = 0.1 * k * np.cos(k * x[..., 2])
            B[..., 2] = 0.1 * k * np.cos(k * x[..., 0])
            return B
        if self.name in SHOCK_TUBES:
            r, _, st, _, phat, _ = self._tube(x)
            wL, wR = self._tanh_weights(r)
            _, _, _, _, bL, bR, _ = SHOCK_TUBES[self.name]
            return ((bL * wL + bR * wR) * st)[..., None] * phat + self.radial_field(x)
        return np.broadcast_to(self.B0, x.shape).copy()

    def conserved_at(self, x):
        rho, v, p = self.primitive(x)
        B = self.magnetic(x)
        U = np.empty(x.shape[:-1] + (8,))
        U[..., 0] = rho
        U[..., 1:4] = rho[..., None] * v
        U[..., 4] = p / (self.gamma - 1.0) + 0.5 * rho * (v * v).sum(-1) + 0.5 * (B * B).sum(-1)
        U[..., 5:8] = B
        return U

    # ----------------------------------------------------------- averaging
    def zone_averages(self, pts, wts):
        """pts (Z, G, 3) physical cubature points, wts (Z, G) physical weights
        (dV) -> zone-averaged conserved variables (Z, 8), with density noise."""
        U = np.einsum("zg,zgv->zv", wts, self.conserved_at(pts)) / wts.sum(1)[:, None]
        if self.noise:
            u = uniform_pm1(np.arange(U.shape[0]))
            fac = 1.0 + self.noise * u
            rho_old = U[:, 0].copy()
            kin_old = 0.5 * (U[:, 1:4] ** 2).sum(1) / rho_old
            U[:, 0] *= fac
            U[:, 1:4] *= fac[:, None]
            U[:, 4] += 0.5 * (U[:, 1:4] ** 2).sum(1) / U[:, 0] - kin_old
        return U

    def edge_circulation(self, pts, tw):
        """pts (E, S, 3) edge points, tw (E, S, 3) tangent x |dl| x weight ->
        line integral of A along each edge (E,)."""
        return (self.vector_potential(pts) * tw).sum(-1).sum(-1)


def make_problem(name, **kw):
    return Problem(name, **kw)
