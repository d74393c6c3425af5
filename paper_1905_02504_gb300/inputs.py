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


class Problem:
    def __init__(self, name, gamma=GAMMA, noise=0.0, v0=(0.5, 0.5, 0.5), B0=(0.0, 0.0, 0.0)):
        self.name = name
        self.gamma = gamma
        self.noise = noise
        self.v0 = np.asarray(v0, dtype=np.float64)
        self.B0 = np.asarray(B0, dtype=np.float64)
        if name == "blast":
            self.B0 = np.array([0.0, 0.0, 10.0 / np.sqrt(4.0 * np.pi)])
        elif name == "lowbeta":
            self.B0 = np.array([1.0, 1.0, 0.0]) * np.sqrt(2.0 * 0.1 / 0.01) / np.sqrt(2.0)

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
        return 0.5 * np.cross(np.broadcast_to(self.B0, x.shape), x)

    def magnetic(self, x):
        if self.name == "smooth":
            k = 2.0 * np.pi
            B = np.empty(x.shape)
            B[..., 0] = 0.1 * k * np.cos(k * x[..., 1])
            B[..., 1] = 0.1 * k * np.cos(k * x[..., 2])
            B[..., 2] = 0.1 * k * np.cos(k * x[..., 0])
            return B
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
