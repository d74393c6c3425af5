"""Reference solutions for the spherical Sod problem (Sec. VIII.c) -- oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. VIII.c compares the three-dimensional spherical Sod run with "the analytical
result for the spherical Riemann problem", a one-dimensional spherically
symmetric solution.  This module computes such a solution of the radial Euler
equations
    d/dt (r^2 U) + d/dr (r^2 F(U)) = (0, 2 r p, 0),   U = (rho, rho v, E),
by a plain second-order finite-volume method on a fine radial grid: cells
[r_{i-1/2}, r_{i+1/2}] with volumes (r_{i+1/2}^3 - r_{i-1/2}^3)/3 and face areas
r^2, minmod-limited linear reconstruction of the primitive variables, HLL
fluxes with Davis wave speeds, the pressure source p (A_{i+1/2} - A_{i-1/2}) / V_i
(which balances a uniform pressure exactly), Heun's method in time, and
continuative (copied) boundary cells.

exact_riemann() is the textbook exact solution of the planar Riemann problem for
an ideal gas (Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics,
ch. 4: Newton iteration for the star pressure, then the self-similar sampling).

Pinned by: tests/test_oracle_sphere1d.py -- on a thin shell far from the origin
(r in [1000, 1001]) the radial solver reproduces the exact planar Sod solution
to its discretisation error, converging under refinement; mass and energy are
conserved up to the boundary fluxes; a uniform state at rest stays at rest.
"""
import numpy as np


def _prim(U, g):
    rho = U[0]
    v = U[1] / rho
    p = (g - 1.0) * (U[2] - 0.5 * rho * v * v)
    return rho, v, p


def _hll(rL, vL, pL, rR, vR, pR, g):
    def flux(r, v, p):
        E = p / (g - 1.0) + 0.5 * r * v * v
        return np.stack([r * v, r * v * v + p, (E + p) * v]), np.stack([r, r * v, E])
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    sL = np.minimum(vL - cL, vR - cR)
    sR = np.maximum(vL + cL, vR + cR)
    FL, UL = flux(rL, vL, pL)
    FR, UR = flux(rR, vR, pR)
    Fm = (sR * FL - sL * FR + sL * sR * (UR - UL)) / (sR - sL)
    return np.where(sL >= 0.0, FL, np.where(sR <= 0.0, FR, Fm))


def _minmod(a, b):
    return np.where(a * b > 0.0, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)


def radial_solve(r_in, r_out, ncell, rho0, v0, p0, t_end, gamma, cfl=0.4):
    """Cell averages (rho, v, p) at t_end on ncell equal cells of [r_in, r_out];
    rho0, v0, p0: functions of the cell-centre radius."""
    rf = np.linspace(r_in, r_out, ncell + 1)
    rc = 0.5 * (rf[1:] + rf[:-1])
    A = rf * rf
    V = (rf[1:] ** 3 - rf[:-1] ** 3) / 3.0
    g = gamma
    rho, v, p = rho0(rc), v0(rc), p0(rc)
    U = np.stack([rho, rho * v, p / (g - 1.0) + 0.5 * rho * v * v])

    def rhs(U):
        r, u, pp = _prim(U, g)
        W = np.stack([r, u, pp])
        We = np.concatenate([W[:, :1], W, W[:, -1:]], axis=1)          # continuative ghosts
        dW = _minmod(We[:, 1:-1] - We[:, :-2], We[:, 2:] - We[:, 1:-1])
        WL = W + 0.5 * dW                                             # right face of each cell
        WR = W - 0.5 * dW                                             # left face of each cell
        WLe = np.concatenate([WR[:, :1], WL], axis=1)                 # left state at every face
        WRe = np.concatenate([WR, WL[:, -1:]], axis=1)                # right state at every face
        F = _hll(WLe[0], WLe[1], WLe[2], WRe[0], WRe[1], WRe[2], g)
        AF = A[None, :] * F
        out = -(AF[:, 1:] - AF[:, :-1]) / V[None, :]
        out[1] += pp * (A[1:] - A[:-1]) / V
        return out

    t = 0.0
    dr = rf[1] - rf[0]
    while t < t_end:
        r, u, pp = _prim(U, g)
        dt = cfl * dr / np.max(np.abs(u) + np.sqrt(g * pp / r))
        dt = min(dt, t_end - t)
        U1 = U + dt * rhs(U)
        U = 0.5 * (U + U1 + dt * rhs(U1))
        t += dt
    return rf, _prim(U, g)


def exact_riemann(xi, left, right, gamma):
    """Exact planar Riemann solution (rho, v, p) at similarity coordinates
    xi = (x - x0) / t for left / right states (rho, v, p)."""
    g = gamma
    rL, uL, pL = left
    rR, uR, pR = right
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)

    def fk(p, rk, pk, ck):
        if p > pk:
            A, B = 2.0 / ((g + 1.0) * rk), (g - 1.0) / (g + 1.0) * pk
            f = (p - pk) * np.sqrt(A / (p + B))
            df = np.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pk) / (B + p))
        else:
            f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
            df = 1.0 / (rk * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
        return f, df

    p = 0.5 * (pL + pR)
    for _ in range(100):
        f1, d1 = fk(p, rL, pL, cL)
        f2, d2 = fk(p, rR, pR, cR)
        dp = (f1 + f2 + uR - uL) / (d1 + d2)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-14 * p:
            break
    f1, _ = fk(p, rL, pL, cL)
    f2, _ = fk(p, rR, pR, cR)
    us = 0.5 * (uL + uR) + 0.5 * (f2 - f1)
    out = np.empty((3,) + np.shape(xi))
    for n, s in np.ndenumerate(np.asarray(xi)):
        if s <= us:   # left of the contact
            if p > pL:
                rs = rL * ((p / pL + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pL + 1))
                sh = uL - cL * np.sqrt((g + 1) / (2 * g) * p / pL + (g - 1) / (2 * g))
                val = (rL, uL, pL) if s < sh else (rs, us, p)
            else:
                rs = rL * (p / pL) ** (1.0 / g)
                cs = cL * (p / pL) ** ((g - 1) / (2 * g))
                if s < uL - cL:
                    val = (rL, uL, pL)
                elif s > us - cs:
                    val = (rs, us, p)
                else:
                    c = 2.0 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    val = (rL * (c / cL) ** (2 / (g - 1)), 2.0 / (g + 1) * (cL + (g - 1) / 2 * uL + s),
                           pL * (c / cL) ** (2 * g / (g - 1)))
        else:          # right of the contact
            if p > pR:
                rs = rR * ((p / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pR + 1))
                sh = uR + cR * np.sqrt((g + 1) / (2 * g) * p / pR + (g - 1) / (2 * g))
                val = (rR, uR, pR) if s > sh else (rs, us, p)
            else:
                rs = rR * (p / pR) ** (1.0 / g)
                cs = cR * (p / pR) ** ((g - 1) / (2 * g))
                if s > uR + cR:
                    val = (rR, uR, pR)
                elif s < us + cs:
                    val = (rs, us, p)
                else:
                    c = 2.0 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    val = (rR * (c / cR) ** (2 / (g - 1)), 2.0 / (g + 1) * (-cR + (g - 1) / 2 * uR + s),
                           pR * (c / cR) ** (2 * g / (g - 1)))
        out[(slice(None),) + n] = val
    return out
