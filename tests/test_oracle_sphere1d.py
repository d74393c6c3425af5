"""Pins of the one-dimensional spherical reference solver (Sec. VIII.c) used to
judge the three-dimensional spherical Sod run."""
import numpy as np

from oracle import sphere1d

SOD_L, SOD_R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)


def _sod(r0):
    return (lambda r: np.where(r <= r0, 1.0, 0.125), lambda r: np.zeros_like(r),
            lambda r: np.where(r <= r0, 1.0, 0.1))


def test_planar_limit_matches_exact_riemann_solution():
    """On a thin shell far from the origin the spherical terms vanish and the
    solution is the planar Sod problem (Toro's exact solution); the L1 error of
    the density falls under refinement (first order at the discontinuities)."""
    errs = []
    for n in (200, 800):
        rf, (rho, v, p) = sphere1d.radial_solve(1000.0, 1001.0, n, *_sod(1000.5), 0.2, 1.4)
        rc = 0.5 * (rf[1:] + rf[:-1])
        ex = sphere1d.exact_riemann((rc - 1000.5) / 0.2, SOD_L, SOD_R, 1.4)
        errs.append(np.abs(rho - ex[0]).mean())
        assert np.abs(v - ex[1]).mean() < 0.05 and np.abs(p - ex[2]).mean() < 0.02
    assert errs[1] < 0.006 and errs[1] < errs[0] / 2.0, errs


def test_exact_riemann_star_state():
    """Sod's star state (Toro, Table 4.2, test 1): p* = 0.30313, u* = 0.92745."""
    ex = sphere1d.exact_riemann(np.array([0.9]), SOD_L, SOD_R, 1.4)
    assert abs(ex[2][0] - 0.30313) < 1e-4 and abs(ex[1][0] - 0.92745) < 1e-4


def test_spherical_sod_conserves_mass_and_energy():
    """Before any wave reaches r = 2 or r = 3 the radial fluxes telescope: the
    volume integrals of rho and E stay fixed to rounding."""
    g = 1.4
    n = 400
    rho0, v0, p0 = _sod(2.5)
    rf = np.linspace(2.0, 3.0, n + 1)
    V = (rf[1:] ** 3 - rf[:-1] ** 3) / 3.0
    rc = 0.5 * (rf[1:] + rf[:-1])
    m0 = (rho0(rc) * V).sum()
    e0 = (p0(rc) / (g - 1.0) * V).sum()
    _, (rho, v, p) = sphere1d.radial_solve(2.0, 3.0, n, rho0, v0, p0, 0.15, g)
    assert abs((rho * V).sum() / m0 - 1.0) < 1e-13
    E = p / (g - 1.0) + 0.5 * rho * v * v
    assert abs((E * V).sum() / e0 - 1.0) < 1e-13


def test_uniform_state_stays_at_rest():
    _, (rho, v, p) = sphere1d.radial_solve(2.0, 3.0, 100, lambda r: np.ones_like(r),
                                           lambda r: np.zeros_like(r), lambda r: np.full_like(r, 0.7), 0.1, 1.4)
    assert np.abs(v).max() < 1e-14 and np.abs(p - 0.7).max() < 1e-14 and np.abs(rho - 1.0).max() < 1e-14
