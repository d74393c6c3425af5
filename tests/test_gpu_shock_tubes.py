"""The spherical shock tubes of Sec. VIII.c on the GPU path (FP64).

* Spherical Sod, r in [2, 3], t = 0.2: the cubed-sphere solution, averaged over
  each radial shell, against the one-dimensional spherically symmetric reference
  (oracle/sphere1d.py, 4000 cells) averaged over the same shells; the spread of
  the zones of a shell measures how well the mesh keeps the spherical symmetry.
* Spherical Brio-Wu (t = 0.1) and Ryu-Jones (t = 0.06): the tanh-tapered toroidal
  field from A_r and the r^-2 radial field from its face fluxes; the state stays
  physical and div B stays at rounding.  The paper shows these two only as
  figures, so no profile is compared.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")


def run(name, n, nr, p, t_end, positivity=False, cfl=0.4):
    from paper_1905_02504_gb300 import geomhd
    from paper_1905_02504_gb300.inputs import domain, make_problem
    r_in, r_out = domain(name)
    pr = make_problem(name, delta=0.5 * (r_out - r_in) / nr)
    m = geomhd.Mesh(n, nr, r_in, r_out, p, gamma=pr.gamma)
    if positivity:
        geomhd.geo_set_positivity(m.h, 1)
    U0, phi0 = m.initial_state(pr)
    m.upload(U0, phi0)
    t, steps = 0.0, 0
    while t < t_end - 1e-14:
        dt = min(m.cfl_dt(cfl), t_end - t)
        m.step(dt)
        t += dt
        steps += 1
    U, phi = m.download()
    _, rdiv = m.divB()
    return m, U, phi, rdiv, steps


def test_spherical_sod_matches_radial_reference():
    from oracle import sphere1d
    from paper_1905_02504_gb300 import geomhd
    n, nr = 12, 64
    m, U, phi, rdiv, steps = run("sod", n, nr, 3, 0.2)
    assert np.isfinite(U).all() and rdiv < 1e-13
    xc, vol = geomhd.geo_zone_geometry(m.h)
    k = np.arange(m.Z) % nr
    rho3 = np.bincount(k, U[0] * vol, nr) / np.bincount(k, vol, nr)
    spread = np.array([np.ptp(U[0][k == s]) for s in range(nr)])
    # reference on 4000 equal cells, averaged over each log-ratioed shell
    rf, (rho1, _, _) = sphere1d.radial_solve(2.0, 3.0, 4000, lambda r: np.where(r <= 2.5, 1.0, 0.125),
                                            lambda r: np.zeros_like(r), lambda r: np.where(r <= 2.5, 1.0, 0.1),
                                            0.2, 1.4)
    v1 = (rf[1:] ** 3 - rf[:-1] ** 3) / 3.0
    rc1 = 0.5 * (rf[1:] + rf[:-1])
    shells = 2.0 * 1.5 ** (np.arange(nr + 1) / nr)
    sid = np.clip(np.searchsorted(shells, rc1) - 1, 0, nr - 1)
    ref = np.bincount(sid, rho1 * v1, nr) / np.bincount(sid, v1, nr)
    err = np.abs(rho3 - ref)
    print("spherical Sod: %d steps, mean |rho - ref| %.3e, max %.3e, max shell spread %.3e"
          % (steps, err.mean(), err.max(), spread.max()))
    assert err.mean() < 0.02 and spread.max() < 0.05, (err.mean(), err.max(), spread.max())
    m.close()


# both with the positivity scaling (without it the order-3 Brio-Wu run on this
# coarse mesh reaches a negative pressure; the paper's flattener is not built)
@pytest.mark.parametrize("name,t_end,positivity", [("briowu", 0.1, True), ("ryujones", 0.06, True)])
def test_mhd_shock_tubes_stay_physical_and_divergence_free(name, t_end, positivity):
    from paper_1905_02504_gb300 import geomhd
    m, U, phi, rdiv, steps = run(name, 8, 48, 3, t_end, positivity=positivity)
    assert np.isfinite(U).all() and np.isfinite(phi).all()
    assert geomhd.geo_check_state(m.h) == 0
    assert rdiv < 1e-13, rdiv
    print("%s: %d steps, rho in [%.3f, %.3f], div B %.2e" % (name, steps, U[0].min(), U[0].max(), rdiv))
    m.close()
