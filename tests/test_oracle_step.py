"""Pins of the oracle's full step (Sec. VI): free-stream preservation, discrete div B,
conservation with the boundary-flux ledger, and (opt-in, slow) the design order."""
import os

import numpy as np
import pytest

from oracle.step import Oracle
from paper_1905_02504_gb300.inputs import make_problem


@pytest.fixture(scope="module", params=[2, 3, 4])
def orc(request):
    return Oracle(3, 3, 1.0, 2.0, request.param)


def test_free_stream_preserved(orc):
    pr = make_problem("uniform", v0=(0.4, -0.3, 0.2), B0=(0.3, -0.2, 0.5))
    U, phi = orc.initial_state(pr)
    dt = orc.cfl_dt(U, 0.3)
    U1, phi1 = U, phi
    for _ in range(2):
        U1, phi1 = orc.step(U1, phi1, dt)
    # rounding only: order 4 performs several times the operations of order 2 per
    # zone (32 nodes, 4 time levels, 10 flux evaluations), hence its wider bound
    tol = 1e-14 if orc.mesh.p < 4 else 4e-14
    assert (np.abs(U1 - U).max(0) / np.abs(U).max(0)).max() < tol
    assert np.abs(phi1 - phi).max() < tol * np.abs(phi).max()


def test_divb_and_conservation_ledger(orc):
    U, phi = orc.initial_state(make_problem("smooth"))
    a0, r0 = orc.divB(phi)
    assert r0 < 1e-14
    dt = orc.cfl_dt(U, 0.4)
    m = orc.mesh
    V = orc.V
    for _ in range(2):
        U1, phi1, st = orc.step(U, phi, dt, return_stages=True)
        F = st["Fface"]
        inner = np.arange(m.ncol) * (m.nr + 1)
        outer = inner + m.nr
        ledger = F[inner].sum(0) - F[outer].sum(0)
        # the zone B is overwritten by the divergence-free means before the update
        Ustart = U.copy()
        Ustart[:, 5:8] = st["Bmean"]
        change = (V[:, None] * (U1 - Ustart)).sum(0)
        scale = (V[:, None] * np.abs(U1)).sum(0)
        assert (np.abs(change - ledger) / scale).max() < 1e-13
        U, phi = U1, phi1
        assert orc.divB(phi)[1] < 1e-13


@pytest.mark.skipif(not os.environ.get("GEOMHD_SLOW"), reason="set GEOMHD_SLOW=1 (several minutes)")
def test_design_order_entropy_wave():
    """Exact advected entropy wave with a uniform field: L1 error of rho over the
    shells r in (1.3, 1.7) at t = 0.1 drops at the design order 2 between 8 and 16
    columns per cube-face edge."""
    errs = []
    T = 0.1
    for n in (8, 16):
        o = Oracle(n, n, 1.0, 2.0, 2)
        pr = make_problem("entropy", v0=(0.5, 0.5, 0.5), B0=(0.2, 0.1, -0.1))
        U, phi = o.initial_state(pr)
        nst = int(np.ceil(T / (0.4 / n)))
        for _ in range(nst):
            U, phi = o.step(U, phi, T / nst)
        g = o.weno.geo0
        ex = np.einsum("zg,zg->z", g["dV"], pr.primitive(g["xg"] - T * 0.5)[0]) / g["V"]
        r = np.linalg.norm(g["xc"], axis=1)
        mask = (r > 1.3) & (r < 1.7)
        errs.append(np.sum(np.abs(U[:, 0] - ex)[mask] * g["V"][mask]) / np.sum(g["V"][mask]))
    assert np.log2(errs[0] / errs[1]) > 1.8
