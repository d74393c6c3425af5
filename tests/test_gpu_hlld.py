"""The HLLD face solver (geo_set_riemann) against the oracle's HLLD step: face
fluxes and the updated state over several steps at relative L1 1e-12 (FP64), the
FP32-bulk form within its 2e-5 bound, div B at rounding, and the adjoint's
refusal (its reverse sweep differentiates HLL only)."""
import numpy as np
import pytest

from conftest import gpu_available
from test_gpu_parity import RTOL, rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")


def hlld_case(n, nr, p, prec=None, problem="blast"):
    from oracle.step import Oracle
    from paper_1905_02504_gb300 import geomhd
    from paper_1905_02504_gb300.inputs import make_problem
    o = Oracle(n, nr, 1.0, 2.0, p, riemann="hlld")
    U, phi = o.initial_state(make_problem(problem))
    m = geomhd.Mesh(n, nr, 1.0, 2.0, p, prec=geomhd.GEO_FP64 if prec is None else prec)
    geomhd.geo_set_riemann(m.h, geomhd.GEO_RIEMANN_HLLD)
    m.upload(np.ascontiguousarray(U.T), phi.copy())
    return o, m, U, phi


@pytest.mark.parametrize("n,nr,p,steps", [(5, 3, 2, 4), (4, 4, 3, 3), (3, 5, 4, 2)])
def test_hlld_step_matches_oracle(n, nr, p, steps):
    """On the smooth problem (the blast at rest has mostly rounding-level face
    fluxes, whose relative L1 is noise)."""
    from paper_1905_02504_gb300 import geomhd
    o, m, U, phi = hlld_case(n, nr, p, problem="smooth")
    dt = o.cfl_dt(U, 0.4)
    U1, phi1, st = o.step(U, phi, dt, return_stages=True)
    m.step(dt)
    Ff = geomhd.geo_debug_buffer(m.h, 4, 8 * m.F).reshape(8, m.F)
    for v in range(8):
        assert rel_l1(Ff[v], st["Fface"][:, v]) < RTOL, ("face flux", v)
    Uo, po = U1, phi1
    for _ in range(steps - 1):
        Uo, po = o.step(Uo, po, dt)
        m.step(dt)
    Ug, pg = m.download()
    for v in range(8):
        assert rel_l1(Ug[v], Uo[:, v]) < RTOL, ("U", v, rel_l1(Ug[v], Uo[:, v]))
    assert rel_l1(pg, po) < RTOL
    assert m.divB()[1] < 1e-13
    # HLLD is not HLL on this state
    from oracle.physics import hll
    o.riemann = hll
    U_hll, _ = o.step(U, phi, dt)
    assert rel_l1(U_hll[:, 0], U1[:, 0]) > 1e-8
    m.close()


def test_hlld_fp32_bulk_within_bound():
    from paper_1905_02504_gb300 import geomhd
    o, m, U, phi = hlld_case(4, 4, 3, prec=geomhd.GEO_FP32_BULK, problem="smooth")
    dt = o.cfl_dt(U, 0.4)
    Uo, po = U, phi
    for _ in range(3):
        Uo, po = o.step(Uo, po, dt)
        m.step(dt)
    Ug, pg = m.download()
    for v in range(8):
        assert rel_l1(Ug[v], Uo[:, v]) < 2e-5, v
    assert m.divB()[1] < 1e-13
    m.close()


def test_adjoint_refuses_hlld():
    import torch
    from paper_1905_02504_gb300 import geomhd
    o, m, U, phi = hlld_case(3, 3, 3, problem="smooth")
    Ut = torch.from_numpy(np.ascontiguousarray(U.T)).cuda()
    pt = torch.from_numpy(phi.copy()).cuda()
    with pytest.raises(geomhd.GeoError) as e:
        geomhd.geo_step_adjoint(m.h, 1e-3, Ut, pt, Ut, pt, torch.empty_like(Ut), torch.empty_like(pt))
    assert e.value.code == -1
    m.close()
