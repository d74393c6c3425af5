"""The physical-state flag of the U update (rho > 0, p > 0, finite energy):
geo_check_state reads and clears it, and a geo_step after a flagged step (once
the flag's copy has landed on the host) refuses with GEO_ERR_NONPHYSICAL.
A negative density only produces negative or NaN values on the device (no fault)."""
import numpy as np
import pytest

from conftest import gpu_available
from test_gpu_parity import setup_case

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")


def test_physical_state_flag():
    import torch
    from paper_1905_02504_gb300 import geomhd
    o, m, U, phi = setup_case(4, 3, 2)
    dt = m.cfl_dt(0.4)
    m.step(dt)
    assert geomhd.geo_check_state(m.h) == 0
    # zone 7 with a negative density (one step of inflow cannot restore it; a
    # negative pressure alone can be cured by the neighbours' energy inflow)
    bad = U.copy()
    bad[7, 0] = -bad[7, 0]
    m.upload(np.ascontiguousarray(bad.T), phi.copy())
    m.step(dt)
    with pytest.raises(geomhd.GeoError) as e:
        geomhd.geo_check_state(m.h)
    assert e.value.code == geomhd.GEO_ERR_NONPHYSICAL
    assert geomhd.geo_check_state(m.h) == 0          # cleared by the check
    # the delayed report of geo_step itself
    m.upload(np.ascontiguousarray(bad.T), phi.copy())
    m.step(dt)
    torch.cuda.synchronize()
    with pytest.raises(geomhd.GeoError) as e:
        m.step(dt)
    assert e.value.code == geomhd.GEO_ERR_NONPHYSICAL
    # a fresh upload clears the flag
    m.upload(np.ascontiguousarray(U.T), phi.copy())
    m.step(dt)
    m.step(dt)
    assert geomhd.geo_check_state(m.h) == 0
    m.close()
