"""The allocation-free CFL entry point agrees with geo_cfl_dt.

geo_cfl_dt_noalloc exists for callers that cannot allocate device memory when
they need a time step (a memory pool owned by someone else, no device
synchronisation allowed, externally managed buffers).  It keeps its scratch in a
fixed device array and writes into a caller-owned device buffer.  This file is
collected last so that a failure here never hides the other GPU tests.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = pytest.mark.gpu


@pytest.mark.skipif(not gpu_available(), reason="no CUDA device")
def test_noalloc_cfl_matches_allocating_entry_point_twice():
    import torch
    from paper_1905_02504_gb300 import geomhd
    from paper_1905_02504_gb300.inputs import make_problem

    m = geomhd.Mesh(5, 3, 1.0, 2.0, 2)
    U, phi = m.initial_state(make_problem("smooth"))
    m.upload(U, phi)
    dt_ref = m.cfl_dt(0.4)
    U_dev = torch.from_numpy(U).cuda()
    for _ in range(2):                                   # two calls in a row share the scratch
        dt_dev = torch.full((1,), -7.0, dtype=torch.float64, device="cuda")
        geomhd.geo_cfl_dt_noalloc(m.h, U_dev, 0.4, dt_dev)
        torch.cuda.synchronize()
        dt = dt_dev.item()
        assert abs(dt - dt_ref) <= 1e-13 * dt_ref, (dt, dt_ref)
    # a second, different state through the same scratch
    U2 = U.copy()
    U2[1] *= 3.0                                         # faster flow -> smaller dt
    U2[4] += 0.5 * (U2[1] ** 2 - U[1] ** 2) / U2[0]
    m.upload(U2, phi)
    dt_ref2 = m.cfl_dt(0.4)
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    geomhd.geo_cfl_dt_noalloc(m.h, torch.from_numpy(U2).cuda(), 0.4, dt_dev)
    torch.cuda.synchronize()
    assert dt_ref2 < dt_ref
    assert abs(dt_dev.item() - dt_ref2) <= 1e-13 * dt_ref2
    m.close()
