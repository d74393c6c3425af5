"""The benchmark's own workload, 6x64x64 x 64 shells (1,572,864 zones) at order 4
in the launch configuration `bench.py` times (default predictor schedule, FP64
and FP32-bulk), checked through properties that hold at any size: a uniform
state stays uniform (free stream on the curved zones, Sec. V's metric
identities), the CT update keeps div B at rounding (Sec. VI), and the FP32-bulk
form stays within its error bound of the FP64 form on the smooth test.  The
oracle itself is compared element by element on the smaller meshes of
test_gpu_parity.py."""
import numpy as np
import pytest

from conftest import gpu_available
from test_gpu_parity import rel_l1

pytestmark = pytest.mark.gpu

N, NR, P = 64, 64, 4


@pytest.fixture(autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("form,tol", [("fp64", 1e-11), ("fp32", 2e-6)])
def test_full_size_free_stream(form, tol):
    from paper_1905_02504_gb300 import geomhd
    from paper_1905_02504_gb300.inputs import make_problem
    prec = geomhd.GEO_FP64 if form == "fp64" else geomhd.GEO_FP32_BULK
    m = geomhd.Mesh(N, NR, 1.0, 2.0, P, prec=prec)
    U, phi = m.initial_state(make_problem("uniform", B0=(0.3, -0.2, 0.5)))
    m.upload(U, phi)
    dt = m.cfl_dt(0.4)
    for _ in range(2):
        m.step(dt)
    Ug, pg = m.download()
    dev = np.abs(Ug - U).max(axis=1) / np.abs(U).max(axis=1)
    assert dev.max() < tol, dev
    assert np.abs(pg - phi).max() < tol * np.abs(phi).max()
    assert m.divB()[1] < 1e-13
    m.close()


def test_full_size_fp32_bulk_within_bound_of_fp64():
    from paper_1905_02504_gb300 import geomhd
    from paper_1905_02504_gb300.inputs import make_problem
    out = {}
    for form, prec in (("fp64", geomhd.GEO_FP64), ("fp32", geomhd.GEO_FP32_BULK)):
        m = geomhd.Mesh(N, NR, 1.0, 2.0, P, prec=prec)
        U, phi = m.initial_state(make_problem("smooth"))
        m.upload(U, phi)
        dt = 0.5 * m.cfl_dt(0.4) if form == "fp64" else out["dt"]
        out["dt"] = dt
        for _ in range(3):
            m.step(dt)
        out[form] = m.download()
        out[form + "_divb"] = m.divB()[1]
        m.close()
    (U64, p64), (U32, p32) = out["fp64"], out["fp32"]
    for v in range(8):
        assert rel_l1(U32[v], U64[v]) < 2e-5, v
    assert rel_l1(p32, p64) < 2e-5
    assert out["fp64_divb"] < 1e-13 and out["fp32_divb"] < 1e-13
    assert np.isfinite(U64).all()
