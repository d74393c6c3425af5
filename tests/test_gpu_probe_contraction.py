"""The contraction probe (geo_probe_contraction): the predictor's derivative
contraction of Eq. C.34 alone, in the CUDA-core form of the variable-team
predictor and in the tensor-core (TF32, three-pass) form, against the oracle
element's D^alpha applied in FP64 to the same hashed operands.  The probe is a
measurement aid; this test makes sure both timed forms compute the contraction
(every zone, every node, a ragged last block)."""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")


def hashed_f(z, N):
    """F[z, alpha, v, j] of the probe's documented hash, (h mod 2^16) / 2^16 - 1/2."""
    zz = (np.arange(z, dtype=np.uint64) * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)
    al = np.arange(3, dtype=np.uint64) * np.uint64(73856093) & np.uint64(0xFFFFFFFF)
    v = np.arange(8, dtype=np.uint64) * np.uint64(19349663) & np.uint64(0xFFFFFFFF)
    j = np.arange(N, dtype=np.uint64) * np.uint64(83492791) & np.uint64(0xFFFFFFFF)
    h = zz[:, None, None, None] ^ al[None, :, None, None] ^ v[None, None, :, None] ^ j[None, None, None, :]
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(0x5BD1E995)) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(15)
    return (h & np.uint64(0xFFFF)).astype(np.float64) / 65536.0 - 0.5


@pytest.mark.parametrize("p", [2, 3, 4])
def test_probe_forms_compute_the_contraction(p):
    import torch
    from oracle import refelem
    from paper_1905_02504_gb300 import geomhd
    el = refelem.HexElement(p)
    N = el.N
    Z = 1237                                              # not a multiple of any block's zones
    F = hashed_f(Z, N)                                    # [z][alpha][v][j]
    ref = np.einsum("aij,zavj->zvi", el.D, F)             # [z][v][i]
    scale = np.abs(ref).max()
    m = geomhd.Mesh(3, 5, 1.0, 2.0, p, prec=geomhd.GEO_FP32_BULK)    # order 4 needs nr >= 3
    for tensor in (0, 1):
        out = torch.full((Z, 8, N), float("nan"), dtype=torch.float32, device="cuda")
        ms = geomhd.geo_probe_contraction(m.h, tensor, Z, 3, out)
        got = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all(), tensor
        assert np.abs(got - ref).max() <= 1e-5 * scale, (tensor, np.abs(got - ref).max() / scale)
        assert ms > 0.0
    with pytest.raises(geomhd.GeoError):
        geomhd.geo_probe_contraction(m.h, 2, Z, 1, out)
    m.close()


def test_probe_needs_fp32_mesh():
    import torch
    from paper_1905_02504_gb300 import geomhd
    m = geomhd.Mesh(2, 2, 1.0, 2.0, 3)
    out = torch.empty(8 * 20, dtype=torch.float32, device="cuda")
    with pytest.raises(geomhd.GeoError):
        geomhd.geo_probe_contraction(m.h, 0, 1, 1, out)
    m.close()
