"""The ADER-CG predictor on the paper's prism zones (geo_prism_predictor) against
the oracle's predictor run on its prism element (oracle/prism.py, oracle/ader.py):
frustums of the icosahedral geodesic mesh (oracle/geodesic.py) with a smooth MHD
state at the nodes, every level and node at relative L1 1e-12 per variable, a
ragged last block, and a uniform state kept to rounding."""
import numpy as np
import pytest

from conftest import gpu_available
from test_gpu_parity import rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")


def frustum_nodes(p, level=1, nr=3, r_in=1.0, r_out=1.5, zones=None):
    from oracle import geodesic as G
    from oracle import prism as PR
    v, t = G.geodesic_sphere(level)
    r = G.shell_radii(r_in, r_out, nr)
    X = [PR.FrustumZone(p, v[a], v[b], v[c], r[k], r[k + 1]).X[0] for a, b, c in t for k in range(nr)]
    X = np.array(X)
    return X if zones is None else X[:zones]


def smooth_state(X, g):
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    rho = 1.0 + 0.2 * np.sin(2.0 * x + y) * np.cos(z)
    v = np.stack([0.3 + 0.1 * np.cos(y), -0.2 + 0.1 * np.sin(z), 0.1 * np.cos(x)], -1)
    B = np.stack([0.4 + 0.05 * y, -0.3 + 0.05 * z, 0.2 + 0.05 * x], -1)
    p = 0.8 + 0.1 * np.cos(x - z)
    U = np.zeros(X.shape[:-1] + (8,))
    U[..., 0] = rho
    U[..., 1:4] = rho[..., None] * v
    U[..., 4] = p / (g - 1) + 0.5 * rho * (v * v).sum(-1) + 0.5 * (B * B).sum(-1)
    U[..., 5:8] = B
    return U


def run_gpu(p, X, U, dt, g):
    import torch
    from paper_1905_02504_gb300 import geomhd
    Z, N = X.shape[:2]
    Xd = torch.from_numpy(np.ascontiguousarray(X.transpose(2, 1, 0))).cuda()      # [3][N][Z]
    Ud = torch.from_numpy(np.ascontiguousarray(U.transpose(2, 1, 0))).cuda()      # [8][N][Z]
    Uh = torch.full((p, 8, N, Z), float("nan"), dtype=torch.float64, device="cuda")
    geomhd.geo_prism_predictor(p, Xd, Ud, dt, g, Uh)
    torch.cuda.synchronize()
    return Uh.cpu().numpy().transpose(3, 0, 2, 1)                                # (Z, M, N, 8)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_prism_predictor_matches_oracle(p):
    from oracle import prism as PR
    from oracle.ader import AderPredictor
    g = 5.0 / 3.0
    X = frustum_nodes(p, zones=237)          # 237 zones: not a multiple of any block's zone count
    U = smooth_state(X, g)
    dt = 0.01
    ad = AderPredictor(PR.FrustumZone(p, X=X[0]), X, g)
    ref = ad.predict(U, dt)
    got = run_gpu(p, X, U, dt, g)
    assert np.isfinite(got).all()
    for v in range(8):
        assert rel_l1(got[..., v], ref[..., v]) < 1e-12, (v, rel_l1(got[..., v], ref[..., v]))
    # the levels really evolved (the space-time solution is not level 1 repeated)
    assert rel_l1(ref[:, -1, :, 0], ref[:, 0, :, 0]) > 1e-6


@pytest.mark.parametrize("p", [2, 3, 4])
def test_prism_predictor_keeps_a_uniform_state(p):
    g = 5.0 / 3.0
    X = frustum_nodes(p, level=2, nr=2)
    U0 = np.array([1.2, 0.3, -0.1, 0.2, 3.0, 0.4, 0.1, -0.3])
    U = np.broadcast_to(U0, X.shape[:2] + (8,)).copy()
    got = run_gpu(p, X, U, 0.02, g)
    from oracle import prism as PR
    from oracle.ader import AderPredictor
    J = AderPredictor(PR.FrustumZone(p, X=X[0]), X, g).J          # (Z, N)
    assert np.abs(got / J[:, None, :, None] - U0).max() < 1e-13 * np.abs(U0).max()


def test_prism_predictor_refuses_bad_arguments():
    import torch
    from paper_1905_02504_gb300 import geomhd
    X = torch.zeros((3, 6, 4), dtype=torch.float64, device="cuda")
    U = torch.zeros((8, 6, 4), dtype=torch.float64, device="cuda")
    Uh = torch.zeros((2, 8, 6, 4), dtype=torch.float64, device="cuda")
    for order, dt, gam in ((5, 0.1, 1.4), (2, 0.0, 1.4), (2, 0.1, 1.0)):
        with pytest.raises(geomhd.GeoError):
            geomhd.geo_prism_predictor(order, X, U, dt, gam, Uh)
