"""GPU path vs the FP64 oracle, stage by stage and over several full steps.

Both sides start from the same seeded state (the oracle's zone averages and
edge-circulation face fluxes); the GPU runs through the C ABI.  Tolerance: the
per-variable relative L1 of 1e-12 required for the FP64 form, on meshes that
span several thread blocks and end in a ragged tail.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def rel_l1(a, b, axis=None):
    num = np.abs(a - b).sum(axis=axis)
    den = np.abs(b).sum(axis=axis)
    return num / np.maximum(den, 1e-300)


_CACHE = {}


def setup_case(n, nr, p, problem="smooth", schedule=None):
    from oracle.step import Oracle
    from paper_1905_02504_gb300 import geomhd
    from paper_1905_02504_gb300.inputs import make_problem
    key = (n, nr, p)
    if key not in _CACHE:
        _CACHE[key] = Oracle(n, nr, 1.0, 2.0, p)
    o = _CACHE[key]
    pr = make_problem(problem) if problem != "uniform" else make_problem("uniform", B0=(0.3, -0.2, 0.5))
    U, phi = o.initial_state(pr)
    m = geomhd.Mesh(n, nr, 1.0, 2.0, p)
    if schedule is not None:
        geomhd.geo_set_predictor(m.h, schedule)
    assert (m.Z, m.F, m.E) == (o.mesh.Z, o.mesh.F, o.mesh.E)
    m.upload(np.ascontiguousarray(U.T), phi.copy())
    return o, m, U, phi


@pytest.fixture(autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")


# predictor: one thread per zone; a team of one thread per node; the team with the
# contraction and point evaluations in the variable layout
SCHEDULES = [0, 1, 2]
_STAGES = {}


def oracle_stages(o, key, U, phi, dt):
    if key not in _STAGES:
        _STAGES[key] = o.step(U, phi, dt, return_stages=True)
    return _STAGES[key]


# (5, 3, 3): 450 zones, not a multiple of the 8 zones of an order-3 node-team block
@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("n,nr,p", [(5, 3, 2), (4, 4, 3), (5, 3, 3), (3, 5, 4)])
def test_stages_match_oracle(n, nr, p, schedule):
    from paper_1905_02504_gb300 import geomhd
    o, m, U, phi = setup_case(n, nr, p, schedule=schedule)
    dt = o.cfl_dt(U, 0.4)
    dt_gpu = m.cfl_dt(0.4)
    assert abs(dt_gpu - dt) <= 1e-13 * dt
    U1, phi1, st = oracle_stages(o, (n, nr, p), U, phi, dt)
    m.step(dt)
    Ug, phig = m.download()
    om = o.mesh
    Z, F, E = om.Z, om.F, om.E
    nc1 = o.weno.nc1
    # a1: WENO-AO coefficients
    W = geomhd.geo_debug_buffer(m.h, 0, 8 * nc1 * Z).reshape(8, nc1, Z)
    Wo = np.transpose(st["coeffs"], (1, 2, 0))
    for v in range(8):
        assert rel_l1(W[v], Wo[v]) < RTOL, ("weno", v, rel_l1(W[v], Wo[v]))
    # a2: nodal normal fields per face
    nqmax = max(o.dfb.nq)
    Bp = geomhd.geo_debug_buffer(m.h, 1, nqmax * F).reshape(nqmax, F)
    Bo = np.zeros((nqmax, F))
    mask = np.zeros((nqmax, F), bool)
    for f, b in st["bperp"].items():
        Bo[:len(b), f] = b
        mask[:len(b), f] = True
    assert rel_l1(Bp[mask], Bo[mask]) < RTOL
    # a3: predictor states at face points
    M = p
    nqt = sum(o.dfb.nq)
    trF = geomhd.geo_debug_buffer(m.h, 2, (M - 1) * nqt * 8 * Z).reshape(M - 1, nqt, 8, Z)
    tro = np.concatenate([o.ader.point_values(st["Uh"], o.face_ref[lf]) for lf in range(6)], axis=2)
    tro = np.transpose(tro[:, 1:], (1, 2, 3, 0))
    for v in range(8):
        assert rel_l1(trF[:, :, v], tro[:, :, v]) < RTOL, ("traces", v)
    # a4, a5: face fluxes and edge EMFs
    Ff = geomhd.geo_debug_buffer(m.h, 4, 8 * F).reshape(8, F)
    for v in range(8):
        assert rel_l1(Ff[v], st["Fface"][:, v]) < RTOL, ("face flux", v, rel_l1(Ff[v], st["Fface"][:, v]))
    Ee = geomhd.geo_debug_buffer(m.h, 5, E)
    assert rel_l1(Ee, st["Eedge"]) < RTOL
    # a6: updated state
    for v in range(8):
        assert rel_l1(Ug[v], U1[:, v]) < RTOL, ("U", v, rel_l1(Ug[v], U1[:, v]))
    assert rel_l1(phig, phi1) < RTOL
    m.close()


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("n,nr,p,steps", [(5, 3, 2, 10), (4, 4, 3, 4), (3, 5, 4, 2)])
def test_multistep_parity_and_divb(n, nr, p, steps, schedule):
    o, m, U, phi = setup_case(n, nr, p, schedule=schedule)
    dt = o.cfl_dt(U, 0.4)
    for _ in range(steps):
        U, phi = o.step(U, phi, dt)
        m.step(dt)
    Ug, phig = m.download()
    for v in range(8):
        assert rel_l1(Ug[v], U[:, v]) < RTOL, (v, rel_l1(Ug[v], U[:, v]))
    assert rel_l1(phig, phi) < RTOL
    a, r = m.divB()
    assert r < 1e-13
    m.close()


@pytest.mark.parametrize("n,nr,p", [(5, 3, 2), (3, 5, 4)])
def test_divb_of_a_non_solenoidal_field(n, nr, p):
    """a9 on a field that is not divergence-free: a seeded random Phi uploaded
    directly; the GPU's max |sum_f s_f Phi_f| and max relative value match the
    oracle's divB on the same Phi."""
    o, m, U, phi = setup_case(n, nr, p)
    rng = np.random.default_rng(99)
    phi_r = rng.uniform(-1.0, 1.0, phi.shape)
    m.upload(np.ascontiguousarray(U.T), phi_r)
    a, r = m.divB()
    ao, ro = o.divB(phi_r)
    assert ao > 0.1 and ro > 0.05
    assert abs(a - ao) <= 1e-14 * ao and abs(r - ro) <= 1e-14 * ro, (a, ao, r, ro)
    m.close()


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("p", [2, 3, 4])
def test_free_stream_on_gpu(p, schedule):
    o, m, U, phi = setup_case(4 if p < 4 else 3, 3 if p < 4 else 5, p, problem="uniform", schedule=schedule)
    dt = m.cfl_dt(0.3)
    for _ in range(3):
        m.step(dt)
    Ug, phig = m.download()
    dev = np.abs(Ug - U.T).max(axis=1) / np.abs(U).max(axis=0)
    assert dev.max() < 1e-13, dev
    assert np.abs(phig - phi).max() < 1e-13 * np.abs(phi).max()
    m.close()


def rough_state(U, seed=7):
    """Seeded rough zone averages (density over 1.5 decades, pressure over 2) with the
    smooth field's B: strong jumps make the reconstruction overshoot, so the
    positivity scaling is active in many zones."""
    from paper_1905_02504_gb300.inputs import uniform_pm1
    Z = U.shape[0]
    u = uniform_pm1(np.arange(4 * Z), seed=seed).reshape(4, Z)
    rho = 10.0 ** (-1.5 + 1.5 * u[0])
    p = 10.0 ** (-2.0 + 2.0 * u[1])
    v = 0.5 * np.stack([u[2], u[3], u[2] * u[3]], 1)
    B = U[:, 5:8]
    E = p / (2.0 / 3.0) + 0.5 * rho * (v * v).sum(1) + 0.5 * (B * B).sum(1)
    return np.concatenate([rho[:, None], rho[:, None] * v, E[:, None], B], 1)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("n,nr,p", [(5, 3, 2), (5, 3, 3), (3, 5, 4)])
def test_positivity_parity(n, nr, p, schedule):
    from paper_1905_02504_gb300 import geomhd
    o, m, U, phi = setup_case(n, nr, p, schedule=schedule)
    U = rough_state(U)
    m.upload(np.ascontiguousarray(U.T), phi.copy())
    geomhd.geo_set_positivity(m.h, 1)
    o.positivity = True
    try:
        dt = o.cfl_dt(U, 0.3)
        U1, phi1 = o.step(U, phi, dt)
        m.step(dt)
    finally:
        o.positivity = False
    Ug, phig = m.download()
    for v in range(8):
        assert rel_l1(Ug[v], U1[:, v]) < RTOL, (v, rel_l1(Ug[v], U1[:, v]))
    assert rel_l1(phig, phi1) < RTOL
    # without the limiter the same step differs (or breaks down with a negative
    # pressure): the scaling did act
    m.upload(np.ascontiguousarray(U.T), phi.copy())
    geomhd.geo_set_positivity(m.h, 0)
    m.step(dt)
    U0g, _ = m.download()
    d = max(rel_l1(U0g[v], U1[:, v]) for v in range(8))
    assert not np.isfinite(d) or d > 1e-8
    m.close()


def test_face_geometry_matches_oracle_and_closes():
    from paper_1905_02504_gb300 import geomhd
    o, m, U, phi = setup_case(4, 4, 3)
    area, nrm = geomhd.geo_face_geometry(m.h)
    om = o.mesh
    ref_a = np.empty(om.F)
    ref_n = np.empty((om.F, 3))
    for f in range(om.F):
        zL, lfL = om.face_L[f]
        zR, lfR = om.face_R[f]
        z0, lf0, sgn = (zL, lfL, 1.0) if zL >= 0 else (zR, lfR, -1.0)
        fg = o.dfb.fgeo[lf0]
        ref_a[f] = o.dfb.area[z0, lf0]
        ref_n[f] = sgn * (fg["w"][:, None] * fg["dA"][z0][:, None] * fg["n"][z0]).sum(0)
    assert np.abs(area - ref_a).max() <= 1e-13 * ref_a.max()
    assert np.abs(nrm - ref_n).max() <= 1e-13 * ref_a.max()
    # closure: the six signed area vectors of every zone sum to zero
    close = (om.zone_face_sign[..., None] * nrm[om.zone_face]).sum(1)
    assert np.abs(close).max() <= 1e-14 * ref_a.max()
    m.close()
