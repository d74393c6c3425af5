"""Transpose checks of the hand-written reverse kernels, one forward stage at a
time (Sec. VI read backwards): for stage y = f(x) and seeded random x-directions
d and y-cotangents w, <w, (f(x + h d) - f(x - h d)) / 2h> (fourth-order central
differences of the GPU forward stage alone) must equal <f'(x)^T w, d> from the
stage's reverse kernel alone.

  WENO-AO    x = zone averages U            y = Taylor coefficients
  predictor  x = Taylor coefficients        y = face- and edge-point states
             (nodal normal fields and U held fixed: their paths are the KKT and
             MinMod reverse kernels, covered by the full-step checks)
  faces      x = face-point states          y = time-integrated HLL face fluxes
  edges      x = edge-point states          y = time-integrated edge EMFs

The base state carries 10 % seeded noise (as in the full-step checks), so most
MinMod / HLL / Rusanov and |beta_H - beta_k| decisions sit far from their
switches compared with the +-2h stencil.  The face and edge directions touch a
seeded 5 % of the point states, so that a stencil meets few of the solver
decisions.  The differences are taken at three steps.  A direction counts when
the two largest steps already agree to 2e-8 (truncation below rounding: the
smooth predictor) or when the differences settle at the fourth-order rate;
otherwise a switch was crossed and it is skipped (at least two of six must
count).  The adjoint must match the Richardson extrapolation of the settled
pair."""
import numpy as np
import pytest

from conftest import gpu_available
from test_gpu_parity import setup_case

pytestmark = pytest.mark.gpu

H = (1e-5, 2.5e-6, 6.25e-7)   # relative steps of the fourth-order differences
TOL = 1e-7                    # relative agreement with their Richardson extrapolation
ST_WENO, ST_BPERP, ST_ADER, ST_FACE, ST_EDGE = 0, 1, 2, 3, 4


@pytest.fixture(autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")


def forward_stage(mesh, stage, dt, U, phi, x, fixed):
    """y = f(x) of one stage on the GPU, the other inputs from `fixed`."""
    from paper_1905_02504_gb300 import geomhd
    g = geomhd
    if stage == ST_WENO:
        mesh.upload(np.ascontiguousarray(x.reshape(8, -1)), phi)
        g.geo_debug_run_stage(mesh.h, ST_WENO, dt)
        return g.geo_debug_buffer(mesh.h, 0, fixed["nW"])
    if stage == ST_ADER:
        mesh.upload(U, phi)                          # the predictor rewrites the zone B means
        g.geo_debug_set_buffer(mesh.h, 0, x)
        g.geo_debug_set_buffer(mesh.h, 1, fixed["Bp"])
        g.geo_debug_run_stage(mesh.h, ST_ADER, dt)
        return np.concatenate([g.geo_debug_buffer(mesh.h, 2, fixed["nF"]), g.geo_debug_buffer(mesh.h, 3, fixed["nE"])])
    if stage == ST_FACE:
        g.geo_debug_set_buffer(mesh.h, 2, x)
        g.geo_debug_run_stage(mesh.h, ST_FACE, dt)
        return g.geo_debug_buffer(mesh.h, 4, 8 * mesh.F)
    g.geo_debug_set_buffer(mesh.h, 3, x)
    g.geo_debug_run_stage(mesh.h, ST_EDGE, dt)
    return g.geo_debug_buffer(mesh.h, 5, mesh.E)


@pytest.mark.parametrize("stage", [ST_WENO, ST_ADER, ST_FACE, ST_EDGE], ids=["weno", "predictor", "faces", "edges"])
@pytest.mark.parametrize("n,nr,p", [(4, 3, 2), (4, 3, 3), (3, 5, 4)])
def test_stage_transpose(n, nr, p, stage):
    from paper_1905_02504_gb300 import geomhd
    g = geomhd
    o, mesh, U0, phi = setup_case(n, nr, p)
    rng = np.random.default_rng(7 + 10 * p + stage)
    Uz = U0 * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, U0.shape))
    U = np.ascontiguousarray(Uz.T)                  # [8][Z]
    dt = o.cfl_dt(Uz, 0.4)
    Z = mesh.Z
    nc1 = len(o.weno.exps)
    M = p
    nqt = sum(o.dfb.nq)
    ns = {2: 1, 3: 2, 4: 3}[p]
    nqmax = max(o.dfb.nq)
    fixed = {"nW": 8 * nc1 * Z, "nF": (M - 1) * nqt * 8 * Z, "nE": (M - 1) * 12 * ns * 8 * Z}
    # base intermediates of the noisy state
    mesh.upload(U, phi)
    for s in (ST_WENO, ST_BPERP, ST_ADER):
        g.geo_debug_run_stage(mesh.h, s, dt)
    base = {ST_WENO: U.ravel().copy(), ST_ADER: g.geo_debug_buffer(mesh.h, 0, fixed["nW"]),
            ST_FACE: g.geo_debug_buffer(mesh.h, 2, fixed["nF"]), ST_EDGE: g.geo_debug_buffer(mesh.h, 3, fixed["nE"])}
    fixed["Bp"] = g.geo_debug_buffer(mesh.h, 1, nqmax * mesh.F)
    x0 = base[stage]
    y0 = forward_stage(mesh, stage, dt, U, phi, x0, fixed)
    checked, seen = 0, []
    for trial in range(6):
        w = rng.standard_normal(y0.size)
        d = rng.uniform(-1.0, 1.0, x0.size) * np.maximum(np.abs(x0), 1e-3 * np.abs(x0).max())
        if stage in (ST_FACE, ST_EDGE):
            d *= rng.uniform(size=x0.size) < 0.05

        def fd(h):
            # difference the stage outputs first, then project: a projection of
            # ~1e4 terms before differencing would leave ~1e-7 relative rounding
            f = lambda t: forward_stage(mesh, stage, dt, U, phi, x0 + t * d, fixed)
            return float(w @ ((8.0 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12.0 * h)))

        f0, f1, f2 = (fd(h) for h in H)
        seen.append((f0, f1, f2))
        if abs(f0 - f1) <= 2e-8 * abs(f1):
            # truncation already below rounding at the two largest steps
            best = f1 + (f1 - f0) / 255.0
        elif abs(f1 - f2) <= min(abs(f0 - f1) / 16.0, 1e-6 * abs(f2)):
            # smooth within the stencils: the O(h^4) error shrinks ~256-fold per
            # step; a switch crossed gives no such rate
            best = f2 + (f2 - f1) / 255.0
        else:
            continue
        gx = g.geo_debug_stage_vjp(mesh.h, stage, dt, U, phi, w, x0.size)
        adj = float(gx @ d)
        assert abs(adj - best) <= TOL * abs(best), (trial, adj, f0, f1, f2)
        checked += 1
    assert checked >= 2, (checked, seen)
    mesh.close()


@pytest.mark.parametrize("n,nr,p", [(4, 3, 2), (4, 3, 3), (3, 5, 4)])
def test_reverse_predictor_schedules_agree(n, nr, p):
    """The node-team reverse predictor (default) and the one-thread-per-zone one
    (used with GEO_PRED_ZONE_THREAD) apply the same transpose: their cotangents
    of the Taylor coefficients agree to rounding."""
    from paper_1905_02504_gb300 import geomhd
    g = geomhd
    o, mesh, U0, phi = setup_case(n, nr, p)
    rng = np.random.default_rng(11 + p)
    U = np.ascontiguousarray((U0 * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, U0.shape))).T)
    dt = o.cfl_dt(U.T, 0.4)
    M, nqt, ns, nc1 = p, sum(o.dfb.nq), {2: 1, 3: 2, 4: 3}[p], len(o.weno.exps)
    n_out = (M - 1) * nqt * 8 * mesh.Z + (M - 1) * 12 * ns * 8 * mesh.Z
    w = rng.standard_normal(n_out)
    out = []
    for sched in (geomhd.GEO_PRED_NODE_TEAM, geomhd.GEO_PRED_ZONE_THREAD):
        g.geo_set_predictor(mesh.h, sched)
        out.append(g.geo_debug_stage_vjp(mesh.h, ST_ADER, dt, U, phi, w, 8 * nc1 * mesh.Z))
    assert np.abs(out[0] - out[1]).max() <= 1e-12 * np.abs(out[1]).max()
    mesh.close()
