"""Hand-written adjoint of the step against finite differences.

* A generic linear functional of one step's output, J = <wU, U'> + <wphi, phi'>,
  exercises the whole transposed Jacobian; its adjoint gradient is compared
  along seeded random directions with fourth-order central differences of the GPU
  FP64 forward step and of the FP64 oracle (eps = 2.5e-7, relative agreement 1e-6),
  from zone averages with 10 % seeded noise; the noise seed is the first whose
  step keeps every branch decision at least 1e-6 (normalised) from its switch.
* The differentiation objective (outer-shell B_r^2 after a window of K steps,
  with per-step checkpoints) through torch.autograd, against central differences
  with eps = 1e-6.
MinMod, the HLL wave-speed choices and the Rusanov max are kinks; directions whose
central-difference stencil crosses one (detected with the oracle's branch
signature) are counted separately and not compared.
Directions for phi are discrete curls of random edge values (divergence-free).
"""
import numpy as np
import pytest

from conftest import gpu_available
from test_gpu_parity import setup_case

pytestmark = pytest.mark.gpu

EPS = 1e-6          # the configured central-difference step
EPS_STEP = 2.5e-7   # one step, fourth-order stencil over +-h, +-2h
ROUGH = 0.1         # seeded relative noise on the zone averages of the one-step check
MARGIN = 1e-6       # smallest normalised branch margin accepted in the one-step base state
TOL = 1e-6


@pytest.fixture(autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")


def direction(o, U, rng):
    """Per-variable scaled random direction for U; a curl direction for phi."""
    m = o.mesh
    scale = np.abs(U).mean(axis=0)
    dU = rng.uniform(-1.0, 1.0, U.shape) * scale
    dU[:, 5:8] = 0.0            # the zone B is overwritten by the reconstruction; probe it too below
    a = rng.uniform(-1.0, 1.0, m.E) * 1e-2
    dphi = (m.face_edge_sign * a[m.face_edges]).sum(1)
    return dU, dphi


def gpu_step(mesh, U, phi, dt):
    import torch
    from paper_1905_02504_gb300 import geomhd
    Ut = torch.from_numpy(np.ascontiguousarray(U.T)).cuda()
    pt = torch.from_numpy(phi.copy()).cuda()
    geomhd.geo_state_upload(mesh.h, Ut, pt)
    geomhd.geo_step(mesh.h, dt)
    Uo = torch.empty_like(Ut)
    po = torch.empty_like(pt)
    geomhd.geo_state_download(mesh.h, Uo, po)
    return Uo.cpu().numpy().T, po.cpu().numpy()


def roughen(U, rng, amp=ROUGH):
    """Seeded relative noise on every zone average.  In the smooth field the two
    states of a face differ by little, so the Davis min/max choices, the Rusanov
    max and MinMod sit next to their switch points (or on them: exact MinMod ties
    of the symmetric field), and even a 1e-5 stencil crosses several.  With 10 %
    noise the choices are clear and a +-2e-6 stencil crosses few or none."""
    return U * (1.0 + amp * rng.uniform(-1.0, 1.0, U.shape))


def branch_flips(o, U, phi, dU, dphi, dt, eps):
    """Number of MinMod / HLL / max branch decisions of the oracle step that differ
    between x + eps d and x - eps d (a central difference across a kink)."""
    from oracle import physics
    sigs = []
    for s in (1.0, -1.0):
        physics.BRANCHES = []
        o.step(U + s * eps * dU, phi + s * eps * dphi, dt)
        sigs.append(physics.BRANCHES)
        physics.BRANCHES = None
    return sum(int((np.sign(a[1]) != np.sign(b[1])).sum()) for a, b in zip(*sigs))


def clean_base_state(o, U0, phi, p, K=1, margin=MARGIN, tries=16):
    """First seeded 10 %-noise state whose oracle step takes every MinMod / HLL /
    Rusanov decision with a normalised margin above MARGIN (exact structural ties,
    margin 0 on both sides of every stencil, excepted).  In any noisy state a few
    of the ~1e5 decisions sit within 1e-7 of their switch, and every direction
    then crosses them; such states are skipped.  Returns the state and the
    generator, positioned after the noise draw.  K > 1 checks the decisions of K
    steps."""
    from oracle import physics
    for s in range(tries):
        rng = np.random.default_rng(1905 + p + 1000 * s)
        U = roughen(U0, rng)
        dt = o.cfl_dt(U, 0.4)
        physics.BRANCHES = []
        try:
            Ux, px = U, phi
            for _ in range(K):
                Ux, px = o.step(Ux, px, dt)
            m = np.abs(np.concatenate([np.ravel(x[1]) for x in physics.BRANCHES]))
        finally:
            physics.BRANCHES = None
        if m[m != 0.0].min() > margin:
            return U, rng
    pytest.fail("no seeded state without near-ties in %d tries" % tries)


def central4(J, U, phi, dU, dphi, h):
    """Fourth-order central difference (8 [J(h) - J(-h)] - [J(2h) - J(-2h)]) / 12h: its
    truncation error is O(h^4); at h = 2.5e-7 and 1e-6 the oracle's values agree to a
    few 1e-9 relative, far below the 1e-6 tolerance."""
    d1 = J(U + h * dU, phi + h * dphi) - J(U - h * dU, phi - h * dphi)
    d2 = J(U + 2 * h * dU, phi + 2 * h * dphi) - J(U - 2 * h * dU, phi - 2 * h * dphi)
    return (8.0 * d1 - d2) / (12.0 * h)


@pytest.mark.parametrize("n,nr,p", [(5, 3, 2), (4, 4, 3), (3, 5, 4)])
def test_adjoint_matches_finite_differences(n, nr, p):
    import torch
    from paper_1905_02504_gb300 import geomhd
    o, mesh, U, phi = setup_case(n, nr, p)
    U, rng = clean_base_state(o, U, phi, p)
    dt = o.cfl_dt(U, 0.4)
    wU = rng.standard_normal(U.shape)
    wphi = rng.standard_normal(phi.shape)
    # adjoint gradient of J = <wU, U'> + <wphi, phi'>
    U_in = torch.from_numpy(np.ascontiguousarray(U.T)).cuda()
    phi_in = torch.from_numpy(phi.copy()).cuda()
    gU = torch.empty_like(U_in)
    gphi = torch.empty_like(phi_in)
    geomhd.geo_step_adjoint(mesh.h, dt, U_in, phi_in, torch.from_numpy(np.ascontiguousarray(wU.T)).cuda(),
                            torch.from_numpy(wphi.copy()).cuda(), gU, gphi)
    torch.cuda.synchronize()
    gU = gU.cpu().numpy().T
    gphi = gphi.cpu().numpy()

    def J_gpu(Ux, phix):
        U1, p1 = gpu_step(mesh, Ux, phix, dt)
        return (wU * (U1 - Ux)).sum() + (wphi * (p1 - phix)).sum()

    def J_orc(Ux, phix):
        U1, p1 = o.step(Ux, phix, dt)
        return (wU * (U1 - Ux)).sum() + (wphi * (p1 - phix)).sum()

    checked, crossing, oracle_checked = 0, 0, False
    for trial in range(9):
        dU, dphi = direction(o, U, rng)
        if trial % 3 == 2:      # the zone B (helper) enters through the reconstruction
            dU[:, 5:8] = rng.uniform(-1.0, 1.0, (U.shape[0], 3)) * np.abs(U[:, 5:8]).mean(0)
        h = EPS_STEP
        if branch_flips(o, U, phi, dU, dphi, dt, h) or branch_flips(o, U, phi, dU, dphi, dt, 2 * h):
            crossing += 1       # reported separately: the central difference straddles a kink
            continue
        # compare the part of the derivative the step itself adds: the increment
        # functional <wU, U' - U> + <wphi, phi' - phi> has gradient g - w
        lin = (wU * dU).sum() + (wphi * dphi).sum()
        adj = (gU * dU).sum() + (gphi * dphi).sum() - lin
        fd = central4(J_gpu, U, phi, dU, dphi, h)
        assert abs(adj - fd) <= TOL * abs(fd), (trial, adj, fd)
        checked += 1
        if not oracle_checked:
            fdo = central4(J_orc, U, phi, dU, dphi, h)
            assert abs(adj - fdo) <= TOL * abs(fdo), (adj, fdo)
            oracle_checked = True
    print("order %d: %d directions checked, %d crossed a branch switch" % (p, checked, crossing))
    assert checked >= 6 and oracle_checked
    mesh.close()


def test_window_objective_gradient_with_checkpoints():
    """J = integral of B_r^2 over the outer shell after K = 3 steps (order 3), from a
    noisy state whose K steps take every decision clear of its switch (as in the
    one-step check), against fourth-order central differences."""
    import torch
    from paper_1905_02504_gb300 import autodiff, geomhd
    K = 3
    o, mesh, U, phi = setup_case(3, 3, 3)
    # three steps take ~1.3e5 decisions: margin 5e-7, stencil reach 2e-7
    U, _ = clean_base_state(o, U, phi, 3, K=K, margin=5e-7)
    dt = o.cfl_dt(U, 0.4)
    eps = 1e-7
    Ut = torch.from_numpy(np.ascontiguousarray(U.T)).cuda().requires_grad_(True)
    pt = torch.from_numpy(phi.copy()).cuda().requires_grad_(True)
    UK, pK = autodiff.step_window(mesh, Ut, pt, dt, K)
    J = autodiff.outer_br2(mesh, pK)
    J.backward()
    gU = Ut.grad.cpu().numpy().T
    gphi = pt.grad.cpu().numpy()
    # objective definition check on the final state
    m = o.mesh
    outer = np.arange(m.ncol) * (m.nr + 1) + m.nr
    area = o.dfb.area[m.face_L[outer, 0], 5]
    assert abs(J.item() - (pK.detach().cpu().numpy()[outer] ** 2 / area).sum()) <= 1e-12 * J.item()

    def J_of(Ux, phix):
        with torch.no_grad():
            a = torch.from_numpy(np.ascontiguousarray(Ux.T)).cuda()
            b = torch.from_numpy(phix.copy()).cuda()
            _, pk = autodiff.StepWindow.apply(a, b, mesh, dt, K)
            return geomhd.geo_outer_Br2(mesh.h, pk)

    def window_flips(dU, dphi, h):
        from oracle import physics
        sigs = []
        for s in (1.0, -1.0):
            physics.BRANCHES = []
            Ux, px = U + s * h * dU, phi + s * h * dphi
            for _ in range(K):
                Ux, px = o.step(Ux, px, dt)
            sigs.append(physics.BRANCHES)
            physics.BRANCHES = None
        return sum(int((np.sign(a[1]) != np.sign(b[1])).sum()) for a, b in zip(*sigs))

    rng = np.random.default_rng(64)
    checked = 0
    for _ in range(6):
        dU, dphi = direction(o, U, rng)
        if window_flips(dU, dphi, eps) or window_flips(dU, dphi, 2 * eps):
            continue
        adj = (gU * dU).sum() + (gphi * dphi).sum()
        fd = central4(J_of, U, phi, dU, dphi, eps)
        assert abs(adj - fd) <= TOL * abs(fd), (adj, fd)
        checked += 1
    assert checked >= 4
    mesh.close()


def test_fp32_bulk_window_gradient_matches_fp64():
    """The FP32-bulk form is differentiated by the FP64 adjoint applied to its own
    (FP32-bulk) checkpoints.  Its window gradient agrees with the FP64 form's to
    the FP32-bulk state error (directional derivatives within 1e-4 relative), and
    differs from it (the checkpoints really are the FP32-bulk ones)."""
    import torch
    from paper_1905_02504_gb300 import autodiff, geomhd
    K = 3
    o, m64, U, phi = setup_case(3, 3, 3)
    U, _ = clean_base_state(o, U, phi, 3, K=K, margin=5e-7)
    dt = o.cfl_dt(U, 0.4)
    m32 = geomhd.Mesh(3, 3, 1.0, 2.0, 3, prec=geomhd.GEO_FP32_BULK)
    grads = []
    for mesh in (m64, m32):
        Ut = torch.from_numpy(np.ascontiguousarray(U.T)).cuda().requires_grad_(True)
        pt = torch.from_numpy(phi.copy()).cuda().requires_grad_(True)
        _, pK = autodiff.step_window(mesh, Ut, pt, dt, K)
        autodiff.outer_br2(mesh, pK).backward()
        grads.append((Ut.grad.cpu().numpy().T, pt.grad.cpu().numpy()))
    rng = np.random.default_rng(32)
    worst, differs = 0.0, False
    for _ in range(4):
        dU, dphi = direction(o, U, rng)
        d64 = (grads[0][0] * dU).sum() + (grads[0][1] * dphi).sum()
        d32 = (grads[1][0] * dU).sum() + (grads[1][1] * dphi).sum()
        worst = max(worst, abs(d32 - d64) / abs(d64))
        differs = differs or d32 != d64
    assert worst < 1e-4 and differs, worst
    m32.close()
    m64.close()


def test_window_on_a_side_stream_matches_default_stream():
    """A mesh created on a torch side stream gives the same window output and
    gradient (to rounding) as one on the default stream: the binding orders the mesh stream
    after torch's current stream (inputs written by torch) and torch's current
    stream after the mesh stream (outputs written by the library)."""
    import torch
    from paper_1905_02504_gb300 import autodiff, geomhd
    K = 2
    o, m0, U, phi = setup_case(3, 3, 3)
    dt = o.cfl_dt(U, 0.4)
    side = torch.cuda.Stream()
    m1 = geomhd.Mesh(3, 3, 1.0, 2.0, 3, stream=side.cuda_stream)
    outs = []
    for mesh in (m0, m1):
        # torch writes the inputs on its current stream right before the call
        Ut = torch.from_numpy(np.ascontiguousarray(U.T)).cuda()
        pt = torch.from_numpy(phi.copy()).cuda()
        Ut = (Ut * 1.0).requires_grad_(True)
        pt = (pt * 1.0).requires_grad_(True)
        UK, pK = autodiff.step_window(mesh, Ut, pt, dt, K)
        J = autodiff.outer_br2(mesh, pK)
        J.backward()
        outs.append((UK.detach().cpu().numpy(), pK.detach().cpu().numpy(),
                     Ut.grad.cpu().numpy(), pt.grad.cpu().numpy()))
    # the forward step is deterministic; the reverse sweep scatters into the WENO
    # stencils with FP64 atomics, so the gradients agree to rounding
    for a, b in zip(outs[0][:2], outs[1][:2]):
        assert np.array_equal(a, b)
    for a, b in zip(outs[0][2:], outs[1][2:]):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    m1.close()
    m0.close()


@pytest.mark.parametrize("n,nr,p", [(4, 3, 2), (4, 3, 3), (3, 5, 4)])
def test_reverse_sweep_with_stored_iterates_matches_recompute(n, nr, p):
    """geo_step_adjoint with a team schedule stores the checkpoint predictor's
    Picard iterates in its forward recompute and the reverse team reads them;
    with one thread per zone the reverse predictor recomputes them.  Both give
    the same transpose of the step: gradients equal to rounding."""
    import torch
    from paper_1905_02504_gb300 import geomhd
    o, m, U0, phi = setup_case(n, nr, p)
    rng = np.random.default_rng(23 + p)
    U = np.ascontiguousarray((U0 * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, U0.shape))).T)
    dt = o.cfl_dt(U.T, 0.4)
    Ut = torch.from_numpy(U).cuda()
    pt = torch.from_numpy(phi.copy()).cuda()
    gUo = torch.from_numpy(rng.standard_normal(U.shape)).cuda()
    gpo = torch.from_numpy(rng.standard_normal(phi.shape)).cuda()
    out = []
    for sched in (geomhd.GEO_PRED_NODE_TEAM, geomhd.GEO_PRED_ZONE_THREAD):
        geomhd.geo_set_predictor(m.h, sched)
        gU, gp = torch.empty_like(Ut), torch.empty_like(pt)
        geomhd.geo_step_adjoint(m.h, dt, Ut, pt, gUo, gpo, gU, gp)
        torch.cuda.synchronize()
        out.append((gU.cpu().numpy(), gp.cpu().numpy()))
    for a, b in zip(out[0], out[1]):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    m.close()
