"""Pins of the oracle's divergence-free reconstruction (Sec. IV) and ADER predictor (Sec. V)."""
import numpy as np
import pytest

from oracle import mesh as M
from oracle import refelem
from oracle.ader import AderPredictor
from oracle.divfree import DivFreeB
from oracle.weno import WenoAO
from paper_1905_02504_gb300.inputs import Problem


class LinearB(Problem):
    """Uniform fluid with a linear, divergence-free field B = B0 + (x(a3-a2), y(a1-a3), z(a2-a1)),
    the curl of the quadratic potential A = (a1 y z, a2 z x, a3 x y) + B0 x r / 2."""

    def __init__(self):
        super().__init__("uniform", v0=(0.1, -0.2, 0.3), B0=(0.3, -0.2, 0.5))
        self.a = np.array([0.7, -0.4, 0.25])

    def vector_potential(self, x):
        a = self.a
        A = np.stack([a[0] * x[..., 1] * x[..., 2], a[1] * x[..., 2] * x[..., 0],
                      a[2] * x[..., 0] * x[..., 1]], -1)
        return A + 0.5 * np.cross(np.broadcast_to(self.B0, x.shape), x)

    def magnetic(self, x):
        a = self.a
        return self.B0 + np.stack([x[..., 0] * (a[2] - a[1]), x[..., 1] * (a[0] - a[2]),
                                   x[..., 2] * (a[1] - a[0])], -1)


def divergence(dfb, coef, pts):
    """Analytic div of the reconstructed polynomial at physical points (Z, np, 3)."""
    g0 = dfb.weno.geo0
    s = (pts - g0["xc"][:, None, :]) / g0["l0"][:, None, None]
    out = np.zeros(pts.shape[:2])
    for d in range(3):
        for t, e in enumerate(dfb.terms[d]):
            if e[d] == 0:
                continue
            ee = e.copy()
            ee[d] -= 1
            out += coef[:, d, t][:, None] * e[d] * np.prod(s ** ee, axis=-1)
    return out / g0["l0"][:, None]


@pytest.fixture(scope="module", params=[2, 3])
def setup(request):
    from oracle.step import Oracle
    return Oracle(3, 5, 1.0, 2.0, request.param)


def test_field_reproduced_exactly(setup):
    """A linear field is reproduced exactly where the face rule integrates n dA . B
    exactly (straight-sided order-2 zones); on curved order-3 zones the 2x2 face
    rule is exact for n dA but not for n dA . (linear B), so there a uniform field
    is the exact case."""
    o = setup
    pr = LinearB()
    if o.mesh.p == 3:
        pr.a = np.zeros(3)
    U, phi = o.initial_state(pr)
    co = o.weno.reconstruct(U)
    coef, mean = o.dfb.reconstruct(co, U, phi)
    k = np.arange(o.mesh.Z) % o.mesh.nr
    ok = k == 2                      # every face neighbour has an exact WENO fit
    pts = o.weno.geo0["xg"][:, ::9]
    B = o.dfb.evaluate(coef, pts)
    assert np.abs(B - pr.magnetic(pts))[ok].max() < 1e-12
    # the zone mean equals the exact zone average of B
    assert np.abs(mean - U[:, 5:8])[ok].max() < 1e-12


def test_divergence_free_and_face_consistent(setup):
    o = setup
    from paper_1905_02504_gb300.inputs import make_problem
    U, phi = o.initial_state(make_problem("smooth"))
    co = o.weno.reconstruct(U)
    coef, mean, bperp = o.dfb.reconstruct(co, U, phi, return_bperp=True)
    pts = o.weno.geo0["xg"][:, ::4]
    div = divergence(o.dfb, coef, pts)
    scale = np.abs(o.dfb.evaluate(coef, pts)).max() / o.weno.geo0["l0"].min()
    # every non-constant coefficient of div B is constrained to zero
    assert (np.abs(div - div[:, :1]).max()) < 1e-12 * scale
    # the constant one is fixed by the face constraints (Eq. 4.14); it vanishes
    # where the face rule integrates n dA . B exactly (order 2, bilinear faces) and
    # is a truncation-size remainder on curved order-3 faces
    tol = 1e-10 if o.mesh.p == 2 else 2e-3
    assert np.abs(div).max() < tol * scale
    # Eq. 4.13: the shifted nodal fields have the primal face mean
    m = o.mesh
    for f, b in bperp.items():
        zL, lfL = m.face_L[f]
        z0, lf0 = (zL, lfL) if zL >= 0 else tuple(m.face_R[f])
        fg = o.dfb.fgeo[lf0]
        w = fg["w"] * fg["dA"][z0] / o.dfb.area[z0, lf0]
        assert abs((w * b).sum() - phi[f] / o.dfb.area[z0, lf0]) < 1e-14 * (1 + abs(phi[f]))
    # Eq. 4.14 holds for the reconstructed field on every face of every zone
    for lf in range(6):
        fg = o.dfb.fgeo[lf]
        Bq = o.dfb.evaluate(coef, fg["x"])
        w = fg["w"][None] * fg["dA"] / o.dfb.area[:, lf:lf + 1]
        lhs = (w * (fg["n"] * Bq).sum(-1)).sum(1)
        f = m.zone_face[:, lf]
        rhs = m.zone_face_sign[:, lf] * phi[f] / o.dfb.area[:, lf]
        assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("p", [2, 3, 4])
def test_predictor_uniform_state(p):
    m = M.Mesh(3, 2, 1.0, 2.0, p)
    c = np.repeat(np.arange(m.ncol), m.nr)[:20]
    k = np.tile(np.arange(m.nr), m.ncol)[:20]
    X = m.zone_nodes(c, k)
    ad = AderPredictor(m, X, 5.0 / 3.0)
    U = np.array([1.2, 0.3, -0.1, 0.2, 3.0, 0.4, 0.1, -0.3])
    Uh = ad.predict(np.broadcast_to(U, X.shape[:2] + (8,)).copy(), 0.05)
    Up = Uh / ad.J[:, None, :, None]
    assert np.abs(Up - U).max() < 1e-14 * np.abs(U).max() * 10


@pytest.mark.parametrize("p", [2, 3, 4])
def test_predictor_exact_for_advected_polynomial_on_affine_zone(p):
    """Affine zone, uniform v and pressure, B = 0: the space-time solution rho(x - v t)
    (degree p-1 in x) is reproduced at every node and time level after p Picard
    iterations (the iteration operator is nilpotent on this space)."""
    g = 5.0 / 3.0
    m = M.Mesh(2, 2, 1.0, 2.0, p)
    rng = np.random.default_rng(7)
    A = np.eye(3) * 0.2 + 0.03 * rng.standard_normal((3, 3))
    X = (m.el.nodes @ A.T + np.array([1.0, 0.2, -0.3]))[None]
    ad = AderPredictor(m, X, g)
    v = np.array([0.7, -0.4, 0.3])
    p0 = 0.8
    from oracle.mesh import taylor_exponents
    ex = taylor_exponents(p - 1, 0)
    co = rng.standard_normal(len(ex)) * 0.1

    def rho(x):
        out = np.full(x.shape[:-1], 1.5)
        for e, c in zip(ex, co):
            out += c * np.prod(x ** e, axis=-1)
        return out

    def cons(x):
        r = rho(x)
        U = np.zeros(x.shape[:-1] + (8,))
        U[..., 0] = r
        U[..., 1:4] = r[..., None] * v
        U[..., 4] = p0 / (g - 1) + 0.5 * r * (v @ v)
        return U

    dt = 0.05
    Uh = ad.predict(cons(X), dt)
    tau = refelem.time_nodes(p)
    for mi, t in enumerate(tau):
        exact = cons(X - v * t * dt)
        assert np.abs(Uh[:, mi] / ad.J[..., None] - exact).max() < 1e-13, (p, mi)
