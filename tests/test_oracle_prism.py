"""Pins of the paper's prism element and frustum zones (oracle/prism.py): the node
sets against the printed appendices, the isoparametric frustum against the
geodesic mesh's own factorised map, and the ADER-CG predictor of oracle/ader.py
run on the paper's element (Sec. V, App. B-D)."""
import os

import numpy as np
import pytest

from oracle import geodesic as G
from oracle import prism as PR
from oracle import refelem
from oracle.ader import AderPredictor

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _eval(expr):
    return float(eval(expr, {"s3": np.sqrt(3.0)}))


def printed_nodes(p):
    """Eqs. C.2-C.16 (the first six are the order-2 nodes) and Eqs. D.2-D.27."""
    path = os.path.join(GOLD, "prism_bases.txt" if p < 4 else "prism_nodes_p4.txt")
    nodes = []
    for line in open(path):
        if line.startswith("node "):
            nodes.append([_eval(t) for t in line.split(":")[1].split()])
    return np.array(nodes[:{2: 6, 3: 15, 4: 26}[p]])


def _same_set(A, B):
    d = np.linalg.norm(A[:, None] - B[None], axis=2)
    return len(A) == len(B) and (d.min(axis=1) < 1e-14).all() and (d.min(axis=0) < 1e-14).all()


@pytest.mark.parametrize("p", [2, 3, 4])
def test_nodes_are_the_printed_nodes(p):
    assert _same_set(PR.prism_nodes(p), printed_nodes(p))


@pytest.mark.parametrize("p", [2, 3, 4])
def test_element_basis_and_derivatives(p):
    el = PR.PrismElement(p)
    assert np.allclose(el.basis(el.nodes), np.eye(el.N), atol=1e-12)
    # every monomial of the space and its derivatives are reproduced
    rng = np.random.default_rng(p)
    pts = np.column_stack([rng.uniform(-0.3, 0.3, 20), rng.uniform(-0.2, 0.3, 20), rng.uniform(-0.5, 0.5, 20)])
    vals = refelem.monomials(el.nodes, el.exps)
    assert np.allclose(el.basis(pts) @ vals, refelem.monomials(pts, el.exps), atol=1e-12)
    for a in range(3):
        assert np.allclose(el.dbasis(pts, a) @ vals, refelem.monomial_derivative(pts, el.exps, a), atol=1e-11)


def _triangle(level=1, k=5):
    v, t = G.geodesic_sphere(level)
    return v[t[k, 0]], v[t[k, 1]], v[t[k, 2]]


@pytest.mark.parametrize("p", [2, 3, 4])
def test_frustum_map_equals_the_factorised_map(p):
    """The prism's serendipity space holds r(zeta) S(x, y) (S of degree p-1 across,
    linear in zeta) and the nodes follow the same placement rule, so the
    isoparametric frustum is geodesic.py's frustum: equal volumes through two
    different computations."""
    a, b, c = _triangle()
    z = PR.FrustumZone(p, a, b, c, 1.0, 1.3)
    assert abs(z.volume() - G.frustum_volume(a, b, c, 1.0, 1.3, p)) < 1e-13 * z.volume()


@pytest.mark.parametrize("p", [2, 3, 4])
def test_predictor_exact_for_advected_polynomial_on_affine_prism(p):
    """Affine prism zone, uniform v and pressure, B = 0: rho(x - v t) of degree
    p-1 is reproduced at every node and time level after p Picard iterations."""
    g = 5.0 / 3.0
    rng = np.random.default_rng(11)
    A = np.eye(3) * 0.2 + 0.03 * rng.standard_normal((3, 3))
    el = PR.PrismElement(p)
    z = PR.FrustumZone(p, X=el.nodes @ A.T + np.array([1.0, 0.2, -0.3]))
    X = z.X
    ad = AderPredictor(z, X, g)
    v = np.array([0.7, -0.4, 0.3])
    p0 = 0.8
    ex = [e for e in el.exps if sum(e) <= p - 1]
    co = rng.standard_normal(len(ex)) * 0.1

    def cons(x):
        r = np.full(x.shape[:-1], 1.5)
        for e, cc in zip(ex, co):
            r += cc * np.prod(x ** np.array(e), axis=-1)
        U = np.zeros(x.shape[:-1] + (8,))
        U[..., 0] = r
        U[..., 1:4] = r[..., None] * v
        U[..., 4] = p0 / (g - 1) + 0.5 * r * (v @ v)
        return U

    dt = 0.05
    Uh = ad.predict(cons(X), dt)
    for mi, t in enumerate(refelem.time_nodes(p)):
        exact = cons(X - v * t * dt)
        assert np.abs(Uh[:, mi] / ad.J[..., None] - exact).max() < 1e-13, (p, mi)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_predictor_keeps_a_uniform_state_on_a_curved_frustum(p):
    a, b, c = _triangle()
    z = PR.FrustumZone(p, a, b, c, 1.0, 1.3)
    ad = AderPredictor(z, z.X, 5.0 / 3.0)
    U = np.array([1.2, 0.3, -0.1, 0.2, 3.0, 0.4, 0.1, -0.3])
    Uh = ad.predict(np.broadcast_to(U, z.X.shape[:2] + (8,)).copy(), 0.02)
    assert np.abs(Uh / ad.J[:, None, :, None] - U).max() < 1e-13 * np.abs(U).max()
    assert (ad.J > 0).all()
