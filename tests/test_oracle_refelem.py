"""Pins of the oracle's reference-element generator against what the paper prints
and what the mathematics fixes (Sec. V.b-V.c, App. A-D)."""
import os

import numpy as np
import pytest

from oracle import quadrature, refelem

GOLD = os.path.join(os.path.dirname(__file__), "golden")
s3 = np.sqrt(3.0)
s15 = np.sqrt(15.0)


def _eval(expr):
    return float(eval(expr, {"s3": s3, "s15": s15, "sqrt": np.sqrt}))


def load_r_matrices():
    out, cur = {}, None
    for line in open(os.path.join(GOLD, "r_matrices.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("order"):
            cur = int(line.split()[1])
            out[cur] = []
            continue
        out[cur].append([_eval(t) for t in line.split()])
    return {k: np.array(v) for k, v in out.items()}


@pytest.mark.parametrize("p", [2, 3, 4])
def test_r_matrix_equals_printed(p):
    R, K0 = refelem.r_matrix(p)
    gold = load_r_matrices()[p]
    assert np.abs(R - gold).max() < 1e-14
    # Eq. 5.29: K_tau^0 = -(K_tau^11)^-1 K_tau^10 = [1, ..., 1]
    assert np.abs(K0 - 1.0).max() < 1e-14


@pytest.mark.parametrize("p", [2, 3, 4])
def test_time_nodes_are_gauss_points(p):
    tau, w = quadrature.time_gauss(p)
    printed = {2: [0, 0.5], 3: [0, 0.5 - 0.5 / s3, 0.5 + 0.5 / s3],
               4: [0, 0.5 - 0.5 * np.sqrt(0.6), 0.5, 0.5 + 0.5 * np.sqrt(0.6)]}[p]
    assert np.allclose(tau, printed, atol=1e-15)
    # the Gauss rule on tau_2..tau_M integrates polynomials of degree 2M-3 exactly
    for k in range(2 * (p - 1)):
        assert abs((w * tau[1:] ** k).sum() - 1.0 / (k + 1)) < 1e-14


def load_prism():
    bases, nodes = {}, {}
    for line in open(os.path.join(GOLD, "prism_bases.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, body = line.split(":")
        h = head.split()
        if h[0] == "node":
            nodes[int(h[1])] = [_eval(t) for t in body.split()]
        else:
            terms = {}
            for t in body.split():
                e, c = t.split("=")
                terms[tuple(int(x) for x in e)] = _eval(c)
            bases[(int(h[0]), int(h[1]))] = terms
    return bases, nodes


@pytest.mark.parametrize("p", [2, 3])
def test_generator_reproduces_printed_prism_bases(p):
    bases, nodes = load_prism()
    nn = 6 if p == 2 else 15
    X = np.array([nodes[i] for i in range(1, nn + 1)])
    exps = refelem.prism_exponents(p)
    C = refelem.lagrange_coefficients(X, exps)
    for (order, j), terms in bases.items():
        if order != p:
            continue
        for row, e in enumerate(map(tuple, exps)):
            assert abs(C[row, j - 1] - terms.get(e, 0.0)) < 1e-13, (p, j, e)


def test_nodal_flux_difference_row_b16():
    """Eq. B.16: at node 1 the flux difference is (-F1+F2) + (-G1-G2+2G3)/sqrt3 + (H1-H4),
    i.e. the derivative of the basis at the node (nodal collocation, Eq. C.34)."""
    _, nodes = load_prism()
    X = np.array([nodes[i] for i in range(1, 7)])
    exps = refelem.prism_exponents(2)
    C = refelem.lagrange_coefficients(X, exps)
    d = [refelem.monomial_derivative(X[:1], exps, a) @ C for a in range(3)]
    assert np.allclose(d[0][0], [-1, 1, 0, 0, 0, 0], atol=1e-14)
    assert np.allclose(d[1][0], np.array([-1, -1, 2, 0, 0, 0]) / s3, atol=1e-14)
    assert np.allclose(d[2][0], [1, 0, 0, -1, 0, 0], atol=1e-14)


@pytest.mark.parametrize("p,N", [(2, 8), (3, 20), (4, 32)])
def test_hex_serendipity_element(p, N):
    el = refelem.HexElement(p)
    assert el.N == N
    assert np.abs(el.basis(el.nodes) - np.eye(N)).max() < 1e-13
    rng = np.random.default_rng(1)
    pts = rng.uniform(-0.5, 0.5, (40, 3))
    # every monomial of the space is reproduced exactly by interpolation ...
    vals_nodes = refelem.monomials(el.nodes, el.exps)
    interp = el.basis(pts) @ vals_nodes
    assert np.abs(interp - refelem.monomials(pts, el.exps)).max() < 1e-12
    # ... and so are its derivatives (the space is closed under d/dxi)
    for a in range(3):
        dint = el.dbasis(pts, a) @ vals_nodes
        assert np.abs(dint - refelem.monomial_derivative(pts, el.exps, a)).max() < 1e-11
    # complete polynomials of degree p-1 are in the space
    deg = el.exps.sum(1)
    for tot in range(p):
        n_tot = (tot + 1) * (tot + 2) // 2
        assert (deg == tot).sum() >= n_tot


def test_appendix_a_rules():
    rules = quadrature.appendix_a_rules()
    for name, (pts, w) in rules.items():
        assert abs(w.sum() - 1.0) < 1e-15, name
    # A.4 is the 2x2 Gauss rule on the unit square
    x, wg = quadrature.gauss_legendre(2)
    pts, w = rules["A4"]
    g = np.array([[a + 0.5, b + 0.5] for b in x for a in x])
    assert np.allclose(np.sort(pts, axis=0), np.sort(g, axis=0), atol=1e-15)
    # A.4 integrates x^a y^b exactly for a, b <= 3 on the unit square
    for a in range(4):
        for b in range(4):
            exact = 1.0 / ((a + 1) * (b + 1))
            assert abs((w * pts[:, 0] ** a * pts[:, 1] ** b).sum() - exact) < 1e-14
    # A.6 is exact to degree 3 in x and 5 in y
    pts, w = rules["A6"]
    for a in range(4):
        for b in range(6):
            exact = 1.0 / ((a + 1) * (b + 1))
            assert abs((w * pts[:, 0] ** a * pts[:, 1] ** b).sum() - exact) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 3, 6, 11])
def test_gauss_legendre_exactness(n):
    x, w = quadrature.gauss_legendre(n)
    for k in range(2 * n):
        exact = ((0.5) ** (k + 1) - (-0.5) ** (k + 1)) / (k + 1)
        assert abs((w * x ** k).sum() - exact) < 1e-15
