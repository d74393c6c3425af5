"""Quadrature rules used by the oracle.

Gauss-Legendre rules come from numpy's ``leggauss`` (a library primitive) mapped
to the reference interval [-1/2, 1/2] with weights summing to one.  The
reference element of the build is the unit cube [-1/2,1/2]^3 (unit edges,
centroid at the origin, as the paper's reference prism in App. B-C).

``appendix_a_rules`` transcribes the face rules printed in App. A (Eqs. A.1-A.6)
on the paper's reference triangle / unit square; they are only used as pins.

Face and edge rules of the hexahedral build (paper silent for hexahedra):
  order 2 : faces 2x2 Gauss (Eq. A.4), edges 1 point (midpoint)
  order 3 : faces 2x2 Gauss (Eq. A.4), edges 2-point Gauss
  order 4 : radial faces 3x3 Gauss, side faces 3 (angular) x 2 (radial) Gauss (the
            structure of Eq. A.6), edges 3-point Simpson (Sec. II.c)
Time: the Gauss points tau_2..tau_M of Eqs. 5.15-5.17 with their Gauss weights.

Pinned by: tests/test_oracle_refelem.py (exactness on monomials, App. A weights
summing to one, the 2x2 rule equal to Eq. A.4, Gauss points equal to Eqs. 5.15-5.17).
"""
import numpy as np


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1/2, 1/2]; weights sum to 1."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * x, 0.5 * w


def face_rule(order, radial_face):
    """Tensor face rule (u, v) -> points (nq, 2) in [-1/2,1/2]^2 and weights (nq,).

    For side faces the parameters are (angular, radial); u is outer, v inner."""
    if order in (2, 3):
        nu, nv = 2, 2
    elif order == 4:
        nu, nv = (3, 3) if radial_face else (3, 2)
    else:
        raise ValueError("order must be 2, 3 or 4")
    xu, wu = gauss_legendre(nu)
    xv, wv = gauss_legendre(nv)
    pts = np.array([[a, b] for a in xu for b in xv])
    wts = np.array([wa * wb for wa in wu for wb in wv])
    return pts, wts


def edge_rule(order):
    """Edge rule on [-1/2, 1/2]: points and weights summing to 1."""
    if order == 2:
        return np.array([0.0]), np.array([1.0])
    if order == 3:
        return gauss_legendre(2)
    if order == 4:
        return np.array([-0.5, 0.0, 0.5]), np.array([1.0, 4.0, 1.0]) / 6.0
    raise ValueError("order must be 2, 3 or 4")


def time_gauss(order):
    """Scaled time nodes tau_1..tau_M (Eqs. 5.15-5.17) and the Gauss weights of
    tau_2..tau_M on [0,1] (tau_1 = 0 carries no weight)."""
    M = order
    x, w = gauss_legendre(M - 1)
    tau = np.concatenate([[0.0], 0.5 + x])
    return tau, w


def appendix_a_rules():
    """Face rules of App. A on the reference triangle (unit sides) and the unit
    square, as printed (Eqs. A.1-A.6)."""
    s3 = np.sqrt(3.0)
    s5 = np.sqrt(5.0)
    g = 1.0 / s3
    A1 = (np.array([[1 / 4, 1 / (4 * s3)], [3 / 4, 1 / (4 * s3)], [1 / 2, 1 / s3]]),
          np.array([1 / 3, 1 / 3, 1 / 3]))
    A2 = (np.array([[(1 - g) / 2, (1 + g) / 2], [(1 + g) / 2, (1 + g) / 2],
                    [1 / 2, (1 - g) / 2]]), np.array([1 / 4, 1 / 4, 1 / 2]))
    A3 = (np.array([[1 / 8, 1 / (8 * s3)], [7 / 8, 1 / (8 * s3)], [1 / 2, 5 / (4 * s3)],
                    [3 / 8, s3 / 8], [5 / 8, s3 / 8], [1 / 2, s3 / 4]]),
          np.array([1 / 8, 1 / 8, 1 / 8, 5 / 24, 5 / 24, 5 / 24]))
    A4 = (np.array([[(1 - g) / 2, (1 - g) / 2], [(1 + g) / 2, (1 - g) / 2],
                    [(1 - g) / 2, (1 + g) / 2], [(1 + g) / 2, (1 + g) / 2]]),
          np.array([1 / 4] * 4))
    A5 = (np.array([[1 / 8, s3 / 24], [7 / 8, s3 / 24], [1 / 2, 5 * s3 / 12],
                    [3 / 8, s3 / 24], [5 / 8, s3 / 24], [3 / 4, s3 / 6],
                    [5 / 8, 7 * s3 / 24], [3 / 8, 7 * s3 / 24], [1 / 4, s3 / 6],
                    [1 / 2, s3 / 6]]),
          np.array([32 / 405] * 3 + [14 / 135] * 6 + [19 / 135]))
    h = s3 / s5
    A6 = (np.array([[(1 - g) / 2, (1 - h) / 2], [(1 + g) / 2, (1 - h) / 2],
                    [(1 - g) / 2, (1 + h) / 2], [(1 + g) / 2, (1 + h) / 2],
                    [(1 - g) / 2, 1 / 2], [(1 + g) / 2, 1 / 2]]),
          np.array([5 / 36] * 4 + [2 / 9] * 2))
    return {"A1": A1, "A2": A2, "A3": A3, "A4": A4, "A5": A5, "A6": A6}
