"""Pins of the oracle's fluxes and Riemann solvers (Eq. 2.2; readings of Sec. VI)."""
import numpy as np
import pytest

from oracle import physics as ph

G = 5.0 / 3.0


def rand_state(rng, n=1):
    rho = rng.uniform(0.5, 2.0, n)
    v = rng.uniform(-1, 1, (n, 3))
    p = rng.uniform(0.2, 2.0, n)
    B = rng.uniform(-1, 1, (n, 3))
    return ph.conserved(rho, v, p, B, G)


def rot(rng):
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return q * np.sign(np.linalg.det(q))


def rotate_state(U, Q):
    V = U.copy()
    V[..., 1:4] = U[..., 1:4] @ Q.T
    V[..., 5:8] = U[..., 5:8] @ Q.T
    return V


def test_flux_matches_eq_2_2_along_x():
    rng = np.random.default_rng(0)
    U = rand_state(rng)[0]
    rho, v, p, B = ph.primitives(U, G)
    pt = p + 0.5 * B @ B
    F = ph.flux_dir(U, np.array([1.0, 0, 0]), G)
    expect = [rho * v[0], rho * v[0] ** 2 + pt - B[0] ** 2, rho * v[0] * v[1] - B[0] * B[1],
              rho * v[0] * v[2] - B[0] * B[2], (U[4] + pt) * v[0] - B[0] * (v @ B), 0.0,
              v[0] * B[1] - v[1] * B[0], -(v[2] * B[0] - v[0] * B[2])]
    assert np.allclose(F, expect, atol=1e-14)


def test_hll_consistency_and_rotation():
    rng = np.random.default_rng(1)
    UL, UR = rand_state(rng, 2)
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    assert np.allclose(ph.hll(UL, UL, n, G), ph.flux_dir(UL, n, G), atol=1e-13)
    Q = rot(rng)
    F = ph.hll(UL, UR, n, G)
    Fr = ph.hll(rotate_state(UL, Q), rotate_state(UR, Q), Q @ n, G)
    Fb = F.copy()
    Fb[1:4] = Q @ F[1:4]
    Fb[5:8] = Q @ F[5:8]
    assert np.allclose(Fr, Fb, atol=1e-12)


def test_hll_upwinds_supersonic_flow():
    rng = np.random.default_rng(2)
    UL, UR = rand_state(rng, 2)
    n = np.array([1.0, 0, 0])
    for U in (UL, UR):
        U[1:4] = U[0] * np.array([20.0, 0, 0])
        U[4] = 1.0 / (G - 1) + 0.5 * U[0] * 400.0 + 0.5 * U[5:8] @ U[5:8]
    assert np.allclose(ph.hll(UL, UR, n, G), ph.flux_dir(UL, n, G), atol=1e-12)


def test_edge_emf_identical_states_is_minus_v_cross_b():
    rng = np.random.default_rng(3)
    U = rand_state(rng)[0]
    t = np.array([0.0, 0.0, 1.0])
    faces = [(0, 1, np.array([1.0, 0, 0])), (1, 2, np.array([0, 1.0, 0]))]
    st = np.stack([U] * 4)
    rho, v, p, B = ph.primitives(U, G)
    assert abs(ph.edge_emf(st, faces, t, G) - (-np.cross(v, B)) @ t) < 1e-14


def test_edge_emf_reduces_to_1d_rusanov():
    """Four zones around a z edge, states varying only in x: the EMF equals the 1D
    Rusanov flux of the induction equation for B_y (E_z = -F(B_y))."""
    rng = np.random.default_rng(4)
    UW, UE = rand_state(rng, 2)
    # zones: 0 = SW, 1 = SE, 2 = NE, 3 = NW ; faces between W and E have normal +x
    st = np.stack([UW, UE, UE, UW])
    x, y = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    faces = [(0, 1, x), (3, 2, x), (0, 3, y), (1, 2, y)]
    t = np.array([0, 0, 1.0])
    E = ph.edge_emf(st, faces, t, G)
    a = max(ph.rusanov_speed(UW, x, G), ph.rusanov_speed(UE, x, G))
    FW = ph.flux_dir(UW, x, G)[6]
    FE = ph.flux_dir(UE, x, G)[6]
    rus = 0.5 * (FW + FE) - 0.5 * a * (UE[6] - UW[6])
    assert abs(E - (-rus)) < 1e-13


# ---------------------------------------------------------------- HLLD
def _state(rho, v, p, B, g=5.0 / 3.0):
    from oracle.physics import conserved
    return conserved(np.array(rho), np.array(v, dtype=float), np.array(p), np.array(B, dtype=float), g)


def test_hlld_consistency_and_supersonic_upwinding():
    """Identical states give the physical flux; a supersonic flow gives the
    upwind flux (Miyoshi & Kusano 2005, consistency and upwinding)."""
    from oracle.physics import flux_dir, hlld
    g = 5.0 / 3.0
    n = np.array([0.6, 0.0, 0.8])
    U = _state(1.2, [0.3, -0.2, 0.1], 0.9, [0.4, 0.5, -0.3])
    assert np.abs(hlld(U, U, n, g) - flux_dir(U, n, g)).max() < 1e-15
    UL = _state(1.0, 8.0 * n, 0.5, [0.2, 0.1, 0.0])
    UR = _state(0.5, 7.0 * n, 0.3, [0.1, 0.3, -0.2])
    # upwinding: the left state with the mean normal field
    ex = _state(1.0, 8.0 * n, 0.5, [0.2, 0.1, 0.0] + (0.5 * (0.12 + (0.06 - 0.16)) - 0.12) * n)
    assert np.abs(hlld(UL, UR, n, g) - flux_dir(ex, n, g)).max() < 1e-13


def test_hlld_rotation_invariance():
    from oracle.physics import hlld
    g = 5.0 / 3.0
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    n = np.array([0.0, 0.6, 0.8])
    UL = _state(1.0, [0.2, -0.1, 0.3], 1.0, [0.5, 0.3, -0.4])
    UR = _state(0.3, [-0.4, 0.2, 0.0], 0.2, [0.1, -0.6, 0.2])

    def rot(U):
        V = U.copy()
        V[1:4] = Q @ U[1:4]
        V[5:8] = Q @ U[5:8]
        return V

    a = hlld(rot(UL), rot(UR), Q @ n, g)
    b = rot(hlld(UL, UR, n, g))
    assert np.abs(a - b).max() < 1e-13


@pytest.mark.parametrize("Bn", [0.0, 0.7])
def test_hlld_resolves_a_stationary_contact(Bn):
    """A stationary contact (density jump, equal pressure, continuous tangential
    v and B) carries no mass: the HLLD flux is the exact flux, while HLL
    diffuses it."""
    from oracle.physics import flux_dir, hll, hlld
    g = 5.0 / 3.0
    n = np.array([1.0, 0.0, 0.0])
    UL = _state(1.0, [0.0, 0.3, 0.1], 1.0, [Bn, 0.5, 0.2])
    UR = _state(0.2, [0.0, 0.3, 0.1], 1.0, [Bn, 0.5, 0.2])
    assert np.abs(hlld(UL, UR, n, g) - flux_dir(UL, n, g)).max() < 1e-14
    assert abs(hll(UL, UR, n, g)[0]) > 0.1


@pytest.mark.parametrize("sgn", [1.0, -1.0])
def test_hlld_resolves_an_isolated_alfven_discontinuity(sgn):
    """A rotational discontinuity: equal rho, p, B_n and |B_t|, tangential field
    rotated and [v_t] = sgn [B_t] / sqrt(rho).  With sgn = -1 (B_n > 0) it moves
    to the right, and the flux at the interface is the left state's; with sgn = +1
    it moves left and the flux is the right state's.  HLLD returns either exactly."""
    from oracle.physics import flux_dir, hlld
    g = 5.0 / 3.0
    n = np.array([1.0, 0.0, 0.0])
    BtL, BtR, vtL = np.array([0.6, 0.0]), np.array([0.0, 0.6]), np.array([0.1, -0.2])
    vtR = vtL + sgn * (BtR - BtL)
    UL = _state(1.0, [0.0, *vtL], 1.0, [0.8, *BtL])
    UR = _state(1.0, [0.0, *vtR], 1.0, [0.8, *BtR])
    up = UL if sgn < 0 else UR
    assert np.abs(hlld(UL, UR, n, g) - flux_dir(up, n, g)).max() < 1e-14
