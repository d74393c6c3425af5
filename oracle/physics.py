"""Ideal MHD fluxes (Eq. 2.2), the 1D HLL Riemann solver and the multidimensional
edge electric field -- oracle version.

Units: rationalised (Heaviside-Lorentz): the Gaussian factors 1/(4 pi) and
1/(8 pi) of Eq. 2.2 become 1 and 1/2; B_G = sqrt(4 pi) B_HL.  Conserved
variables U = (rho, rho v, eps, B) with eps = rho v^2/2 + P/(gamma-1) + B^2/2.

Readings (the paper does not name its solvers):
  * 1D Riemann solver at face points (Sec. VI step 5): HLL with Davis wave speeds
    S_L = min(vn_L - cf_L, vn_R - cf_R), S_R = max(vn_L + cf_L, vn_R + cf_R),
    cf the fast magnetosonic speed along the unit normal; all 8 components.
  * Multidimensional Riemann solver at edge points (MuSIC in the paper): a
    multidimensional Rusanov electric field for the k zones around an edge with
    unit tangent t,
      E.t = (1/k) [ sum_z (-v_z x B_z).t + sum_f a_f (B_R(f) - B_L(f)).(t x n_f) ],
    a_f = max(|vn| + cf) of the two states of face f along its unit normal n_f.
    It reduces to the 2D Rusanov/UCT field on an orthogonal 4-zone edge and to
    -v x B for identical states.
  * Optional higher-fidelity face solver (Sec. I names such solvers without
    choosing one): HLLD (Miyoshi & Kusano 2005) with the same fast-wave speeds,
    the normal field taken as the mean of the two sides'.

Pinned by: tests/test_oracle_physics.py -- consistency (identical states give the
exact flux / -v x B), rotational invariance, HLL equal to upwind flux for
supersonic states, the 4-zone Cartesian reduction to 1D Rusanov induction; HLLD:
consistency, supersonic upwinding, rotational invariance, exact fluxes of an
isolated stationary contact (with and without normal field, where HLL diffuses)
and of an isolated rotational discontinuity moving either way.
"""
import numpy as np

RHO, MX, MY, MZ, EN, BX, BY, BZ = range(8)

# Optional branch recorder (tests use it to detect finite-difference stencils that
# cross a MinMod / HLL / max switch): a list that the branchy routines append to.
# Each entry holds signed margins, normalised to O(1) scales: the sign of a margin
# is the branch taken, its size the relative distance to the switch.
BRANCHES = None


def record(tag, margins):
    if BRANCHES is not None:
        BRANCHES.append((tag, np.asarray(margins, dtype=np.float64).copy()))


def primitives(U, gamma):
    rho = U[..., RHO]
    v = U[..., MX:MZ + 1] / rho[..., None]
    B = U[..., BX:BZ + 1]
    p = (gamma - 1.0) * (U[..., EN] - 0.5 * rho * (v * v).sum(-1) - 0.5 * (B * B).sum(-1))
    return rho, v, p, B


def conserved(rho, v, p, B, gamma):
    U = np.zeros(np.shape(rho) + (8,))
    U[..., RHO] = rho
    U[..., MX:MZ + 1] = rho[..., None] * v
    U[..., EN] = p / (gamma - 1.0) + 0.5 * rho * (v * v).sum(-1) + 0.5 * (B * B).sum(-1)
    U[..., BX:BZ + 1] = B
    return U


def flux_dir(U, nvec, gamma):
    """Physical flux F(U).n for an arbitrary (not necessarily unit) vector n."""
    rho, v, p, B = primitives(U, gamma)
    vn = (v * nvec).sum(-1)
    Bn = (B * nvec).sum(-1)
    pt = p + 0.5 * (B * B).sum(-1)
    vB = (v * B).sum(-1)
    F = np.empty_like(U)
    F[..., RHO] = rho * vn
    F[..., MX:MZ + 1] = rho[..., None] * v * vn[..., None] + pt[..., None] * nvec - B * Bn[..., None]
    F[..., EN] = (U[..., EN] + pt) * vn - Bn * vB
    F[..., BX:BZ + 1] = B * vn[..., None] - v * Bn[..., None]
    return F


def fast_speed(U, nhat, gamma):
    rho, v, p, B = primitives(U, gamma)
    a2 = gamma * p / rho
    b2 = (B * B).sum(-1) / rho
    bn2 = (B * nhat).sum(-1) ** 2 / rho
    s = a2 + b2
    return np.sqrt(0.5 * (s + np.sqrt(np.maximum(s * s - 4.0 * a2 * bn2, 0.0))))


def hll(UL, UR, nhat, gamma):
    """HLL flux along the unit normal nhat."""
    vnL = (UL[..., MX:MZ + 1] * nhat).sum(-1) / UL[..., RHO]
    vnR = (UR[..., MX:MZ + 1] * nhat).sum(-1) / UR[..., RHO]
    cL = fast_speed(UL, nhat, gamma)
    cR = fast_speed(UR, nhat, gamma)
    SL = np.minimum(vnL - cL, vnR - cR)
    SR = np.maximum(vnL + cL, vnR + cR)
    FL = flux_dir(UL, nhat, gamma)
    FR = flux_dir(UR, nhat, gamma)
    Fs = (SR[..., None] * FL - SL[..., None] * FR
          + (SL * SR)[..., None] * (UR - UL)) / (SR - SL)[..., None]
    out = np.where((SL >= 0.0)[..., None], FL, np.where((SR <= 0.0)[..., None], FR, Fs))
    if BRANCHES is not None:
        sc = np.abs(vnL) + cL + np.abs(vnR) + cR
        record("hll", np.stack([SL / sc, -SR / sc, ((vnR - cR) - (vnL - cL)) / sc,
                                ((vnL + cL) - (vnR + cR)) / sc]))
    return out


def hlld(UL, UR, nhat, gamma):
    """HLLD flux along the unit normal nhat (Miyoshi & Kusano 2005): five waves,
    the fast waves S_L, S_R (Davis speeds, as in hll), the Alfven waves S*_L, S*_R
    and the entropy wave S_M, with the total pressure constant across the Riemann
    fan.  The normal field is the mean of the two sides' normal fields (each
    state takes it, keeping its pressure).  Tangential vectors are handled as
    3-vectors orthogonal to nhat, so no tangent basis is chosen.  Degenerate
    cases: where rho (S - u)(S - S_M) = B_n^2 the tangential fields are left
    unchanged across the fast wave, and where B_n^2 vanishes the Alfven waves
    collapse onto S_M (the ** states equal the * states)."""
    n = nhat
    g = gamma
    rL, vL, pL, BL = primitives(UL, g)
    rR, vR, pR, BR = primitives(UR, g)
    Bn = 0.5 * ((BL * n).sum(-1) + (BR * n).sum(-1))
    BL = BL + (Bn - (BL * n).sum(-1))[..., None] * n
    BR = BR + (Bn - (BR * n).sum(-1))[..., None] * n
    UL = conserved(rL, vL, pL, BL, g)
    UR = conserved(rR, vR, pR, BR, g)
    uL, uR = (vL * n).sum(-1), (vR * n).sum(-1)
    ptL = pL + 0.5 * (BL * BL).sum(-1)
    ptR = pR + 0.5 * (BR * BR).sum(-1)
    cL, cR = fast_speed(UL, n, g), fast_speed(UR, n, g)
    SL = np.minimum(uL - cL, uR - cR)
    SR = np.maximum(uL + cL, uR + cR)
    dL, dR = (SL - uL) * rL, (SR - uR) * rR
    SM = (dR * uR - dL * uL - ptR + ptL) / (dR - dL)
    pts = (dR * ptL - dL * ptR + dL * dR * (uR - uL)) / (dR - dL)
    Bn2 = Bn * Bn

    def star(r, v, u, B, U, S, d, pt):
        rs = d / (S - SM)
        vt = v - u[..., None] * n
        Bt = B - Bn[..., None] * n
        den = d * (S - SM) - Bn2
        ok = np.abs(den) > 1e-12 * (np.abs(d * (S - SM)) + Bn2)
        safe = np.where(ok, den, 1.0)
        vts = np.where(ok[..., None], vt - (Bn * (SM - u) / safe)[..., None] * Bt, vt)
        Bts = np.where(ok[..., None], Bt * ((d * (S - u) - Bn2) / safe)[..., None], Bt)
        vs = SM[..., None] * n + vts
        Bs = Bn[..., None] * n + Bts
        E = U[..., EN]
        Es = ((S - u) * E - pt * u + pts * SM + Bn * ((v * B).sum(-1) - (vs * Bs).sum(-1))) / (S - SM)
        Us = np.empty_like(U)
        Us[..., RHO] = rs
        Us[..., MX:MZ + 1] = rs[..., None] * vs
        Us[..., EN] = Es
        Us[..., BX:BZ + 1] = Bs
        return Us, vts, Bts

    UsL, vtL, BtL = star(rL, vL, uL, BL, UL, SL, dL, ptL)
    UsR, vtR, BtR = star(rR, vR, uR, BR, UR, SR, dR, ptR)
    sL, sR = np.sqrt(UsL[..., RHO]), np.sqrt(UsR[..., RHO])
    SsL = SM - np.abs(Bn) / sL
    SsR = SM + np.abs(Bn) / sR
    sg = np.sign(Bn)[..., None]
    w = (sL + sR)[..., None]
    vtt = (sL[..., None] * vtL + sR[..., None] * vtR + (BtR - BtL) * sg) / w
    Btt = (sL[..., None] * BtR + sR[..., None] * BtL + (sL * sR)[..., None] * (vtR - vtL) * sg) / w
    vss = SM[..., None] * n + vtt
    Bss = Bn[..., None] * n + Btt
    vBss = (vss * Bss).sum(-1)
    mag = Bn2 > 1e-12 * (pts + 1e-300)

    def dstar(Us, s, sign):
        Uss = Us.copy()
        vs = Us[..., MX:MZ + 1] / Us[..., RHO][..., None]
        Bs = Us[..., BX:BZ + 1]
        Uss[..., MX:MZ + 1] = Us[..., RHO][..., None] * vss
        Uss[..., BX:BZ + 1] = Bss
        Uss[..., EN] = Us[..., EN] + sign * s * ((vs * Bs).sum(-1) - vBss) * np.sign(Bn)
        return np.where(mag[..., None], Uss, Us)

    UssL = dstar(UsL, sL, -1.0)
    UssR = dstar(UsR, sR, 1.0)
    FL, FR = flux_dir(UL, n, g), flux_dir(UR, n, g)
    FsL = FL + SL[..., None] * (UsL - UL)
    FsR = FR + SR[..., None] * (UsR - UR)
    FssL = FsL + SsL[..., None] * (UssL - UsL)
    FssR = FsR + SsR[..., None] * (UssR - UsR)
    out = np.where((SL > 0.0)[..., None], FL,
          np.where((SsL > 0.0)[..., None], FsL,
          np.where((SM > 0.0)[..., None], FssL,
          np.where((SsR > 0.0)[..., None], FssR,
          np.where((SR > 0.0)[..., None], FsR, FR)))))
    if BRANCHES is not None:
        sc = np.abs(uL) + cL + np.abs(uR) + cR
        record("hlld", np.stack([SL / sc, SsL / sc, SM / sc, SsR / sc, SR / sc,
                                 ((uR - cR) - (uL - cL)) / sc, ((uL + cL) - (uR + cR)) / sc]))
    return out


def rusanov_speed(U, nhat, gamma):
    vn = (U[..., MX:MZ + 1] * nhat).sum(-1) / U[..., RHO]
    return np.abs(vn) + fast_speed(U, nhat, gamma)


def edge_emf(states, faces, tvec, gamma):
    """Multidimensional Rusanov E.t at one edge point.

    states: (k, 8) zone states; faces: list of (iL, iR, nhat(3,)); tvec unit tangent."""
    k = states.shape[0]
    rho = states[:, RHO]
    v = states[:, MX:MZ + 1] / rho[:, None]
    B = states[:, BX:BZ + 1]
    E = -np.cross(v, B)
    acc = (E @ tvec).sum()
    for iL, iR, nh in faces:
        aL, aR = rusanov_speed(states[iL], nh, gamma), rusanov_speed(states[iR], nh, gamma)
        if BRANCHES is not None:
            vL = states[iL][MX:MZ + 1] @ nh / states[iL][RHO]
            vR = states[iR][MX:MZ + 1] @ nh / states[iR][RHO]
            record("emf", [(aL - aR) / (aL + aR), vL / aL, vR / aR])
        a = max(aL, aR)
        acc += a * np.dot(B[iR] - B[iL], np.cross(tvec, nh))
    return acc / k
