"""Positivity limiting of point states (Sec. I: WENO "ruggedized to have a
positivity-preserving property", details in Balsara 2012b, not available) -- oracle.

Reading taken: a scaling limiter of the Zhang-Shu type.  For one zone with mean
state Ubar (zone averages, B from the divergence-free means) and point states
U_q (the initial nodal states of the predictor, or the predicted states at the
zone's face and edge points and Gauss times):
  theta_rho = min(1, min over q with rho_q < eps_rho of (rhobar - eps_rho)/(rhobar - rho_q))
  U'_q      = Ubar + theta_rho (U_q - Ubar)
  theta_p   = min(1, min over q with p(U'_q) < eps_p of (pbar - eps_p)/(pbar - p(U'_q)))
  U''_q     = Ubar + theta_rho theta_p (U_q - Ubar)
with eps_rho = min(1e-13, rhobar), eps_p = min(1e-13, pbar).  Pressure is a
concave function of the conserved variables, so (1-t) pbar + t p(U'_q) is a lower
bound of p along the segment and the scaled states keep p >= eps_p.

Pinned by: tests/test_oracle_positivity.py -- states that are already positive are
untouched, limited states satisfy rho, p >= eps, the mean is unchanged, and the
limiter is exactly the identity when theta = 1 (zones with theta = 1 are left
bit-for-bit unchanged).
"""
import numpy as np

from .physics import primitives


def limit(states, mean, gamma):
    """states (Z, n, 8), mean (Z, 8) -> limited states and theta (Z,)."""
    rho_b = mean[:, 0]
    p_b = primitives(mean, gamma)[2]
    eps_r = np.minimum(1e-13, rho_b)
    eps_p = np.minimum(1e-13, p_b)
    d = states - mean[:, None, :]
    rho = states[..., 0]
    with np.errstate(divide="ignore", invalid="ignore"):
        tr = np.where(rho < eps_r[:, None], (rho_b - eps_r)[:, None] / (rho_b[:, None] - rho), 1.0)
    th_r = np.minimum(1.0, tr.min(axis=1))
    s1 = mean[:, None, :] + th_r[:, None, None] * d
    p1 = primitives(s1, gamma)[2]
    with np.errstate(divide="ignore", invalid="ignore"):
        tp = np.where(p1 < eps_p[:, None], (p_b - eps_p)[:, None] / (p_b[:, None] - p1), 1.0)
    th_p = np.minimum(1.0, tp.min(axis=1))
    theta = th_r * th_p
    lim = np.where((theta < 1.0)[:, None, None], mean[:, None, :] + theta[:, None, None] * d, states)
    return lim, theta
