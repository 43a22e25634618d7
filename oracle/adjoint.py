"""Gradient of one LM step's solution delta through the linear solve.

delta solves H delta = g with H = J^T J + D and g = -J^T f (Section 2.1).  For a
cotangent vbar = dL/ddelta and mu = H^-1 vbar (H is symmetric), differentiating
H delta = g gives

    dL = mu^T (dg - dH delta)
       = -[ (dJ mu)^T f + (J mu)^T df + (dJ mu)^T (J delta) + (J mu)^T (dJ delta)
            + sum_k mu_k delta_k dD_kk ].

Observations enter only through f = pi - obs, so dL/dobs_o = (J mu)_o.  For the
camera and point parameters theta_o of observation o the bracket is the derivative
of  (J_o mu)^T f_o + (J_o mu)^T (J_o delta) + lam sum_k m_k mu_k delta_k |J_o[:,k]|^2
at fixed mu, delta (m_k = 1 where the Marquardt diagonal is above its floor).

The second derivatives of the residual are taken by the complex-step method
(Squire & Trapp 1998): d/dt J(theta + i h t).imag / h is exact to rounding.  mu is
obtained through the Schur complement with a dense solve of S (small problems).
"""
from __future__ import annotations

import numpy as np

from . import camera, schur
from .schur import DIAG_FLOOR

H_CS = 1e-30


def _jacobian_12(cams, pts, cam_idx, pt_idx):
    F, E = camera.jacobians(cams, pts, cam_idx, pt_idx)
    return np.concatenate([F, E], axis=2)           # [n_o, 2, 12]


def _directional_jacobian(cams, pts, cam_idx, pt_idx, dirs):
    """d/dt J_o(theta_o + t dirs_o) for per-observation directions dirs [n_o, 12]."""
    C = cams[cam_idx].astype(complex) + 1j * H_CS * dirs[:, :9]
    X = pts[pt_idx].astype(complex) + 1j * H_CS * dirs[:, 9:]
    n = len(cam_idx)
    idx = np.arange(n)
    F, E = camera.jacobians(C, X, idx, idx)
    return np.concatenate([F, E], axis=2).imag / H_CS


def solve_delta(sch: schur.Schur):
    """delta = [delta_c; delta_p] by a dense solve of S and back-substitution."""
    dc = np.linalg.solve(sch.S.toarray(), sch.b)
    return dc, sch.back_substitute(dc)


def adjoint(cams, pts, cam_idx, pt_idx, obs, lam, vbar, damping_mode="marquardt"):
    """Returns (dL/dobs [n_o,2], dL/dcams [n_c,9], dL/dpts [n_p,3], delta)."""
    n_c, n_p = cams.shape[0], pts.shape[0]
    sch = schur.linearize(cams, pts, cam_idx, pt_idx, obs, lam, damping_mode)
    dc, dp = solve_delta(sch)
    vc, vp = vbar[:9 * n_c], vbar[9 * n_c:]
    mu_c = np.linalg.solve(sch.S.toarray(), vc - sch.B @ (sch.Cinv @ vp))
    mu_p = sch.Cinv @ (vp - sch.B.T @ mu_c)
    J = _jacobian_12(cams, pts, cam_idx, pt_idx)
    f = sch.f
    mu_o = np.concatenate([mu_c.reshape(-1, 9)[cam_idx], mu_p.reshape(-1, 3)[pt_idx]], axis=1)
    de_o = np.concatenate([dc.reshape(-1, 9)[cam_idx], dp.reshape(-1, 3)[pt_idx]], axis=1)
    if damping_mode == "marquardt":
        dcj = np.asarray(sch.Fm.multiply(sch.Fm).sum(axis=0)).ravel().reshape(-1, 9)
        dpj = np.asarray(sch.Em.multiply(sch.Em).sum(axis=0)).ravel().reshape(-1, 3)
        m_o = np.concatenate([(dcj > DIAG_FLOOR)[cam_idx], (dpj > DIAG_FLOOR)[pt_idx]], axis=1)
    else:
        m_o = np.zeros_like(mu_o, dtype=bool)
    u = np.einsum("nik,nk->ni", J, mu_o)
    w = np.einsum("nik,nk->ni", J, de_o)
    h = f + w
    a = (mu_o[:, None, :] * h[:, :, None] + de_o[:, None, :] * u[:, :, None]
         + 2.0 * lam * (m_o * mu_o * de_o)[:, None, :] * J)          # [n_o, 2, 12]
    HV0 = _directional_jacobian(cams, pts, cam_idx, pt_idx, a[:, 0, :])[:, 0, :]
    HV1 = _directional_jacobian(cams, pts, cam_idx, pt_idx, a[:, 1, :])[:, 1, :]
    grad = HV0 + HV1 + np.einsum("nik,ni->nk", J, u)
    g_cam = np.zeros((n_c, 9))
    g_pt = np.zeros((n_p, 3))
    np.add.at(g_cam, cam_idx, -grad[:, :9])
    np.add.at(g_pt, pt_idx, -grad[:, 9:])
    return u, g_cam, g_pt, np.concatenate([dc, dp])
