"""Residuals and analytic Jacobians of the 9-parameter reprojection model.

The paper fixes only that the camera has 9 parameters and a reprojection
residual (Section 6) and uses the BAL datasets (Section 4).  The reading taken
here is the BAL/Snavely model:

    cam = [r (angle-axis, 3), t (3), f, k1, k2]
    P   = R(r) X + t                  (Rodrigues rotation)
    p   = -P_xy / P_z                 (camera looks down -z)
    d   = 1 + k1 |p|^2 + k2 |p|^4
    f_o = f d p - obs_o               (residual of observation o)

Small-angle branch: when theta^2 = r.r < 1e-16 the rotation is taken to first
order, R X = X + r x X, with Jacobian -[X]_x in r.

The Jacobian in r is obtained by differentiating the Rodrigues formula
    R X = cos(th) X + (sin(th)/th) (r x X) + ((1-cos(th))/th^2) (r.X) r
term by term (product and chain rules).
"""
from __future__ import annotations

import numpy as np

SMALL_ANGLE_EPS = 1e-16


def _cross(a, b):
    return np.cross(a, b)


def rotate(r: np.ndarray, X: np.ndarray) -> np.ndarray:
    """R(r) X for row-stacked angle-axis vectors r and points X ([n, 3])."""
    th2 = np.sum(r * r, axis=1)
    small = np.real(th2) < SMALL_ANGLE_EPS   # real part: complex-step safe
    th = np.sqrt(np.where(small, 1.0, th2))
    c = np.cos(th)
    s = np.sin(th)
    alpha = s / th
    beta = (1.0 - c) / (th * th)
    rdX = np.sum(r * X, axis=1)
    full = c[:, None] * X + alpha[:, None] * _cross(r, X) + (beta * rdX)[:, None] * r
    first = X + _cross(r, X)
    return np.where(small[:, None], first, full)


def _skew(v):
    z = np.zeros(v.shape[0])
    return np.stack([np.stack([z, -v[:, 2], v[:, 1]], 1),
                     np.stack([v[:, 2], z, -v[:, 0]], 1),
                     np.stack([-v[:, 1], v[:, 0], z], 1)], 1)


def rotate_jacobians(r, X):
    """(d(RX)/dr, d(RX)/dX), each [n, 3, 3]."""
    n = r.shape[0]
    th2 = np.sum(r * r, axis=1)
    small = np.real(th2) < SMALL_ANGLE_EPS   # real part: complex-step safe
    th = np.sqrt(np.where(small, 1.0, th2))
    c = np.cos(th)
    s = np.sin(th)
    alpha = s / th                              # sin/th
    beta = (1.0 - c) / (th * th)                # (1-cos)/th^2
    dalpha = (c * th - s) / (th * th)           # d alpha / d th
    dbeta = (s * th - 2.0 * (1.0 - c)) / th ** 3  # d beta / d th
    k = r / th[:, None]                         # d th / d r
    rxX = _cross(r, X)
    rdX = np.sum(r * X, axis=1)
    eye = np.broadcast_to(np.eye(3), (n, 3, 3))
    # d/dr [cos(th) X]            = -sin(th) X k^T
    # d/dr [alpha (r x X)]        = dalpha (r x X) k^T + alpha (-[X]_x)
    # d/dr [beta (r.X) r]         = dbeta (r.X) r k^T + beta r X^T + beta (r.X) I
    dr = (-s[:, None, None] * np.einsum("ni,nj->nij", X, k)
          + dalpha[:, None, None] * np.einsum("ni,nj->nij", rxX, k)
          - alpha[:, None, None] * _skew(X)
          + (dbeta * rdX)[:, None, None] * np.einsum("ni,nj->nij", r, k)
          + beta[:, None, None] * np.einsum("ni,nj->nij", r, X)
          + (beta * rdX)[:, None, None] * eye)
    dX = (c[:, None, None] * eye + alpha[:, None, None] * _skew(r)
          + beta[:, None, None] * np.einsum("ni,nj->nij", r, r))
    dr_small = -_skew(X)
    dX_small = eye + _skew(r)
    dr = np.where(small[:, None, None], dr_small, dr)
    dX = np.where(small[:, None, None], dX_small, dX)
    return dr, dX


def project(cams: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Predicted pixel coordinates pi(cam, X) for row-matched cams [n,9], X [n,3]."""
    P = rotate(cams[:, 0:3], X) + cams[:, 3:6]
    p = -P[:, 0:2] / P[:, 2:3]
    r2 = np.sum(p * p, axis=1)
    d = 1.0 + cams[:, 7] * r2 + cams[:, 8] * r2 * r2
    return (cams[:, 6] * d)[:, None] * p


def residuals(cams, pts, cam_idx, pt_idx, obs):
    """f_o = pi(cam_c, X_p) - obs_o for every observation o = (c, p); [n_obs, 2]."""
    return project(cams[cam_idx], pts[pt_idx]) - obs


def cost(cams, pts, cam_idx, pt_idx, obs, huber=None) -> float:
    """Objective 1/2 sum_o |f_o|^2 (the squared sum of Section 2.1); with huber = a, the
    robust objective 1/2 sum_o loss(|f_o|^2) of Section 5."""
    f = residuals(cams, pts, cam_idx, pt_idx, obs)
    if huber is not None:
        from . import robust
        return robust.cost(f, huber)
    return 0.5 * float(np.sum(f * f))


def jacobians(cams, pts, cam_idx, pt_idx):
    """Per-observation blocks F_o = d f_o / d cam (2x9) and E_o = d f_o / d X (2x3)."""
    C = cams[cam_idx]
    X = pts[pt_idx]
    r = C[:, 0:3]
    P = rotate(r, X) + C[:, 3:6]
    dPdr, dPdX = rotate_jacobians(r, X)
    iz = 1.0 / P[:, 2]
    p = -P[:, 0:2] * iz[:, None]
    n = len(iz)
    # dp/dP (2x3)
    dpdP = np.zeros((n, 2, 3), dtype=P.dtype)
    dpdP[:, 0, 0] = -iz
    dpdP[:, 1, 1] = -iz
    dpdP[:, 0, 2] = P[:, 0] * iz * iz
    dpdP[:, 1, 2] = P[:, 1] * iz * iz
    f, k1, k2 = C[:, 6], C[:, 7], C[:, 8]
    r2 = np.sum(p * p, axis=1)
    d = 1.0 + k1 * r2 + k2 * r2 * r2
    dd_dp = (2.0 * (k1 + 2.0 * k2 * r2))[:, None] * p          # gradient of d in p
    dpi_dp = f[:, None, None] * (d[:, None, None] * np.eye(2)[None]
                                 + np.einsum("ni,nj->nij", p, dd_dp))
    dpi_dP = np.einsum("nij,njk->nik", dpi_dp, dpdP)
    F = np.zeros((n, 2, 9), dtype=P.dtype)
    F[:, :, 0:3] = np.einsum("nij,njk->nik", dpi_dP, dPdr)
    F[:, :, 3:6] = dpi_dP
    F[:, :, 6] = d[:, None] * p
    F[:, :, 7] = (f * r2)[:, None] * p
    F[:, :, 8] = (f * r2 * r2)[:, None] * p
    E = np.einsum("nij,njk->nik", dpi_dP, dPdX)
    return F, E
