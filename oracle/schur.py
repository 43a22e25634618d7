"""Damped normal equations, explicit Schur complement, reduced RHS (Section 2.1).

Literal transcription with SciPy sparse matrices:

    J = [F  E],  g = -J^T f                        (the RHS of Eq. 1, read as -J^T f)
    J^T J + D = [[A, F^T E], [E^T F, C]]           (Eq. 3)
    A = F^T F + D_c,  C = E^T E + D_p
    S = A - F^T E C^-1 E^T F                       (Section 2.1)
    b = g_c - F^T E C^-1 g_p                       (reduced right-hand side)
    delta_p = C^-1 (g_p - E^T F delta_c)           (back-substitution)

Damping (the paper only says "a diagonal damping matrix"): the reading taken
is Marquardt scaling, D = lam * max(diag(J^T J), 1e-6); ``damping='identity'``
gives D = lam * I instead.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

DIAG_FLOOR = 1e-6


def jacobian_matrices(F, E, cam_idx, pt_idx, n_cams, n_pts):
    """Sparse F (2n_o x 9n_c) and E (2n_o x 3n_p) from per-observation blocks."""
    n_o = F.shape[0]
    rows = np.arange(2 * n_o).reshape(n_o, 2)
    rF = np.repeat(rows[:, :, None], 9, axis=2)
    cF = np.broadcast_to((9 * cam_idx[:, None, None] + np.arange(9)[None, None, :]), (n_o, 2, 9))
    Fm = sp.csr_matrix((F.ravel(), (rF.ravel(), cF.ravel())), shape=(2 * n_o, 9 * n_cams))
    rE = np.repeat(rows[:, :, None], 3, axis=2)
    cE = np.broadcast_to((3 * pt_idx[:, None, None] + np.arange(3)[None, None, :]), (n_o, 2, 3))
    Em = sp.csr_matrix((E.ravel(), (rE.ravel(), cE.ravel())), shape=(2 * n_o, 3 * n_pts))
    return Fm, Em


def damping(Fm, Em, lam, damping="marquardt"):
    """Diagonal damping (D_c, D_p) as vectors."""
    if damping == "identity":
        return (np.full(Fm.shape[1], lam), np.full(Em.shape[1], lam))
    dc = np.asarray(Fm.multiply(Fm).sum(axis=0)).ravel()
    dp = np.asarray(Em.multiply(Em).sum(axis=0)).ravel()
    return lam * np.maximum(dc, DIAG_FLOOR), lam * np.maximum(dp, DIAG_FLOOR)


def block_diag_inverse(M, b):
    """Inverse of a block-diagonal sparse matrix with b x b blocks; also returns the blocks."""
    n = M.shape[0] // b
    blocks = np.zeros((n, b, b))
    Mc = M.tocoo()
    bi = Mc.row // b
    if np.any(bi != Mc.col // b):
        raise ValueError("matrix is not block diagonal")
    blocks[bi, Mc.row % b, Mc.col % b] = Mc.data
    inv = np.linalg.inv(blocks)
    return blockdiag_sparse(inv), blocks, inv


def blockdiag_sparse(blocks):
    n, b, _ = blocks.shape
    r = (np.arange(n)[:, None, None] * b + np.arange(b)[None, :, None]) + np.zeros((1, 1, b), int)
    c = (np.arange(n)[:, None, None] * b + np.arange(b)[None, None, :]) + np.zeros((1, b, 1), int)
    return sp.csr_matrix((blocks.ravel(), (r.ravel(), c.ravel())), shape=(n * b, n * b))


class Schur:
    """All pieces of one linearisation's reduced camera system."""

    def __init__(self, F, E, f, cam_idx, pt_idx, n_cams, n_pts, lam, damping_mode="marquardt",
                 explicit=True):
        self.n_cams, self.n_pts = n_cams, n_pts
        self.Fb, self.Eb, self.f = F, E, f
        self.cam_idx, self.pt_idx = cam_idx, pt_idx
        self.lam = lam
        Fm, Em = jacobian_matrices(F, E, cam_idx, pt_idx, n_cams, n_pts)
        self.Fm, self.Em = Fm, Em
        self.Dc, self.Dp = damping(Fm, Em, lam, damping_mode)
        fr = f.ravel()
        self.g_c = -(Fm.T @ fr)
        self.g_p = -(Em.T @ fr)
        self.A = (Fm.T @ Fm + sp.diags(self.Dc)).tocsr()
        self.C = (Em.T @ Em + sp.diags(self.Dp)).tocsr()
        self.Cinv, self.C_blocks, self.Cinv_blocks = block_diag_inverse(self.C, 3)
        self.B = (Fm.T @ Em).tocsr()                       # F^T E
        self.S = None
        if explicit:                                       # large problems use the implicit product
            self.S = (self.A - self.B @ self.Cinv @ self.B.T).tocsr()
            self.S.sum_duplicates()
        self.b = self.g_c - self.B @ (self.Cinv @ self.g_p)

    def implicit_matvec(self, x):
        """S x = A x - F^T (E (C^-1 (E^T (F x))))  (Section 3.6)."""
        Fx = self.Fm @ x
        return self.A @ x - self.Fm.T @ (self.Em @ (self.Cinv @ (self.Em.T @ Fx)))

    def back_substitute(self, delta_c):
        return self.Cinv @ (self.g_p - self.B.T @ delta_c)

    def dense_normal_solve(self):
        """Solve (J^T J + D) delta = g densely (small problems only)."""
        J = sp.hstack([self.Fm, self.Em]).toarray()
        H = J.T @ J + np.diag(np.concatenate([self.Dc, self.Dp]))
        g = np.concatenate([self.g_c, self.g_p])
        return np.linalg.solve(H, g)

    def model_reduction(self, delta_c, delta_p):
        """L(0) - L(delta) of the damped quadratic model: 1/2 (delta.g + delta.D.delta)."""
        dg = delta_c @ self.g_c + delta_p @ self.g_p
        dDd = delta_c @ (self.Dc * delta_c) + delta_p @ (self.Dp * delta_p)
        return 0.5 * (dg + dDd)


def linearize(cams, pts, cam_idx, pt_idx, obs, lam, damping_mode="marquardt", explicit=True, huber=None):
    """huber = a: residuals and Jacobian rows scaled by sqrt(loss'(|f_o|^2)) of the Huber
    loss with scale a (see oracle/robust.py); None: the squared loss."""
    from . import camera, robust
    f = camera.residuals(cams, pts, cam_idx, pt_idx, obs)
    F, E = camera.jacobians(cams, pts, cam_idx, pt_idx)
    if huber is not None:
        w = robust.weights(f, huber)
        f = f * w[:, None]
        F = F * w[:, None, None]
        E = E * w[:, None, None]
    return Schur(F, E, f, cam_idx, pt_idx, cams.shape[0], pts.shape[0], lam, damping_mode, explicit)
