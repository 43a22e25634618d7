"""Unsmoothed-aggregation multigrid of Section 3, in plain NumPy/SciPy (FP64).

Readings of the paper taken here (where it is silent or ambiguous):

* Strength of connection (Section 3.2): G_ij = v_i.v_j / (|v_i| |v_j|) with
  binary visibility v.  With the integer covisibility counts W = V^T V this is
  W_ij / sqrt(W_ii W_jj); neighbours j of i are ordered by decreasing G_ij using
  the exact integer comparison W_ij^2 W_kk > W_ik^2 W_jj, ties to the smaller
  index.  Coarse levels use W_{l+1} = Agg^T W_l Agg (visibility of the summed
  aggregate visibility vectors).
* Algorithm 2 with the size cap 20; a node left unaggregated after the pass
  becomes a singleton aggregate, numbered after all others in node order.
* Near-nullspace (Section 3.1): the 7 similarity gauge modes restricted to the
  cameras plus 9 per-parameter constant columns, in the column order
  [tx, ty, tz, rx, ry, rz, s, const_0..const_8].
* Tentative prolongator (Section 3.3): per-aggregate thin QR by modified
  Gram-Schmidt with one re-orthogonalisation pass; a column whose remaining
  norm is below 1e-10 of its original norm is dropped (zero column of Q, zero
  row of R).  Blocks stay 16 wide; a dropped coarse dof gets diagonal 1 in the
  Galerkin operator.
* Hierarchy depth: coarsen while a level has more than ``coarse_max_nodes``
  nodes and fewer than ``max_levels`` levels exist; the coarsest level is
  solved directly (dense Cholesky here).
* Smoother (Section 3.4): two steps of Chebyshev semi-iteration (Saad,
  Iterative Methods, Alg. 12.1) preconditioned by point-block Jacobi on
  [0.3, 1.1] * lambda_max, lambda_max from 5 steps of Lanczos on A x = lam D x
  (D-inner product) started from the SplitMix64 vector of ``rng``.
"""
from __future__ import annotations

from fractions import Fraction
from functools import cmp_to_key

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .rng import uniform_pm1
from .schur import blockdiag_sparse

MAX_AGG = 20
NULL_DIM = 16
DROP_TOL = 1e-10


# --------------------------------------------------------------------------
# covisibility and strength of connection (Section 3.2)
# --------------------------------------------------------------------------
def covisibility(cam_idx, pt_idx, n_cams, n_pts):
    """W = V^T V with V the binary point-by-camera visibility matrix (int64)."""
    V = sp.csr_matrix((np.ones(len(cam_idx), dtype=np.int64), (pt_idx, cam_idx)),
                      shape=(n_pts, n_cams))
    V.data[:] = 1
    return (V.T @ V).tocsr()


def strength_order(W):
    """For each node i, its neighbours j != i with W_ij > 0, strongest first."""
    W = W.tocsr()
    diag = W.diagonal()
    order = []
    for i in range(W.shape[0]):
        cols = W.indices[W.indptr[i]:W.indptr[i + 1]]
        vals = W.data[W.indptr[i]:W.indptr[i + 1]]
        nb = [(int(j), int(w)) for j, w in zip(cols, vals) if j != i and w > 0]

        def cmp(a, b):
            (j, wj), (k, wk) = a, b
            lhs = wj * wj * int(diag[k])
            rhs = wk * wk * int(diag[j])
            if lhs != rhs:
                return -1 if lhs > rhs else 1
            return -1 if j < k else (1 if j > k else 0)
        nb.sort(key=cmp_to_key(cmp))
        order.append([j for j, _ in nb])
    return order


def strength_matrix(W):
    """G as floats (for inspection and tests only; ordering uses integers)."""
    W = W.tocsr().astype(np.float64)
    d = np.sqrt(W.diagonal())
    G = sp.diags(1.0 / d) @ W @ sp.diags(1.0 / d)
    G = G.tolil()
    G.setdiag(0)
    return G.tocsr()


def aggregate(order, max_agg=MAX_AGG):
    """Algorithm 2: greedy pairing with the strongest unaggregated neighbour, else
    joining the strongest neighbour's aggregate while it has < max_agg members."""
    n = len(order)
    agg = -np.ones(n, dtype=np.int64)
    size = []
    for i in range(n):
        if agg[i] >= 0:
            continue
        for j in order[i]:
            if agg[j] < 0:
                agg[i] = agg[j] = len(size)
                size.append(2)
                break
            k = agg[j]
            if size[k] < max_agg:
                agg[i] = k
                size[k] += 1
                break
    for i in range(n):
        if agg[i] < 0:
            agg[i] = len(size)
            size.append(1)
    return agg


def aggregation_matrix(agg):
    n = len(agg)
    return sp.csr_matrix((np.ones(n, dtype=np.int64), (np.arange(n), agg)),
                         shape=(n, int(agg.max()) + 1))


# --------------------------------------------------------------------------
# near-nullspace (Section 3.1)
# --------------------------------------------------------------------------
def _rodrigues_matrix(r):
    th = np.linalg.norm(r)
    K = np.array([[0, -r[2], r[1]], [r[2], 0, -r[0]], [-r[1], r[0], 0]])
    if th * th < 1e-16:
        return np.eye(3) + K
    return np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * (K @ K)


def _right_jacobian_inverse(r):
    """J_r(r)^-1 of SO(3): R(r + dr) = R(r) exp([J_r dr]_x) to first order."""
    th = np.linalg.norm(r)
    K = np.array([[0, -r[2], r[1]], [r[2], 0, -r[0]], [-r[1], r[0], 0]])
    if th < 1e-6:
        coef = 1.0 / 12.0
    else:
        coef = 1.0 / th ** 2 - (1 + np.cos(th)) / (2 * th * np.sin(th))
    return np.eye(3) + 0.5 * K + coef * (K @ K)


def nullspace_camera_block(cam):
    """9 x 16 rows of the near-nullspace for one camera.

    A similarity X' = s R_g X + t_g of the whole scene leaves every residual
    unchanged when each camera moves to R' = R R_g^T, t' = s t - R' t_g.  The
    derivatives at identity give, per camera:
      translation e_k:  dr = 0,               dt = -R e_k
      rotation e_k:     dr = -J_r(r)^-1 e_k,  dt = 0
      scale:            dr = 0,               dt = t
    then 9 columns constant on each camera parameter."""
    r, t = cam[0:3], cam[3:6]
    R = _rodrigues_matrix(r)
    Jri = _right_jacobian_inverse(r)
    K = np.zeros((9, NULL_DIM))
    for k in range(3):
        K[3:6, k] = -R[:, k]
        K[0:3, 3 + k] = -Jri[:, k]
    K[3:6, 6] = t
    K[:, 7:16] = np.eye(9)
    return K


def nullspace(cams):
    return np.stack([nullspace_camera_block(c) for c in cams])


def nullspace_points(pts):
    """Point part of the 7 gauge modes (used only to pin the camera part)."""
    n = pts.shape[0]
    K = np.zeros((n, 3, 7))
    for k in range(3):
        K[:, k, k] = 1.0
        e = np.zeros(3)
        e[k] = 1.0
        K[:, :, 3 + k] = np.cross(np.broadcast_to(e, pts.shape), pts)
    K[:, :, 6] = pts
    return K


# --------------------------------------------------------------------------
# tentative prolongator (Section 3.3)
# --------------------------------------------------------------------------
def mgs_qr(K):
    """Thin QR of K (m x 16) by modified Gram-Schmidt with one re-orthogonalisation;
    dropped columns give zero columns of Q and zero rows of R."""
    m, k = K.shape
    Q = np.zeros((m, k))
    R = np.zeros((k, k))
    kept = np.zeros(k, dtype=bool)
    for j in range(k):
        v = K[:, j].copy()
        n0 = np.linalg.norm(v)
        for _ in range(2):
            for i in range(j):
                if kept[i]:
                    h = Q[:, i] @ v
                    v -= h * Q[:, i]
                    R[i, j] += h
        nv = np.linalg.norm(v)
        if n0 > 0 and nv > DROP_TOL * n0:
            Q[:, j] = v / nv
            R[j, j] = nv
            kept[j] = True
    return Q, R, kept


def tentative_prolongator(K, agg, b):
    """K: [n, b, 16] per-node near-nullspace rows.  Returns Q blocks [n, b, 16],
    coarse nullspace R blocks [n_agg, 16, 16] and kept masks [n_agg, 16]."""
    n_agg = int(agg.max()) + 1
    Qb = np.zeros((len(agg), b, NULL_DIM))
    Rc = np.zeros((n_agg, NULL_DIM, NULL_DIM))
    kept = np.zeros((n_agg, NULL_DIM), dtype=bool)
    members = [[] for _ in range(n_agg)]
    for i, a in enumerate(agg):
        members[a].append(i)
    for a in range(n_agg):
        mem = members[a]
        Kagg = np.concatenate([K[i] for i in mem], axis=0)
        Q, R, kp = mgs_qr(Kagg)
        for s, i in enumerate(mem):
            Qb[i] = Q[s * b:(s + 1) * b]
        Rc[a] = R
        kept[a] = kp
    return Qb, Rc, kept


def prolongation_matrix(Qb, agg):
    n, b, k = Qb.shape
    n_agg = int(agg.max()) + 1
    rows = (np.arange(n)[:, None, None] * b + np.arange(b)[None, :, None]) + np.zeros((1, 1, k), int)
    cols = (agg[:, None, None] * k + np.arange(k)[None, None, :]) + np.zeros((1, b, 1), int)
    return sp.csr_matrix((Qb.ravel(), (rows.ravel(), cols.ravel())), shape=(n * b, n_agg * k))


def galerkin(A, P, kept):
    """A_{l+1} = P^T A_l P (R = P^T), with a unit diagonal on dropped coarse dofs."""
    Ac = (P.T @ A @ P).tocsr()
    pad = np.flatnonzero(~kept.ravel())
    if len(pad):
        Ac = Ac.tolil()
        for d in pad:
            Ac[d, d] = 1.0
        Ac = Ac.tocsr()
    Ac.sum_duplicates()
    return Ac


# --------------------------------------------------------------------------
# smoother (Section 3.4)
# --------------------------------------------------------------------------
def diag_blocks(A, b):
    n = A.shape[0] // b
    Ac = A.tocoo()
    m = (Ac.row // b) == (Ac.col // b)
    blocks = np.zeros((n, b, b))
    np.add.at(blocks, (Ac.row[m] // b, Ac.row[m] % b, Ac.col[m] % b), Ac.data[m])
    return blocks


def lanczos_lambda_max(A, Dblk, Dinv, steps=5, seed=0):
    """Largest Ritz value of 'steps' Lanczos steps on A x = lam D x in the
    D-inner product (one operator application per step)."""
    n = A.shape[0]
    v = uniform_pm1(seed, n)
    q = v / np.sqrt(v @ (Dblk @ v))
    q_prev = np.zeros(n)
    beta_prev = 0.0
    alphas, betas = [], []
    for j in range(steps):
        Aq = A @ q
        alpha = q @ Aq
        w = Dinv @ Aq - alpha * q - beta_prev * q_prev
        alphas.append(alpha)
        if j == steps - 1:
            break
        beta = np.sqrt(w @ (Dblk @ w))
        if not beta > 0:
            break
        betas.append(beta)
        q_prev, q, beta_prev = q, w / beta, beta
    T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
    return float(np.linalg.eigvalsh(T)[-1]), np.array(alphas), np.array(betas)


def chebyshev(A, Dinv, x, b, lo, hi, steps=2):
    """Chebyshev semi-iteration for A x = b preconditioned by Dinv on [lo, hi]."""
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b - A @ x
    d = (Dinv @ r) / theta
    for k in range(steps):
        x = x + d
        if k == steps - 1:
            break
        r = r - A @ d
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (Dinv @ r)
        rho = rho_new
    return x


# --------------------------------------------------------------------------
# hierarchy and V-cycle (Section 2.3, Algorithm 1)
# --------------------------------------------------------------------------
class Level:
    pass


class Hierarchy:
    def __init__(self, S, W, cams, coarse_max_nodes=64, max_levels=10, max_agg=MAX_AGG,
                 lanczos_steps=5, cheb_lo=0.3, cheb_hi=1.1, pre=2, post=2):
        self.pre, self.post = pre, post
        self.levels = []
        A, Wl, K, b = S.tocsr(), W.tocsr(), nullspace(cams), 9
        while True:
            L = Level()
            L.A, L.W, L.K, L.b = A, Wl, K, b
            L.n = A.shape[0] // b
            self.levels.append(L)
            coarsest = L.n <= coarse_max_nodes or len(self.levels) == max_levels
            if not coarsest:
                L.order = strength_order(Wl)
                L.agg = aggregate(L.order, max_agg)
                if int(L.agg.max()) + 1 >= L.n:
                    coarsest = True
            if coarsest:
                L.dense = A.toarray()
                L.chol = sla.cho_factor(L.dense, lower=True)
                break
            L.Dblk_blocks = diag_blocks(A, b)
            L.Dblk = blockdiag_sparse(L.Dblk_blocks)
            L.Dinv_blocks = np.linalg.inv(L.Dblk_blocks)
            L.Dinv = blockdiag_sparse(L.Dinv_blocks)
            L.lam_max, L.alphas, L.betas = lanczos_lambda_max(A, L.Dblk, L.Dinv, lanczos_steps)
            L.lo, L.hi = cheb_lo * L.lam_max, cheb_hi * L.lam_max
            L.Q, R, L.kept = tentative_prolongator(K, L.agg, b)
            L.P = prolongation_matrix(L.Q, L.agg)
            Agg = aggregation_matrix(L.agg)
            A = galerkin(A, L.P, L.kept)
            Wl = (Agg.T @ Wl @ Agg).tocsr()
            K, b = R, NULL_DIM

    def mgcycle(self, l, x, b):
        """Algorithm 1."""
        L = self.levels[l]
        if l == len(self.levels) - 1:
            return sla.cho_solve(L.chol, b)
        x = chebyshev(L.A, L.Dinv, x, b, L.lo, L.hi, self.pre)        # pre-smoothing
        r = b - L.A @ x                                                 # residual
        rc = L.P.T @ r                                                  # restriction
        xc = np.zeros(rc.shape[0])
        xc = self.mgcycle(l + 1, xc, rc)                                # coarse solve
        x = x + L.P @ xc                                                # prolongation
        x = chebyshev(L.A, L.Dinv, x, b, L.lo, L.hi, self.post)       # post-smoothing
        return x

    def apply(self, r):
        return self.mgcycle(0, np.zeros_like(r), r)
