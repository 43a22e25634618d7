"""One Levenberg-Marquardt step (Section 2.1; settings of Section 5).

The paper delegates the step control to Ceres.  The reading taken here is the
standard gain-ratio update (Madsen, Nielsen & Tingleff 2004, as used by Ceres):

    rho = (cost(x) - cost(x + delta)) / (L(0) - L(delta))
    accept if rho > 1e-3:  lam <- lam * max(1/3, 1 - (2 rho - 1)^3),  nu <- 2
    else:                  lam <- lam * nu,                           nu <- 2 nu

with lam_0 = 1 / (initial trust radius 1e4) = 1e-4 (Section 5).  A step whose linear
solve fails is unsuccessful and handled like a rejection (Ceres does the same).
"""
from __future__ import annotations

import numpy as np

from . import camera, multigrid, pcg as pcg_mod, schur

MIN_RELATIVE_DECREASE = 1e-3


def solve_step(sch: schur.Schur, cams, precond="mg", rtol=1e-8, max_iters=1000, stop="relres", tau=0.1,
               **mg_kw):
    """delta_c by PCG on S (with the chosen preconditioner and stopping rule) and delta_p
    by back-substitution."""
    if precond == "mg":
        W = multigrid.covisibility(sch.cam_idx, sch.pt_idx, sch.n_cams, sch.n_pts)
        H = multigrid.Hierarchy(sch.S, W, cams, **mg_kw)
        M = H.apply
    elif precond == "jacobi":
        blocks = multigrid.diag_blocks(sch.S, 9)
        Minv = schur.blockdiag_sparse(np.linalg.inv(blocks))
        M = lambda r: Minv @ r
    else:
        M = None
    dc, it, rel, hist = pcg_mod.pcg(lambda v: sch.S @ v, sch.b, M, rtol, max_iters, stop=stop, tau=tau)
    dp = sch.back_substitute(dc)
    return dc, dp, it, rel


def lm_step(cams, pts, cam_idx, pt_idx, obs, lam, nu=2.0, precond="mg", rtol=1e-8, huber=None, **kw):
    """Returns (cams', pts', lam', nu', accepted, cost_before, cost_after_or_before, info).
    huber = a: the robust objective and corrected residuals of Section 5 (oracle/robust.py)."""
    sch = schur.linearize(cams, pts, cam_idx, pt_idx, obs, lam, huber=huber)
    cost0 = camera.cost(cams, pts, cam_idx, pt_idx, obs, huber=huber)
    try:
        dc, dp, it, rel = solve_step(sch, cams, precond, rtol, **kw)
    except (np.linalg.LinAlgError, FloatingPointError) as ex:
        # a linear solve that fails (the coarsest factorisation finds the operator not
        # positive definite, or CG breaks down) is an unsuccessful step, as in the Ceres
        # trust-region loop the paper uses: x is kept and lambda grows as after a rejection
        info = dict(iters=0, rel_res=np.inf, rho=-np.inf, model=0.0, cost_new=cost0, failed=str(ex))
        return cams, pts, lam * nu, 2.0 * nu, False, cost0, cost0, info
    cams1 = cams + dc.reshape(-1, 9)
    pts1 = pts + dp.reshape(-1, 3)
    cost1 = camera.cost(cams1, pts1, cam_idx, pt_idx, obs, huber=huber)
    model = sch.model_reduction(dc, dp)
    rho = (cost0 - cost1) / model if model > 0 else -np.inf
    info = dict(iters=it, rel_res=rel, rho=rho, model=model, cost_new=cost1)
    if rho > MIN_RELATIVE_DECREASE:
        lam = lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)
        return cams1, pts1, lam, 2.0, True, cost0, cost1, info
    return cams, pts, lam * nu, 2.0 * nu, False, cost0, cost0, info
