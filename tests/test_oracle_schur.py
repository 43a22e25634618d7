"""Pins of the oracle's damped normal equations and Schur complement (Section 2.1, 3.6)."""
import numpy as np
import scipy.sparse as sp

from conftest import scene
from oracle import camera, multigrid, schur


def _tiny():
    return scene("ring", seed=2, n_cams=6, n_pts=60, kmin=2, kmax=4)


def test_gradient_sign_against_cost_derivative():
    # g = -J^T f must be minus the gradient of 1/2 |f|^2 (the RHS of Eq. 1 read as -J^T f)
    s = _tiny()
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 1e-4)
    j, h = 4, 1e-6
    cp, cm = s.cams.copy(), s.cams.copy()
    cp[2, j] += h
    cm[2, j] -= h
    fd = (camera.cost(cp, s.pts, s.cam_idx, s.pt_idx, s.obs) - camera.cost(cm, s.pts, s.cam_idx, s.pt_idx, s.obs)) / (2 * h)
    assert np.isclose(-sch.g_c[9 * 2 + j], fd, rtol=1e-6)


def test_schur_solution_equals_dense_normal_equations():
    s = _tiny()
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 1e-3)
    full = sch.dense_normal_solve()
    dc = np.linalg.solve(sch.S.toarray(), sch.b)
    dp = sch.back_substitute(dc)
    nc = 9 * s.n_cams
    assert np.linalg.norm(dc - full[:nc]) <= 1e-9 * np.linalg.norm(full[:nc])
    assert np.linalg.norm(dp - full[nc:]) <= 1e-9 * np.linalg.norm(full[nc:])


def test_schur_is_symmetric_psd_and_implicit_equals_explicit():
    s = scene("ring", seed=0, n_cams=16, n_pts=800)
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 1e-4)
    S = sch.S.toarray()
    assert np.abs(S - S.T).max() <= 1e-13 * np.abs(S).max()
    ev = np.linalg.eigvalsh(S)
    assert ev.min() > 0
    x = np.random.default_rng(0).normal(size=S.shape[0])
    assert np.linalg.norm(sch.implicit_matvec(x) - S @ x) <= 1e-12 * np.linalg.norm(S @ x)


def test_gauge_modes_span_the_nullspace_at_zero_damping():
    # Section 3.1: J^T J has a 7-dimensional nullspace (similarity gauge); for the
    # Schur complement it is the camera part K_xc.  Exact at any linearisation point.
    for s in (scene("ring", seed=0, n_cams=16, n_pts=800), scene("street_chain", n_cams=60, n_pts=3000)):
        sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 0.0, "identity")
        K = multigrid.nullspace(s.cams).reshape(-1, 16)[:, :7]
        SK = sch.S @ K
        assert np.abs(SK).max() <= 1e-10 * abs(sch.S).max() * np.abs(K).max()
        # and the full J annihilates the joint gauge vectors
        Kp = multigrid.nullspace_points(s.pts).reshape(-1, 7)
        Jm = sp.hstack([sch.Fm, sch.Em]).tocsr()
        Jn = Jm @ np.vstack([K, Kp])
        assert np.abs(Jn).max() <= 1e-9 * abs(Jm).max() * np.abs(K).max()


def test_marquardt_damping_floor_and_identity_variant():
    s = _tiny()
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 0.5)
    dcj = np.asarray(sch.Fm.multiply(sch.Fm).sum(axis=0)).ravel()
    assert np.allclose(sch.Dc, 0.5 * np.maximum(dcj, 1e-6))
    sid = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 0.5, "identity")
    assert np.all(sid.Dc == 0.5) and np.all(sid.Dp == 0.5)


def test_model_reduction_equals_quadratic_model_decrease():
    s = _tiny()
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 1e-2)
    full = sch.dense_normal_solve()
    nc = 9 * s.n_cams
    J = sp.hstack([sch.Fm, sch.Em]).toarray()
    f = sch.f.ravel()
    direct = 0.5 * f @ f - 0.5 * np.sum((f + J @ full) ** 2)
    assert np.isclose(sch.model_reduction(full[:nc], full[nc:]), direct, rtol=1e-9)
