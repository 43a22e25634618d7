"""Pins of the oracle's camera model (residual and Jacobians)."""
import numpy as np
from scipy.spatial.transform import Rotation

from conftest import scene
from oracle import camera


def test_rotation_matches_scipy():
    rng = np.random.default_rng(0)
    r = rng.normal(size=(200, 3)) * rng.uniform(0.0, 3.0, (200, 1))
    X = rng.normal(size=(200, 3))
    ref = Rotation.from_rotvec(r).apply(X)
    assert np.abs(camera.rotate(r, X) - ref).max() < 1e-13


def test_small_angle_branch_is_first_order():
    rng = np.random.default_rng(1)
    r = rng.normal(size=(50, 3)) * 1e-9          # theta^2 ~ 1e-18 < 1e-16
    X = rng.normal(size=(50, 3))
    assert np.allclose(camera.rotate(r, X), X + np.cross(r, X), rtol=0, atol=1e-15)
    ref = Rotation.from_rotvec(r).apply(X)
    assert np.abs(camera.rotate(r, X) - ref).max() < 1e-15


def test_projection_matches_generator_forward_model():
    # the generator projects with rotation matrices; at the true parameters the
    # oracle residual must be exactly the added pixel noise
    from paper_2007_01941_gb300 import scenes
    s = scene("ring", seed=3, n_cams=8, n_pts=300)
    R = Rotation.from_rotvec(s.cams_true[:, :3]).as_matrix()
    ci, pi = s.cam_idx, s.pt_idx
    uv, _ = scenes._forward_project(R[ci], s.cams_true[ci, 3:6], s.cams_true[ci, 6], s.cams_true[ci, 7],
                                    s.cams_true[ci, 8], s.pts_true[pi])
    pred = camera.project(s.cams_true[ci], s.pts_true[pi])
    assert np.abs(pred - uv).max() < 1e-9 * np.abs(uv).max()


def _fd_jacobian(cams, pts, ci, pi, obs):
    n = len(ci)
    F = np.zeros((n, 2, 9))
    E = np.zeros((n, 2, 3))
    for j in range(9):
        h = 1e-6 * np.maximum(np.abs(cams[:, j]), 1.0)
        cp, cm = cams.copy(), cams.copy()
        cp[:, j] += h
        cm[:, j] -= h
        d = camera.residuals(cp, pts, ci, pi, obs) - camera.residuals(cm, pts, ci, pi, obs)
        F[:, :, j] = d / (2 * h[ci])[:, None]
    for j in range(3):
        h = 1e-6 * np.maximum(np.abs(pts[:, j]), 1e-2)
        pp, pm = pts.copy(), pts.copy()
        pp[:, j] += h
        pm[:, j] -= h
        d = camera.residuals(cams, pp, ci, pi, obs) - camera.residuals(cams, pm, ci, pi, obs)
        E[:, :, j] = d / (2 * h[pi])[:, None]
    return F, E


def test_jacobians_match_central_differences():
    for s in (scene("ring", seed=0, n_cams=12, n_pts=200), scene("street_chain", n_cams=40, n_pts=400)):
        F, E = camera.jacobians(s.cams, s.pts, s.cam_idx, s.pt_idx)
        Ff, Ef = _fd_jacobian(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs)
        for j in range(9):
            scale = np.abs(F[:, :, j]).max()
            assert np.abs(F[:, :, j] - Ff[:, :, j]).max() <= 1e-6 * scale, j
        assert np.abs(E - Ef).max() <= 1e-6 * np.abs(E).max()


def test_jacobian_small_angle_cameras():
    s = scene("ring", seed=0, n_cams=12, n_pts=200)
    cams = s.cams.copy()
    cams[:, :3] *= 1e-10                            # every camera in the first-order branch
    F, E = camera.jacobians(cams, s.pts, s.cam_idx, s.pt_idx)
    X = s.pts[s.pt_idx]
    # d(X + r x X)/dr = -[X]_x ; compare through the chain rule with dP-derivatives
    Ft = F[:, :, 3:6]                               # d f / dP
    skewX = np.zeros((len(X), 3, 3))
    skewX[:, 0, 1], skewX[:, 0, 2] = -X[:, 2], X[:, 1]
    skewX[:, 1, 0], skewX[:, 1, 2] = X[:, 2], -X[:, 0]
    skewX[:, 2, 0], skewX[:, 2, 1] = -X[:, 1], X[:, 0]
    assert np.allclose(F[:, :, 0:3], np.einsum("nij,njk->nik", Ft, -skewX), rtol=1e-12, atol=1e-12)


def test_cost_is_half_squared_sum():
    s = scene("ring", seed=0, n_cams=12, n_pts=200)
    f = camera.residuals(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs)
    assert np.isclose(camera.cost(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs), 0.5 * np.sum(f ** 2))
