"""Pins of the oracle's Huber loss (Section 5) and its use in the LM step."""
import numpy as np

from conftest import scene
from oracle import camera, lm, robust, schur


def test_huber_values_and_continuity():
    a = 1.5
    s = np.array([0.0, 0.5, a * a, 4.0, 100.0])
    rho, rho1 = robust.huber(s, a)
    # quadratic part equals the squared loss; linear-in-|f| part 2 a |f| - a^2
    assert np.allclose(rho[:3], s[:3])
    assert np.allclose(rho[3:], 2 * a * np.sqrt(s[3:]) - a * a)
    # value and slope continuous at s = a^2 (C^1)
    eps = 1e-7
    lo, dlo = robust.huber(a * a - eps, a)
    hi, dhi = robust.huber(a * a + eps, a)
    assert abs(hi - lo) < 1e-6 and abs(dhi - dlo) < 1e-6
    # the paper's form with a = 1: 2 sqrt(s) - 1 beyond s = 1
    r1, _ = robust.huber(np.array([9.0]), 1.0)
    assert r1[0] == 5.0


def test_corrected_system_gives_the_robust_gradient():
    """g = -J~^T f~ = -sum_o loss'(s_o) J_o^T f_o is the negative gradient of
    1/2 sum loss(|f_o|^2): checked against central differences of the robust cost."""
    s = scene("ring", seed=0, n_pts=300, outlier_frac=0.05)
    a = 2.0
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 0.0, huber=a)
    rng = np.random.default_rng(0)
    for _ in range(8):
        if rng.random() < 0.5:
            c, k = int(rng.integers(s.n_cams)), int(rng.integers(9))
            h = 1e-6 * max(1.0, abs(s.cams[c, k]))
            cp, cm = s.cams.copy(), s.cams.copy()
            cp[c, k] += h
            cm[c, k] -= h
            fd = (camera.cost(cp, s.pts, s.cam_idx, s.pt_idx, s.obs, huber=a)
                  - camera.cost(cm, s.pts, s.cam_idx, s.pt_idx, s.obs, huber=a)) / (2 * h)
            g = -sch.g_c[9 * c + k]
        else:
            p, k = int(rng.integers(s.n_pts)), int(rng.integers(3))
            h = 1e-6 * max(1.0, abs(s.pts[p, k]))
            pp, pm = s.pts.copy(), s.pts.copy()
            pp[p, k] += h
            pm[p, k] -= h
            fd = (camera.cost(s.cams, pp, s.cam_idx, s.pt_idx, s.obs, huber=a)
                  - camera.cost(s.cams, pm, s.cam_idx, s.pt_idx, s.obs, huber=a)) / (2 * h)
            g = -sch.g_p[3 * p + k]
        assert abs(fd - g) <= 1e-5 * max(1.0, abs(g)), (fd, g)


def test_large_scale_reduces_to_the_squared_loss():
    s = scene("ring", seed=1, n_pts=400)
    big = 1e6   # every |f_o|^2 below a^2
    r0 = lm.lm_step(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 1e-4, rtol=1e-12, coarse_max_nodes=4)
    r1 = lm.lm_step(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 1e-4, rtol=1e-12, coarse_max_nodes=4, huber=big)
    assert np.allclose(r0[0], r1[0], rtol=0, atol=1e-12) and r0[4] == r1[4]
    assert abs(r0[5] - r1[5]) <= 1e-12 * r0[5]


def test_outliers_are_down_weighted():
    # one residual with |f|^2 = 100 a^2 keeps 1/10 of its squared-loss gradient weight
    a = 1.0
    f = np.array([[0.3, 0.4], [6.0, 8.0]])
    w = robust.weights(f, a)
    assert w[0] == 1.0
    assert np.isclose(w[1] ** 2, a / 10.0)


def test_huber_lm_step_decreases_the_robust_cost():
    s = scene("ring", seed=2, n_pts=800, outlier_frac=0.05)
    out = lm.lm_step(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 1e-4, rtol=1e-10, coarse_max_nodes=4, huber=1.0)
    assert out[4] and out[6] < out[5]
