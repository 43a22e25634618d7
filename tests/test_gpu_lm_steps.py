"""Consecutive LM steps on one problem (Section 2.1; step control of Section 5 read as the
gain-ratio rule), GPU through the C ABI against the oracle stepped from the same start.

Every GPU step after the first reuses the symbolic hierarchy built by the first setup
(covisibility, aggregates, patterns, pair and Galerkin lists) and refreshes only its
numbers at the new cameras and points; the oracle rebuilds everything at every step.  So
these tests are what checks that refresh: a stale value anywhere in it changes the step.
"""
import numpy as np
import pytest

from conftest import scene
from oracle import lm

pytestmark = pytest.mark.gpu

CHAIN = dict(n_cams=300, n_pts=30000)


def _api():
    from paper_2007_01941_gb300 import _ffi, api
    return api, _ffi


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lm_steps_track_oracle(gpu, precision):
    """Four accepted steps on the 300-camera chain with the default (AUTO) level-0
    operator: at every step the acceptance, the cost, lambda and the cameras and points
    agree with the oracle's.  Positions are compared through their displacement from
    the start, x_k - x_0, which is what the solves produce; its error is the solve's
    forward error (<= 1e-8 relative at rtol 1e-12 in FP64 and <= 1e-6 at rtol 1e-10 in
    mixed precision, as in the single-step tests) carried through the steps."""
    api, F_ = _api()
    prec = {"fp64": F_.BA_FP64, "mixed": F_.BA_MIXED}[precision]
    rtol = 1e-12 if precision == "fp64" else 1e-10
    tol_x = 1e-8 if precision == "fp64" else 2e-6
    # the mixed cost carries the paired-FP32 linearisation's error (about 6 kappa u of the
    # residuals, u = 2^-48, kappa ~ 1e2 on the chain), relative to |obs| / |f| ~ 1e2-1e3
    tol_c = 1e-9 if precision == "fp64" else 1e-8
    s = scene("street_chain", **CHAIN)
    prob, cams, pts, obs = api.from_scene(s, device=gpu, precision=prec, coarse_max_nodes=16, rtol=rtol,
                                          max_iters=5000)
    assert prob.options.level0_operator == F_.BA_OP_AUTO
    x, p, lam, nu = s.cams, s.pts, s.lam, 2.0
    lam_g = s.lam
    for k in range(4):
        lam_g, acc_g, cost_g = prob.lm_step(cams, pts, obs, lam_g)
        x, p, lam, nu, acc, cost0, cost1, info = lm.lm_step(x, p, s.cam_idx, s.pt_idx, s.obs, lam, nu, rtol=rtol,
                                                            coarse_max_nodes=16, max_iters=5000)
        assert acc_g == acc and acc, k
        # cost of the accepted point; the two trajectories differ by the solves' forward
        # error, which changes a cost near its minimum only to second order
        assert abs(cost_g - cost1) <= tol_c * cost1, (k, cost_g, cost1)
        # lambda' = lambda max(1/3, 1 - (2 rho - 1)^3): rho is a ratio of cost decreases
        # that shrink as the steps converge, so allow it the cost's error over the decrease
        drho = tol_c * cost1 / max(cost0 - cost1, 1e-300)
        assert abs(lam_g - lam) <= max(1e-9, 6 * drho) * lam, (k, lam_g, lam, info["rho"])
        assert prob.info()["level0_explicit"]
        dx_g, dx_o = _np(cams) - s.cams, x - s.cams
        dp_g, dp_o = _np(pts) - s.pts, p - s.pts
        assert np.linalg.norm(dx_g - dx_o) <= tol_x * np.linalg.norm(dx_o), k
        assert np.linalg.norm(dp_g - dp_o) <= tol_x * np.linalg.norm(dp_o), k
    # the steps moved the cameras: later setups did refresh at new points
    assert np.linalg.norm(x - s.cams) > 1e-3 * np.linalg.norm(s.cams)


def _rejecting_scene():
    # 16-camera ring with starting rotations off by N(0, 0.8^2) per component: steps 1
    # and 5 are accepted, steps 2-4 overshoot (rho about -1e23, -6e22 and -0.12)
    from paper_2007_01941_gb300 import scenes
    return scenes.rotated_start(scene("ring", seed=0, n_cams=16, n_pts=800), 0.8, seed=11)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lm_reject_branch_matches_oracle(gpu, precision):
    """Accept, three rejections in a row, accept: a rejected step leaves the cameras and
    points bit-for-bit unchanged, returns the cost at the current point and multiplies
    lambda by nu, which doubles with every rejection (2, 4, 8) and is reset to 2 by the
    next accepted step."""
    api, F_ = _api()
    prec = {"fp64": F_.BA_FP64, "mixed": F_.BA_MIXED}[precision]
    s = _rejecting_scene()
    prob, cams, pts, obs = api.from_scene(s, device=gpu, precision=prec, coarse_max_nodes=4, rtol=1e-10)
    x, p, lam, nu = s.cams, s.pts, 1e-4, 2.0
    lam_g = 1e-4
    # the accepted costs follow the two trajectories, which differ by the solves' forward
    # error (mixed: about 1e-7 of a step), at points that are not yet minima
    tol_c = 1e-9 if precision == "fp64" else 1e-8
    pattern = []
    for k in range(5):
        c_before, p_before = cams.clone(), pts.clone()
        lam_in = lam_g
        lam_g, acc_g, cost_g = prob.lm_step(cams, pts, obs, lam_g)
        nu_in = nu
        x, p, lam, nu, acc, cost0, cost1, info = lm.lm_step(x, p, s.cam_idx, s.pt_idx, s.obs, lam, nu, rtol=1e-10,
                                                            coarse_max_nodes=4)
        pattern.append(acc)
        assert acc_g == acc, (k, info["rho"])
        if not acc:
            assert torch_equal(cams, c_before) and torch_equal(pts, p_before), k
            assert lam_g == lam_in * nu_in, k                 # lambda nu, exactly
            assert abs(cost_g - cost0) <= 1e-9 * cost0, k     # the cost at the current point
        else:
            assert abs(cost_g - cost1) <= tol_c * cost1, (k, cost_g, cost1)
            assert abs(lam_g - lam) <= 1e-7 * lam, k
            tol = 1e-8 if precision == "fp64" else 1e-6
            assert np.linalg.norm(_np(cams) - x) <= tol * np.linalg.norm(x - _np(c_before)), k
            assert np.linalg.norm(_np(pts) - p) <= tol * np.linalg.norm(p - _np(p_before)), k
    assert pattern == [True, False, False, False, True]


def torch_equal(a, b):
    import torch
    return bool(torch.equal(a, b))
