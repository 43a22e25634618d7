"""The adjoint of the LM step at street-chain size (2,000 cameras, 300,000 points,
1,499,558 observations): gradients of L = vbar . delta with respect to the pixel
observations and the camera parameters, for a seeded cotangent vbar ~ N(0, 1).

ba_adjoint solves (J^T J + D) mu = vbar through the Schur complement with the forward
solve's multigrid hierarchy and rebuilds F and E per observation in its Hessian-vector
pass instead of reading them back.  Checked two ways:
  * central finite differences of the forward solve (FP64, forward PCG to rtol 1e-13)
    on 32 coordinates of the full scene, 16 observation and 16 camera coordinates drawn
    at random among those whose derivative stands above the differences' rounding
    floor, at damping lambda = 1e-2.  At the scene's lambda = 1e-4 the street chain's S
    is so ill-conditioned that central differences in FP64 cannot resolve 1e-5 even with
    exact solves: the oracle's own differences of camera coordinates reach 2e-5 at best
    and 1e-3 at h = 1e-7, rounding amplified by kappa(S).  Observation coordinates, in
    which delta is linear, take plain central differences with h = 1e-6; camera
    coordinates the fourth-order combination of central differences at h = 2e-5 and
    2h (both scaled by the coordinate's magnitude), since delta is strongly nonlinear in
    some of them;
  * the oracle's dense adjoint on the 200-camera / 10,000-point subscene, in FP64 and
    in mixed precision.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj

pytestmark = pytest.mark.gpu


def _api():
    from paper_2007_01941_gb300 import _ffi, api
    return api, _ffi


def _np(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def chain():
    from paper_2007_01941_gb300 import scenes
    return scenes.street_chain()


def _pick(rng, g, k):
    # k coordinates drawn uniformly at random among those whose derivative is at least
    # 5 % of the largest: the central difference of two solves accurate to rtol 1e-13
    # carries an absolute error of about 1.5e-7 max|g| (measured: delta is linear in the
    # observations, so that is all solver rounding), which is 1e-5 of a derivative only
    # from about 1.5 % of max|g| upwards; most of the 3 million observation coordinates
    # move delta far less than that
    a = np.abs(g.ravel())
    cand = np.flatnonzero(a >= 0.05 * a.max())
    if len(cand) < 4 * k:
        cand = np.argsort(a)[-4 * k:]
    return rng.choice(cand, size=k, replace=False)


def test_adjoint_matches_central_differences_at_street_chain_size(gpu, chain):
    api, F_ = _api()
    s = chain
    lam = 1e-2
    prob, cams, pts, obs = api.from_scene(s, device=gpu, precision=F_.BA_FP64, rtol=1e-13, max_iters=5000,
                                          coarse_max_nodes=32)
    prob.solve(cams, pts, obs, lam)
    rng = np.random.default_rng(4)
    vbar = torch.tensor(rng.normal(size=9 * s.n_cams + 3 * s.n_pts), device=gpu)
    go, gc, _ = prob.adjoint(vbar, want_pts=False)
    go, gc = _np(go), _np(gc)

    def loss(cams, obs):
        dc, dp, it, rel = prob.solve(cams, pts, obs, lam)
        assert rel <= 1e-13
        return float(torch.dot(vbar, torch.cat([dc.reshape(-1), dp.reshape(-1)])).item())

    checked = 0
    for which, grad, base in (("obs", go, obs), ("cams", gc, cams)):
        scale = np.abs(grad).max()
        for flat in _pick(rng, grad, 16):
            i, j = np.unravel_index(flat, grad.shape)
            def central(h):
                args = {"cams": cams, "obs": obs}
                plus, minus = base.clone(), base.clone()
                plus[i, j] += h
                minus[i, j] -= h
                lp = loss(**dict(args, **{which: plus}))
                lm = loss(**dict(args, **{which: minus}))
                return (lp - lm) / (2 * h)
            if which == "obs":
                # delta is linear in the observations: the central difference is exact
                fd = central(1e-6 * max(1.0, abs(float(base[i, j]))))
            else:
                # camera coordinates: the fourth-order (Richardson) combination of central
                # differences at h and 2h.  delta is very nonlinear in some of them (cameras
                # near the chain's end: the oracle's exact sparse solves give 0.58, 9e-3 and
                # 1e-4 relative error at h = 1e-3, 1e-4, 1e-5 for one), so the second-order
                # difference alone would need an h where rounding already dominates
                h = 2e-5 * max(1.0, abs(float(base[i, j])))
                fd = (4.0 * central(h) - central(2.0 * h)) / 3.0
            g = float(grad[i, j])
            # 1e-5 relative, over the differences' rounding floor (2e-7 of the largest
            # derivative, a third above the 1.5e-7 measured)
            assert abs(fd - g) <= 1e-5 * abs(fd) + 2e-7 * scale, (which, i, j, fd, g, scale)
            checked += 1
    assert checked == 32


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_matches_dense_oracle_on_subscene(gpu, chain, precision):
    """200 cameras and 10,000 of the points seen only by them (dense S is 1800 x 1800):
    the oracle's adjoint from a dense Schur solve against ba_adjoint."""
    api, F_ = _api()
    from paper_2007_01941_gb300 import scenes
    s = scenes.subscene(chain, 200, 10000, seed=0)
    lam = s.lam
    prec = {"fp64": F_.BA_FP64, "mixed": F_.BA_MIXED}[precision]
    # mixed: the outer operator and residual are FP64-valued, so the solves reach the same
    # relative residual; the V-cycle in FP32 only costs iterations
    prob, cams, pts, obs = api.from_scene(s, device=gpu, precision=prec, rtol=1e-13, max_iters=5000,
                                          coarse_max_nodes=16)
    prob.solve(cams, pts, obs, lam)
    vbar = np.random.default_rng(9).normal(size=9 * s.n_cams + 3 * s.n_pts)
    go, gc, gp = prob.adjoint(torch.tensor(vbar, device=gpu))
    ro, rc, rp, _ = oadj.adjoint(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, lam, vbar)
    tol = 1e-7 if precision == "fp64" else 1e-6
    for got, ref in ((go, ro), (gc, rc), (gp, rp)):
        got = _np(got)
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()
