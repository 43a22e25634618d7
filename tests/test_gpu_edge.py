"""Edge and degenerate cases of the GPU path, and its error statuses."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

from conftest import scene
from oracle import schur
from paper_2007_01941_gb300.scenes import Scene

pytestmark = pytest.mark.gpu


def _api():
    from paper_2007_01941_gb300 import _ffi, api
    return api, _ffi


def _np(t):
    return t.detach().cpu().numpy()


def _drop_camera_obs(s, cam, orphan_points=(0, 1, 2)):
    """Removes every observation of camera `cam` and of the points `orphan_points`."""
    keep = (s.cam_idx != cam) & ~np.isin(s.pt_idx, orphan_points)
    cnt = np.bincount(s.pt_idx[keep], minlength=s.n_pts)
    keep &= cnt[s.pt_idx] >= 2          # keep every remaining point observed twice
    return Scene(s.name, s.n_cams, s.n_pts, int(keep.sum()), s.cam_idx[keep].copy(), s.pt_idx[keep].copy(),
                 s.obs[keep].copy(), s.cams, s.pts, s.cams_true, s.pts_true, s.lam, s.rtol)


def _exact(s, lam):
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, lam)
    return sch, sla.cho_solve(sla.cho_factor(sch.S.toarray()), sch.b)


def test_camera_and_points_without_observations(gpu):
    api, F_ = _api()
    base = scene("ring", seed=1, n_cams=20, n_pts=1500)
    s = _drop_camera_obs(base, 7)
    assert not np.any(s.cam_idx == 7) and np.any(np.bincount(s.pt_idx, minlength=s.n_pts) == 0)
    prob, cams, pts, obs = api.from_scene(s, device=gpu, coarse_max_nodes=4, rtol=1e-12)
    dc, dp, it, rel = prob.solve(cams, pts, obs, 1e-3)
    sch, ex = _exact(s, 1e-3)
    assert np.linalg.norm(_np(dc).ravel() - ex) <= 1e-8 * np.linalg.norm(ex)
    dpn = _np(dp)
    unobserved = np.bincount(s.pt_idx, minlength=s.n_pts) == 0
    assert np.all(dpn[unobserved] == 0.0)


def test_no_observations_gives_a_zero_step(gpu):
    api, F_ = _api()
    e = torch.zeros(0, dtype=torch.int32, device=gpu)
    prob = api.Problem(5, 3, e, e)
    cams = torch.zeros(5, 9, dtype=torch.float64, device=gpu)
    cams[:, 5] = -5.0
    pts = torch.zeros(3, 3, dtype=torch.float64, device=gpu)
    obs = torch.zeros(0, 2, dtype=torch.float64, device=gpu)
    assert prob.linearize(cams, pts, obs) == 0.0
    prob.schur_setup(1e-3)
    prob.mg_setup()
    dc, it, rel = prob.pcg_solve()
    assert it == 0 and torch.all(dc == 0)


def test_invalid_graphs_are_rejected(gpu):
    api, F_ = _api()
    ci = torch.tensor([0, 1, 1], dtype=torch.int32, device=gpu)
    pi = torch.tensor([0, 0, 0], dtype=torch.int32, device=gpu)
    with pytest.raises(api.BAError) as ex:
        api.Problem(2, 1, ci, pi)                       # camera 1 observes point 0 twice
    assert ex.value.status == F_.BA_ERR_INVALID_ARG
    with pytest.raises(api.BAError) as ex:
        api.Problem(2, 1, torch.tensor([0, 2], dtype=torch.int32, device=gpu),
                    torch.tensor([0, 0], dtype=torch.int32, device=gpu))
    assert ex.value.status == F_.BA_ERR_INVALID_ARG


def test_calls_out_of_order_and_nonfinite_input(gpu):
    api, F_ = _api()
    s = scene("ring", seed=0, n_cams=8, n_pts=200)
    prob, cams, pts, obs = api.from_scene(s, device=gpu)
    with pytest.raises(api.BAError) as ex:
        prob.pcg_solve()
    assert ex.value.status == F_.BA_ERR_STATE
    bad = obs.clone()
    bad[3, 1] = float("nan")
    with pytest.raises(api.BAError) as ex:
        prob.linearize(cams, pts, bad)
    assert ex.value.status == F_.BA_ERR_INVALID_ARG
    # the problem stays usable
    assert prob.linearize(cams, pts, obs) > 0


def test_iteration_cap_reports_not_converged_with_the_iterate(gpu):
    api, F_ = _api()
    s = scene("street_chain", n_cams=100, n_pts=8000)
    prob, cams, pts, obs = api.from_scene(s, device=gpu, max_iters=2, rtol=1e-14, coarse_max_nodes=8)
    prob.linearize(cams, pts, obs)
    prob.schur_setup(s.lam)
    prob.mg_setup()
    with pytest.raises(api.BAError) as ex:
        prob.pcg_solve()
    assert ex.value.status == F_.BA_ERR_NOT_CONVERGED
    dc, it, rel = prob.pcg_solve(allow_not_converged=True)
    assert it == 2 and rel > 1e-14 and torch.isfinite(dc).all() and dc.abs().max() > 0


def test_single_level_hierarchy_is_a_direct_solve(gpu):
    api, F_ = _api()
    s = scene("ring", seed=0)                            # 32 cameras <= coarse_max_nodes
    prob, cams, pts, obs = api.from_scene(s, device=gpu, coarse_max_nodes=64, rtol=1e-10)
    dc, dp, it, rel = prob.solve(cams, pts, obs, s.lam)
    assert prob.info()["n_levels"] == 1 and it <= 2
    sch, ex = _exact(s, s.lam)
    assert np.linalg.norm(_np(dc).ravel() - ex) <= 1e-7 * np.linalg.norm(ex)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lm_step_with_a_singular_jacobi_block_is_rejected(gpu, precision):
    """An unobserved camera at lambda = 0 has a zero diagonal block of S, which the Schur
    setup's block inverse finds not positive definite; inside ba_lm_step that failed solve
    is a rejection (x kept, cost unchanged, lambda times nu), and the next step at lambda >
    0 starts clean."""
    api, F_ = _api()
    base = scene("ring", seed=1, n_cams=20, n_pts=1500)
    s = _drop_camera_obs(base, 7)
    prec = F_.BA_FP64 if precision == "fp64" else F_.BA_MIXED
    prob, cams, pts, obs = api.from_scene(s, device=gpu, precision=prec, coarse_max_nodes=4)
    cost0 = prob.linearize(cams, pts, obs)
    c0, p0 = cams.clone(), pts.clone()
    lam, acc, cost = prob.lm_step(cams, pts, obs, 0.0)
    assert acc == 0 and lam == 0.0 and cost == cost0
    assert torch.equal(cams, c0) and torch.equal(pts, p0)
    with pytest.raises(api.BAError):
        prob.pcg_solve()        # the failed step left no setup to solve with
    # at lambda > 0 the step goes through and the observed cameras move
    lam, acc, cost = prob.lm_step(cams, pts, obs, 1e-3)
    assert acc == 1 and cost < cost0
    moved = np.abs(_np(cams) - _np(c0)).max(axis=1)
    assert np.all(np.delete(moved, 7) > 0.0)
