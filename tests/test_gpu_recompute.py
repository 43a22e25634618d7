"""Recompute mode of the implicit Schur product (recompute_jacobian = 1): the FP64 product
S x = D_c x + sum_o F_o^T (F_o x_c - E_o C_p^-1 sum_{o' in p} E_o'^T F_o' x_c') with F_o and
E_o rebuilt from the cameras and points inside the product (Section 3.6's implicit
operator, the camera model of Section 2.1), against the oracle's explicit S x, and the
solves that use it against the dense solution."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

from conftest import scene
from oracle import camera, robust, schur

pytestmark = pytest.mark.gpu

CHAIN = dict(n_cams=300, n_pts=30000)
SCENES = {"ring": lambda: scene("ring", seed=0),
          "chain": lambda: scene("street_chain", **CHAIN),
          # points seen by up to 48 cameras: the >32-observation tile path
          "bigpoints": lambda: scene("ring", seed=7, n_cams=48, n_pts=300, kmin=20, kmax=48)}


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("which", sorted(SCENES))
def test_recompute_product_matches_explicit_oracle(gpu, which):
    from paper_2007_01941_gb300 import _ffi, api
    s = SCENES[which]()
    prob, cams, pts, obs = api.from_scene(s, device=gpu, precision=_ffi.BA_FP64, recompute_jacobian=1)
    prob.linearize(cams, pts, obs)
    prob.schur_setup(s.lam)
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, s.lam)
    for seed in range(2):
        x = np.random.default_rng(seed).normal(size=(s.n_cams, 9))
        ref = sch.S @ x.ravel()
        y = _np(prob.schur_matvec(torch.tensor(x, device=gpu))).ravel()
        assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref), which
    prob.set_kernel_timing(True)
    prob.schur_matvec(torch.tensor(x, device=gpu))
    assert prob.kernel_timing(_ffi.BA_KT_SCHUR_RECOMPUTE)[1] == 1        # the recompute kernel ran
    assert prob.kernel_timing(_ffi.BA_KT_SCHUR_FP64)[1] == 0
    prob.set_kernel_timing(False)


def test_recompute_product_with_huber_weights(gpu):
    """Under the Huber loss the rebuilt blocks carry the robust weight w_o = sqrt(rho'):
    the product is that of the corrected Jacobian."""
    from paper_2007_01941_gb300 import _ffi, api
    s = scene("ring", seed=0, outlier_frac=0.05)
    f = camera.residuals(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs)
    a = float(np.median(np.sqrt(np.sum(f * f, axis=1))))
    prob, cams, pts, obs = api.from_scene(s, device=gpu, precision=_ffi.BA_FP64, recompute_jacobian=1,
                                          loss=_ffi.BA_LOSS_HUBER, loss_scale=a)
    prob.linearize(cams, pts, obs)
    prob.schur_setup(s.lam)
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, s.lam, huber=a)
    w = robust.weights(f, a)
    assert (w < 1.0).any()
    x = np.random.default_rng(1).normal(size=(s.n_cams, 9))
    ref = sch.S @ x.ravel()
    y = _np(prob.schur_matvec(torch.tensor(x, device=gpu))).ravel()
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_recompute_solve_matches_dense(gpu, precision):
    """PCG with the implicit operator in recompute mode (FP64: the PCG product and the
    V-cycle's level 0; mixed: the FP64 outer product, whose records are then never
    formed): the dense solution, in the iterations of the stored mode."""
    from paper_2007_01941_gb300 import _ffi, api
    s = scene("street_chain", **CHAIN)
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, s.lam)
    exact = sla.cho_solve(sla.cho_factor(sch.S.toarray()), sch.b)
    prec = {"fp64": _ffi.BA_FP64, "mixed": _ffi.BA_MIXED}[precision]
    rtol = 1e-12 if precision == "fp64" else 1e-10
    its = {}
    for rc in (0, 1):
        kw = dict(precision=prec, coarse_max_nodes=16, rtol=rtol, max_iters=5000,
                  level0_operator=_ffi.BA_OP_IMPLICIT, recompute_jacobian=rc)
        if precision == "mixed":
            kw["outer_product"] = _ffi.BA_OUTER_FP64
        prob, cams, pts, obs = api.from_scene(s, device=gpu, **kw)
        prob.set_kernel_timing(True)
        dc, dp, it, rel = prob.solve(cams, pts, obs, s.lam)
        n_rc = prob.kernel_timing(_ffi.BA_KT_SCHUR_RECOMPUTE)[1]
        prob.set_kernel_timing(False)
        assert (n_rc > 0) == bool(rc)
        assert rel <= rtol
        d = _np(dc).ravel()
        assert np.linalg.norm(d - exact) <= (1e-8 if precision == "fp64" else 1e-6) * np.linalg.norm(exact)
        its[rc] = it
        prob.close()
    assert abs(its[0] - its[1]) <= 1, its
