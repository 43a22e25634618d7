"""The benchmarked configuration against the oracle, at its full size.

Street-chain scene (2,000 cameras, 300,000 points, 1,499,558 observations), mixed
precision, the default options the benchmark times: AUTO level-0 operator (the assembled
S, Section 3.6), fused V-cycle phases, programmatic dependent launches, coarse_max_nodes
32 (a 5-level hierarchy 2000/727/228/72/21 with a 336-dof coarsest inverse).  The oracle
(Section 2.1, Section 3, Algorithm 1, Algorithm 2) takes about half a minute here, once
per module.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

from oracle import camera, lm, multigrid, pcg, schur

pytestmark = pytest.mark.gpu

CMAX = 32


def _api():
    from paper_2007_01941_gb300 import _ffi, api
    return api, _ffi


def _np(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def chain():
    from paper_2007_01941_gb300 import scenes
    s = scenes.street_chain()
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, s.lam)
    W = multigrid.covisibility(s.cam_idx, s.pt_idx, s.n_cams, s.n_pts)
    H = multigrid.Hierarchy(sch.S, W, s.cams, coarse_max_nodes=CMAX)
    exact = spla.splu(sch.S.tocsc()).solve(sch.b)     # sparse direct solve of S delta_c = b
    return s, sch, H, exact


def _problem(s, gpu, **kw):
    api, F_ = _api()
    opt = dict(precision=F_.BA_MIXED, rtol=1e-6, max_iters=2000, coarse_max_nodes=CMAX)
    opt.update(kw)
    prob, cams, pts, obs = api.from_scene(s, device=gpu, **opt)
    o = prob.options
    assert o.level0_operator == F_.BA_OP_AUTO and o.fused_vcycle == 1 and o.overlap_launches == 1
    return prob, cams, pts, obs


def _bsr(prob, F_, l, b):
    rp = _np(prob.get_array(F_.BA_ARR_LEVEL_ROWPTR, l))
    cols = _np(prob.get_array(F_.BA_ARR_LEVEL_COLS, l))
    vals = _np(prob.get_array(F_.BA_ARR_LEVEL_VALS, l)).reshape(-1, b, b)
    n = len(rp) - 1
    return rp, cols, vals, sp.bsr_matrix((vals, cols, rp), shape=(n * b, n * b))


def test_fullsize_hierarchy_matches_oracle(gpu, chain):
    """Every level: covisibility pattern and counts, strength order, aggregates and kept
    coarse dofs bit-exact; operators, near-nullspace, prolongators, Jacobi inverses,
    lambda_max and the coarsest inverse at the mixed-precision tolerances of the
    300-camera hierarchy test."""
    api, F_ = _api()
    s, sch, H, _ = chain
    prob, cams, pts, obs = _problem(s, gpu)
    prob.linearize(cams, pts, obs)
    prob.schur_setup(s.lam)
    prob.mg_setup()
    info = prob.info()
    assert info["level0_explicit"]
    assert info["n_levels"] == len(H.levels) == 5
    assert info["level_nodes"] == [L.n for L in H.levels]
    for l, L in enumerate(H.levels):
        b = L.b
        rp, cols, vals, Ag = _bsr(prob, F_, l, b)
        Wc = L.W.tocsr()
        Wc.sort_indices()
        assert np.array_equal(rp, Wc.indptr) and np.array_equal(cols, Wc.indices), l        # bit-exact
        assert np.array_equal(_np(prob.get_array(F_.BA_ARR_LEVEL_W, l)), Wc.data), l        # bit-exact
        D = (Ag.tocsr() - L.A).tobsr(blocksize=(b, b))
        scale = np.abs(L.A.data).max()
        if l == 0:
            # the paired-FP32 assembly: FP64-grade blocks, each against the scale of its
            # two diagonal blocks (see the 300-camera hierarchy test)
            assert np.abs(D.data).max() <= 1e-10 * scale
            dg = np.abs(multigrid.diag_blocks(L.A, b)).max(axis=(1, 2))
            row = np.repeat(np.arange(L.n), np.diff(D.indptr))
            err = np.abs(D.data).max(axis=(1, 2))
            assert np.all(err <= 1e-10 * np.sqrt(dg[row] * dg[D.indices])), l
        else:
            assert np.abs(D.data).max() <= 2e-4 * scale, (l, np.abs(D.data).max() / scale)
        K = _np(prob.get_array(F_.BA_ARR_NULLSPACE, l)).reshape(L.n, b, 16)
        assert np.abs(K - L.K).max() <= (1e-11 if l == 0 else 1e-8) * np.abs(L.K).max(), l
        if l == len(H.levels) - 1:
            N = L.n * b
            Ainv = _np(prob.get_array(F_.BA_ARR_COARSE_INV, l))
            Np = int(round(np.sqrt(Ainv.size)))
            ref = np.linalg.inv(L.dense)
            assert np.abs(Ainv.reshape(Np, Np)[:N, :N] - ref).max() <= 5e-3 * np.abs(ref).max()
            continue
        Dinv = _np(prob.get_array(F_.BA_ARR_JACOBI_INV, l)).reshape(L.n, b, b)
        Dref = np.linalg.inv(multigrid.diag_blocks(Ag.tocsr(), b))
        assert np.abs(Dinv - Dref).max() <= 1e-6 * np.abs(Dref).max(), l
        sptr = _np(prob.get_array(F_.BA_ARR_STRENGTH_PTR, l))
        sidx = _np(prob.get_array(F_.BA_ARR_STRENGTH_IDX, l))
        flat = np.concatenate([np.asarray(o, dtype=np.int64) for o in L.order])
        assert np.array_equal(sptr, np.concatenate([[0], np.cumsum([len(o) for o in L.order])])), l   # bit-exact
        assert np.array_equal(sidx, flat), l                                                          # bit-exact
        assert np.array_equal(_np(prob.get_array(F_.BA_ARR_AGG, l)), L.agg), l                       # bit-exact
        kept = _np(prob.get_array(F_.BA_ARR_KEPT, l + 1)).view(np.uint32)
        assert np.array_equal(kept, (L.kept * (1 << np.arange(16))).sum(axis=1).astype(np.uint32)), l
        Q = _np(prob.get_array(F_.BA_ARR_PROLONG, l)).reshape(L.n, b, 16)
        assert np.abs(Q - L.Q).max() < 1e-9, l
        assert abs(info["level_lambda_max"][l] - L.lam_max) <= 1e-3 * L.lam_max, l


def test_fullsize_solution_matches_oracle(gpu, chain):
    """At rtol 1e-10 the mixed solve lands within 1e-6 of the sparse direct solution
    (delta_c and the back-substituted delta_p) and its true FP64 residual reaches the
    target.  At the benchmark's rtol 1e-6 the true FP64 residual is within 1.5e-6, the
    iteration count within 5 % of the oracle's own multigrid PCG, and the iterate as close
    to the direct solution as the oracle's iterate at the same rtol."""
    api, F_ = _api()
    s, sch, H, exact = chain
    nb = np.linalg.norm(sch.b)
    dp_exact = sch.back_substitute(exact)
    for rtol in (1e-10, 1e-6):
        prob, cams, pts, obs = _problem(s, gpu, rtol=rtol)
        dc, dp, it, rel = prob.solve(cams, pts, obs, s.lam)
        assert rel <= rtol
        d = _np(dc).ravel()
        true_rel = np.linalg.norm(sch.b - sch.S @ d) / nb
        err = np.linalg.norm(d - exact) / np.linalg.norm(exact)
        err_p = np.linalg.norm(_np(dp).ravel() - dp_exact) / np.linalg.norm(dp_exact)
        if rtol == 1e-10:
            assert true_rel <= 2e-10, true_rel
            assert err <= 1e-6 and err_p <= 1e-6, (err, err_p)
        else:
            x_o, it_o, rel_o, _ = pcg.pcg(lambda v: sch.S @ v, sch.b, H.apply, rtol, 2000)
            err_o = np.linalg.norm(x_o - exact) / np.linalg.norm(exact)
            assert true_rel <= 1.5e-6, true_rel
            assert abs(it - it_o) <= max(1, it_o // 20), (it, it_o)
            assert err <= 2 * err_o, (err, err_o)
        prob.close()


def test_fullsize_lm_step_matches_oracle(gpu, chain):
    """The benchmark's timed call, ba_lm_step at rtol 1e-6, twice on one problem (the
    second setup refreshes the cached hierarchy at the new point): acceptance, cost and
    lambda as the oracle's, and the camera and point displacements within twice the
    oracle's own forward error at that rtol (one step) of the oracle's."""
    api, F_ = _api()
    s, sch, H, exact = chain
    prob, cams, pts, obs = _problem(s, gpu)
    x, p, lam, nu = s.cams, s.pts, s.lam, 2.0
    lam_g = s.lam
    dx_ex = exact.reshape(-1, 9)
    for k in range(2):
        lam_g, acc_g, cost_g = prob.lm_step(cams, pts, obs, lam_g)
        x, p, lam, nu, acc, cost0, cost1, info = lm.lm_step(x, p, s.cam_idx, s.pt_idx, s.obs, lam, nu, rtol=1e-6,
                                                            max_iters=2000, coarse_max_nodes=CMAX)
        assert acc_g == acc and acc, k
        assert abs(cost_g - cost1) <= 1e-6 * cost1, (k, cost_g, cost1)
        assert abs(lam_g - lam) <= 1e-3 * lam, (k, lam_g, lam)
        if k == 0:
            # one step from the common start: the displacement is delta itself
            err_o = np.linalg.norm((x - s.cams) - dx_ex) / np.linalg.norm(dx_ex)
            err_g = np.linalg.norm((_np(cams) - s.cams) - dx_ex) / np.linalg.norm(dx_ex)
            assert err_g <= 2 * err_o + 1e-6, (err_g, err_o)
    assert abs(camera.cost(_np(cams), _np(pts), s.cam_idx, s.pt_idx, s.obs) - cost_g) <= 1e-9 * cost_g
