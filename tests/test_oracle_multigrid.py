"""Pins of the oracle's multigrid pieces (Section 3, Algorithms 1 and 2)."""
import json
import os

import numpy as np
import scipy.sparse as sp
from numpy.polynomial import chebyshev as npcheb
from scipy.spatial.transform import Rotation

from conftest import scene
from oracle import multigrid, schur
from oracle.rng import splitmix64, uniform_pm1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "aggregation_hand.json")


def test_splitmix64_published_vectors():
    # first outputs of SplitMix64 from state 0 (Steele, Lea & Flood 2014 reference code)
    assert [int(v) for v in splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = uniform_pm1(0, 1000)
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.1


def test_covisibility_counts_brute_force():
    s = scene("ring", seed=1, n_cams=10, n_pts=150, kmin=2, kmax=5)
    W = multigrid.covisibility(s.cam_idx, s.pt_idx, s.n_cams, s.n_pts).toarray()
    seen = [set(s.pt_idx[s.cam_idx == c]) for c in range(s.n_cams)]
    for i in range(s.n_cams):
        for j in range(s.n_cams):
            assert W[i, j] == len(seen[i] & seen[j])


def test_strength_order_and_aggregation_golden():
    g = json.load(open(GOLDEN))
    for case in g["graphs"]:
        W = sp.csr_matrix(np.array(case["W"], dtype=np.int64))
        order = multigrid.strength_order(W)
        assert order == case["order"]
        assert list(multigrid.aggregate(order, 20)) == case["agg_cap20"]
        assert list(multigrid.aggregate(order, 2)) == case["agg_cap2"]


def test_strength_order_matches_float_metric_without_ties():
    s = scene("street_chain", n_cams=80, n_pts=4000)
    W = multigrid.covisibility(s.cam_idx, s.pt_idx, s.n_cams, s.n_pts)
    G = multigrid.strength_matrix(W).toarray()
    order = multigrid.strength_order(W)
    for i, nb in enumerate(order):
        vals = G[i, nb]
        assert np.all(np.diff(vals) <= 1e-15)
        assert set(nb) == set(np.flatnonzero(G[i] > 0))


def test_aggregation_invariants_and_size_statistics():
    # every node aggregated, cap respected; Section 3.2 reports aggregates of about
    # 3 to 8 cameras with a mean a little above 3
    s = scene("street_chain", n_cams=400, n_pts=40000)
    W = multigrid.covisibility(s.cam_idx, s.pt_idx, s.n_cams, s.n_pts)
    agg = multigrid.aggregate(multigrid.strength_order(W), 20)
    sizes = np.bincount(agg)
    assert agg.min() == 0 and np.all(sizes >= 1) and sizes.max() <= 20
    assert 2.0 <= sizes.mean() <= 8.0


def test_nullspace_rotation_columns_match_scipy_derivative():
    rng = np.random.default_rng(4)
    for _ in range(5):
        cam = np.concatenate([rng.normal(size=3) * 1.2, rng.normal(size=3), [500, 0, 0]])
        K = multigrid.nullspace_camera_block(cam)
        Rc = Rotation.from_rotvec(cam[:3])
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            plus = (Rc * Rotation.from_rotvec(-e)).as_rotvec()
            minus = (Rc * Rotation.from_rotvec(e)).as_rotvec()
            fd = (plus - minus) / 2e-6
            assert np.allclose(K[0:3, 3 + k], fd, atol=1e-7)
            assert np.allclose(K[3:6, k], -Rc.as_matrix()[:, k])


def test_mgs_qr_properties_and_rank():
    s = scene("ring", seed=0, n_cams=16, n_pts=800)
    K = multigrid.nullspace(s.cams)
    for members, rank in (([0], 9), ([0, 1], 15), ([0, 1, 2, 3], 16)):
        Ka = np.concatenate([K[i] for i in members])
        Q, R, kept = multigrid.mgs_qr(Ka)
        assert kept.sum() == rank
        assert np.allclose(Q.T @ Q, np.diag(kept.astype(float)), atol=1e-12)
        assert np.abs(Q @ R - Ka).max() <= 1e-12 * np.abs(Ka).max()
        assert np.allclose(np.triu(R), R)


def _hier(s, lam=1e-4, **kw):
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, lam)
    W = multigrid.covisibility(s.cam_idx, s.pt_idx, s.n_cams, s.n_pts)
    return sch, multigrid.Hierarchy(sch.S, W, s.cams, **kw)


def test_galerkin_equals_dense_triple_product():
    s = scene("street_chain", n_cams=60, n_pts=3000)
    sch, H = _hier(s, coarse_max_nodes=4)
    L0, L1 = H.levels[0], H.levels[1]
    P = L0.P.toarray()
    ref = P.T @ sch.S.toarray() @ P
    pad = ~L0.kept.ravel()
    ref[pad, pad] = 1.0
    assert np.abs(L1.A.toarray() - ref).max() <= 1e-12 * np.abs(ref).max()
    # prolongator columns are orthonormal per aggregate
    assert np.allclose(P.T @ P, np.diag((~pad).astype(float)), atol=1e-12)


def test_chebyshev_error_is_the_scaled_chebyshev_polynomial():
    lam = np.linspace(0.05, 1.0, 40)
    A = sp.diags(lam).tocsr()
    Dinv = sp.identity(40, format="csr")
    e = np.random.default_rng(0).normal(size=40)
    lo, hi = 0.3, 1.1
    x = multigrid.chebyshev(A, Dinv, np.zeros(40), A @ e, lo, hi, steps=2)
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    T2 = lambda t: npcheb.chebval(t, [0, 0, 1])
    expect = T2((theta - lam) / delta) / T2(theta / delta) * e
    assert np.allclose(e - x, expect, atol=1e-13)


def test_lanczos_estimate_is_a_lower_bound_close_to_lambda_max():
    s = scene("ring", seed=0, n_cams=16, n_pts=800)
    sch, H = _hier(s, coarse_max_nodes=4)
    L = H.levels[0]
    ev = np.linalg.eigvals(L.Dinv.toarray() @ sch.S.toarray()).real.max()
    assert L.lam_max <= ev * (1 + 1e-10)
    assert L.lam_max >= 0.8 * ev


def test_vcycle_is_symmetric_positive_definite():
    s = scene("street_chain", n_cams=60, n_pts=3000)
    sch, H = _hier(s, coarse_max_nodes=4)
    assert len(H.levels) >= 3
    rng = np.random.default_rng(1)
    u, v = rng.normal(size=(2, sch.S.shape[0]))
    Mu, Mv = H.apply(u), H.apply(v)
    assert abs(u @ Mv - v @ Mu) <= 1e-10 * abs(u @ Mv)
    assert u @ Mu > 0 and v @ Mv > 0


def test_single_level_hierarchy_is_the_exact_inverse():
    s = scene("ring", seed=0, n_cams=16, n_pts=800)
    sch, H = _hier(s, coarse_max_nodes=100)
    assert len(H.levels) == 1
    r = np.random.default_rng(2).normal(size=sch.S.shape[0])
    assert np.allclose(sch.S @ H.apply(r), r, rtol=0, atol=1e-8 * np.abs(r).max())
