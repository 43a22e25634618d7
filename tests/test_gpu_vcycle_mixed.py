"""The mixed-precision V-cycle (Algorithm 1 with the Chebyshev smoother of Section 3.4, in
FP32) against the oracle's FP64 cycle, element by element.

The FP32 cycle cannot match the FP64 one to FP64 rounding, so its bound is derived from a
simulation of what FP32 does to the cycle: the oracle's own hierarchy with every stored
operator rounded to FP32 and the Galerkin products P^T A P formed in FP32 arithmetic
(NumPy float32), applied in FP32 arithmetic.  That simulated cycle's deviation from the
FP64 cycle, eta, measures the sensitivity of this cycle on this scene to FP32 storage
and arithmetic; the GPU cycle must stay within 10 eta of the FP64 cycle (other summation
orders give deviations of the same order; a wrong operator, prolongator or smoother
coefficient gives an O(1) one).  The Lanczos estimate lambda_max is a Ritz value whose FP32
and FP64 computations may differ slightly (Section 3.4 fixes only the procedure), so both
sides use the GPU's estimate for the Chebyshev interval.

A second check isolates the cycle's own arithmetic: the FP64 cycle evaluated on the GPU's
FP32 operators, Jacobi inverses, prolongators and coarsest inverse, against the same
cycle in NumPy float32 arithmetic.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from conftest import scene
from oracle import multigrid, schur

pytestmark = pytest.mark.gpu

CHAIN = dict(n_cams=300, n_pts=30000)
CMAX = 16


def _api():
    from paper_2007_01941_gb300 import _ffi, api
    return api, _ffi


def _np(t):
    return t.detach().cpu().numpy()


def _cycle(levels, r, dtype):
    """Algorithm 1 over given level data: per level A (sparse), Dinv (sparse block
    diagonal), P (sparse prolongator), Chebyshev interval (lo, hi); the coarsest level's
    dense inverse applied in FP64 (as both implementations do).  Vectors in dtype."""
    def cyc(l, b):
        L = levels[l]
        if "inv" in L:
            return (L["inv"] @ b.astype(np.float64)).astype(dtype)
        x = np.zeros_like(b)
        x = multigrid.chebyshev(L["A"], L["Dinv"], x, b, L["lo"], L["hi"], 2)
        rc = L["P"].T @ (b - L["A"] @ x)
        xc = cyc(l + 1, rc.astype(dtype))
        x = x + L["P"] @ xc
        return multigrid.chebyshev(L["A"], L["Dinv"], x, b, L["lo"], L["hi"], 2)
    return cyc(0, r.astype(dtype))


def _levels_from(ops, Ps, lams, dtype, level0_smoother=None):
    """Level data from per-level operators (sparse, FP64 values), prolongators and
    lambda_max: Jacobi inverses from the operator's diagonal blocks, all stored in dtype."""
    out = []
    for l, A in enumerate(ops):
        if l == len(ops) - 1:
            out.append({"inv": np.linalg.inv(A.astype(np.float64).toarray())})
            break
        b = 9 if l == 0 else 16
        Dinv = np.linalg.inv(multigrid.diag_blocks(A.astype(np.float64), b))
        Asm = level0_smoother if (l == 0 and level0_smoother is not None) else A
        out.append({"A": Asm.astype(dtype), "Dinv": schur.blockdiag_sparse(Dinv).astype(dtype),
                    "P": Ps[l].astype(dtype), "lo": 0.3 * lams[l], "hi": 1.1 * lams[l]})
    return out


def _fp32_operators(S0_32, H):
    """Level operators of the oracle's hierarchy rebuilt from the FP32 level-0 S with FP32
    prolongators and Galerkin products in FP32 arithmetic (same aggregates, same Q)."""
    ops, A = [S0_32], S0_32
    for L in H.levels[:-1]:
        A = multigrid.galerkin(A, L.P.astype(np.float32), L.kept).astype(np.float32)
        ops.append(A)
    return ops


def _gpu_levels(prob, F_, n_levels, dtype):
    """The GPU's own stored hierarchy (operators rounded to the FP32 the cycle reads)."""
    out = []
    for l in range(n_levels):
        rp = _np(prob.get_array(F_.BA_ARR_LEVEL_ROWPTR, l))
        if l == n_levels - 1:
            n = len(rp) - 1
            N = n * (9 if l == 0 else 16)
            Ainv = _np(prob.get_array(F_.BA_ARR_COARSE_INV, l))
            Np = int(round(np.sqrt(Ainv.size)))
            out.append({"inv": Ainv.reshape(Np, Np)[:N, :N]})
            break
        b = 9 if l == 0 else 16
        cols = _np(prob.get_array(F_.BA_ARR_LEVEL_COLS, l))
        vals = _np(prob.get_array(F_.BA_ARR_LEVEL_VALS, l)).reshape(-1, b, b).astype(np.float32)
        A = sp.bsr_matrix((vals, cols, rp), shape=((len(rp) - 1) * b,) * 2).tocsr()
        Dinv = _np(prob.get_array(F_.BA_ARR_JACOBI_INV, l)).reshape(-1, b, b).astype(np.float32)
        Q = _np(prob.get_array(F_.BA_ARR_PROLONG, l)).reshape(-1, b, 16).astype(np.float32)
        agg = _np(prob.get_array(F_.BA_ARR_AGG, l))
        lam = prob.info()["level_lambda_max"][l]
        out.append({"A": A.astype(dtype), "Dinv": schur.blockdiag_sparse(Dinv).astype(dtype),
                    "P": multigrid.prolongation_matrix(Q.astype(np.float64), agg).astype(dtype),
                    "lo": 0.3 * lam, "hi": 1.1 * lam})
    return out


def _inf(a):
    return float(np.abs(a).max())


# coarse_max_nodes 40 ends on a 576-dof coarsest level: the restriction into it is not folded
@pytest.mark.parametrize("level0,cmax", [("implicit", CMAX), ("explicit", CMAX), ("explicit", 40)])
def test_mixed_vcycle_matches_oracle(gpu, level0, cmax):
    api, F_ = _api()
    s = scene("street_chain", **CHAIN)
    op = {"implicit": F_.BA_OP_IMPLICIT, "explicit": F_.BA_OP_EXPLICIT}[level0]
    prob, cams, pts, obs = api.from_scene(s, device=gpu, precision=F_.BA_MIXED, coarse_max_nodes=cmax,
                                          level0_operator=op)
    prob.linearize(cams, pts, obs)
    prob.schur_setup(s.lam)
    prob.mg_setup()
    info = prob.info()
    assert info["level0_explicit"] == (level0 == "explicit")
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, s.lam)
    W = multigrid.covisibility(s.cam_idx, s.pt_idx, s.n_cams, s.n_pts)
    H = multigrid.Hierarchy(sch.S, W, s.cams, coarse_max_nodes=cmax)
    nl = len(H.levels)
    assert info["n_levels"] == nl and nl >= 3
    lams = info["level_lambda_max"]

    # FP64 cycle: the oracle's operators and prolongators, the GPU's lambda_max
    ops64 = [L.A for L in H.levels]
    Ps = [L.P for L in H.levels[:-1]]
    lev64 = _levels_from(ops64, Ps, lams, np.float64)
    # the simulated FP32 cycle: level 0 stored in FP32 (with the implicit level 0 the
    # smoother's products come from the FP32 Jacobian records: S formed from blocks
    # rounded to FP32), coarse operators by FP32 Galerkin products
    S0_32 = sch.S.astype(np.float32)
    sm0 = None
    if level0 == "implicit":
        sch32 = schur.Schur(sch.Fb.astype(np.float32).astype(np.float64),
                            sch.Eb.astype(np.float32).astype(np.float64), sch.f, s.cam_idx, s.pt_idx,
                            s.n_cams, s.n_pts, s.lam)
        sm0 = sch32.S.astype(np.float32)
    lev32 = _levels_from(_fp32_operators(S0_32, H), [P.astype(np.float32) for P in Ps], lams, np.float32, sm0)
    if level0 == "explicit":
        # the cycle's arithmetic alone, on the GPU's own stored hierarchy
        gl64 = _gpu_levels(prob, F_, nl, np.float64)
        gl32 = _gpu_levels(prob, F_, nl, np.float32)
    for seed in range(2):
        r = np.random.default_rng(seed).normal(size=9 * s.n_cams)
        z = _np(prob.precond_apply(torch.tensor(r, device=gpu)))
        ref = _cycle(lev64, r, np.float64)
        sim = _cycle(lev32, r, np.float32).astype(np.float64)
        eta = _inf(sim - ref) / _inf(ref)
        err = _inf(z - ref) / _inf(ref)
        assert eta < 1e-2, eta                      # the bound itself is meaningful
        assert err <= 10 * eta, (seed, err, eta)
        if level0 == "explicit":
            ref_g = _cycle(gl64, r, np.float64)
            sim_g = _cycle(gl32, r, np.float32).astype(np.float64)
            eta_g = _inf(sim_g - ref_g) / _inf(ref_g)
            err_g = _inf(z - ref_g) / _inf(ref_g)
            assert err_g <= 10 * eta_g, (seed, err_g, eta_g)


def test_mixed_hierarchy_below_the_damping_floor(gpu):
    """Below precond_lambda_min (1e-5) the mixed-precision hierarchy is built from S with
    its camera diagonal damped at that floor, S(lambda) + (mu - lambda) max(diag(J^T J),
    1e-6), while PCG solves S at the step's lambda: the FP32 cycle at lambda = 1e-8 matches
    the oracle's cycle built from that operator at the bound above, and the solve of
    S(1e-8) reaches its residual in about the iterations of the all-FP64 solve, whose
    hierarchy is built at lambda itself."""
    import scipy.sparse.linalg as spla
    api, F_ = _api()
    s = scene("street_chain", **CHAIN)
    lam, mu = 1e-8, 1e-5
    prob, cams, pts, obs = api.from_scene(s, device=gpu, precision=F_.BA_MIXED, coarse_max_nodes=CMAX,
                                          level0_operator=F_.BA_OP_EXPLICIT, rtol=1e-8, max_iters=3000)
    assert prob.options.precond_lambda_min == mu
    prob.linearize(cams, pts, obs)
    prob.schur_setup(lam)
    prob.mg_setup()
    lams = prob.info()["level_lambda_max"]
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, lam)
    # D_c = lam max(diag, 1e-6): the floor's extra camera damping is (mu - lam) / lam D_c
    S_mu = (sch.S + sp.diags((mu - lam) / lam * sch.Dc)).tocsr()
    W = multigrid.covisibility(s.cam_idx, s.pt_idx, s.n_cams, s.n_pts)
    H = multigrid.Hierarchy(S_mu, W, s.cams, coarse_max_nodes=CMAX)
    Ps = [L.P for L in H.levels[:-1]]
    lev64 = _levels_from([L.A for L in H.levels], Ps, lams, np.float64)
    lev32 = _levels_from(_fp32_operators(S_mu.astype(np.float32), H), [P.astype(np.float32) for P in Ps],
                         lams, np.float32)
    for seed in range(2):
        r = np.random.default_rng(seed).normal(size=9 * s.n_cams)
        z = _np(prob.precond_apply(torch.tensor(r, device=gpu)))
        ref = _cycle(lev64, r, np.float64)
        eta = _inf(_cycle(lev32, r, np.float32).astype(np.float64) - ref) / _inf(ref)
        assert eta < 1e-2 and _inf(z - ref) / _inf(ref) <= 10 * eta, (seed, eta)
    # the solve is of S(lambda), not S(mu)
    dc, it_mixed, rel = prob.pcg_solve()
    assert rel <= 1e-8
    d = _np(dc).ravel()
    assert np.linalg.norm(sch.b - sch.S @ d) <= 2e-8 * np.linalg.norm(sch.b)
    p64, c64, x64, o64 = api.from_scene(s, device=gpu, precision=F_.BA_FP64, coarse_max_nodes=CMAX,
                                        rtol=1e-8, max_iters=3000)
    _, _, it64, _ = p64.solve(c64, x64, o64, lam)
    assert it_mixed <= 1.3 * it64 + 2, (it_mixed, it64)
