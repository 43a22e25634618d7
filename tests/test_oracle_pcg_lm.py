"""Pins of the oracle's PCG, LM step and adjoint."""
import numpy as np
import scipy.linalg as sla

from conftest import scene
from oracle import adjoint, camera, lm, pcg, schur


def test_pcg_multigrid_matches_dense_cholesky():
    s = scene("ring", seed=0)
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, s.lam)
    dc, dp, it, rel = lm.solve_step(sch, s.cams, "mg", rtol=1e-13, coarse_max_nodes=4)
    ref = sla.cho_solve(sla.cho_factor(sch.S.toarray()), sch.b)
    assert np.linalg.norm(dc - ref) <= 1e-8 * np.linalg.norm(ref)


def test_iterations_fall_as_the_preconditioner_strengthens():
    # Section 5: multigrid needs fewer CG iterations than point block Jacobi
    s = scene("street_chain", n_cams=300, n_pts=30000)
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, s.lam)
    its = {}
    for pc in ("none", "jacobi", "mg"):
        _, _, its[pc], rel = lm.solve_step(sch, s.cams, pc, rtol=1e-6, max_iters=3000, coarse_max_nodes=16)
        if pc != "none":               # unpreconditioned CG stalls on the badly scaled system
            assert rel <= 1e-6
    assert its["none"] > its["jacobi"] > its["mg"]


def _spd(n, cond, seed):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.normal(size=(n, n)))
    return (Qm * np.geomspace(1.0, cond, n)) @ Qm.T, rng.normal(size=n)


def test_nash_sofer_stop_matches_textbook_cg_and_definition():
    """Section 2.1's forcing rule: the stop is the first i with i (Q_i - Q_{i-1}) / Q_i <= tau,
    Q_i = 1/2 x_i^T A x_i - x_i^T b, Q_0 = 0.  A textbook CG loop written here, with Q
    from a dense product, finds the same i."""
    A, b = _spd(120, 1e4, 3)
    for tau in (0.5, 0.1, 0.01):
        x_o, it_o, _, _ = pcg.pcg(lambda v: A @ v, b, None, rtol=0.0, max_iters=500, stop="nash_sofer", tau=tau)
        x = np.zeros_like(b)
        r = b.copy()
        d = r.copy()
        q_prev, stop_at = 0.0, None
        for i in range(1, 500):
            Ad = A @ d
            a = (r @ r) / (d @ Ad)
            x = x + a * d
            r_new = r - a * Ad
            d = r_new + ((r_new @ r_new) / (r @ r)) * d
            r = r_new
            q = 0.5 * x @ A @ x - x @ b
            if i * (q - q_prev) / q <= tau:
                stop_at = i
                break
            q_prev = q
        assert stop_at is not None and it_o == stop_at, (tau, it_o, stop_at)
        assert np.linalg.norm(x_o - x) <= 1e-10 * np.linalg.norm(x)


def test_quadratic_model_decreases_to_its_minimum():
    # CG minimises Q over growing Krylov spaces: Q_i decreases towards -1/2 b^T A^-1 b
    A, b = _spd(60, 1e3, 4)
    qs = []
    for it in list(range(1, 40)) + [400]:
        x, _, _, _ = pcg.pcg(lambda v: A @ v, b, None, rtol=0.0, max_iters=it)
        qs.append(pcg.quadratic_model(lambda v: A @ v, b, x))
    assert all(q1 <= q0 + 1e-9 * abs(q0) for q0, q1 in zip(qs, qs[1:]))
    qmin = -0.5 * b @ np.linalg.solve(A, b)
    assert abs(qs[-1] - qmin) <= 1e-10 * abs(qmin)


def test_nash_sofer_solves_tighter_with_the_stronger_preconditioner():
    # Section 2.1: the iteration count in the rule makes a stronger preconditioner stop
    # at a tighter tolerance
    s = scene("street_chain", n_cams=300, n_pts=30000)
    sch = schur.linearize(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, s.lam)
    res = {}
    for pc in ("jacobi", "mg"):
        dc, _, it, _ = lm.solve_step(sch, s.cams, pc, rtol=0.0, max_iters=3000, stop="nash_sofer", tau=0.1,
                                     coarse_max_nodes=16)
        res[pc] = np.linalg.norm(sch.b - sch.S @ dc) / np.linalg.norm(sch.b)
    assert res["mg"] < res["jacobi"]


def test_pcg_zero_rhs_and_identity():
    x, it, rel, _ = pcg.pcg(lambda v: 2 * v, np.zeros(5))
    assert it == 0 and np.all(x == 0)
    b = np.arange(1.0, 6.0)
    x, it, rel, _ = pcg.pcg(lambda v: 2 * v, b)
    assert it == 1 and np.allclose(x, b / 2)


def test_lm_step_decreases_cost_and_updates_lambda():
    s = scene("ring", seed=0)
    c1, p1, lam1, nu1, acc, cost0, cost1, info = lm.lm_step(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 1e-4,
                                                             rtol=1e-10, coarse_max_nodes=4)
    assert acc and cost1 < cost0
    rho = info["rho"]
    assert np.isclose(lam1, 1e-4 * max(1 / 3, 1 - (2 * rho - 1) ** 3))
    assert np.isclose(camera.cost(c1, p1, s.cam_idx, s.pt_idx, s.obs), cost1)


def test_lm_step_near_the_optimum_has_unit_gain_ratio():
    """Close to the optimum the Gauss-Newton model is exact to second order, so the gain
    ratio (actual over predicted decrease, each computed its own way: the cost from the
    camera model, the prediction from g and D) tends to 1 and lambda falls by the factor
    1/3 that the update rule gives at rho = 1."""
    s = scene("ring", seed=0, n_cams=16, n_pts=800)
    x, p, lam, nu = s.cams, s.pts, 1e-4, 2.0
    for _ in range(2):   # two steps bring the start within the quadratic region
        x, p, lam, nu, acc, *_ = lm.lm_step(x, p, s.cam_idx, s.pt_idx, s.obs, lam, nu, rtol=1e-12,
                                            coarse_max_nodes=4)
        assert acc
    c1, p1, lam1, nu1, acc, cost0, cost1, info = lm.lm_step(x, p, s.cam_idx, s.pt_idx, s.obs, lam, nu,
                                                            rtol=1e-12, coarse_max_nodes=4)
    assert acc and cost1 < cost0 and nu1 == 2.0
    assert abs(info["rho"] - 1.0) < 1e-2
    assert abs(lam1 / lam - 1.0 / 3.0) < 1e-6


def rejecting_scene():
    # a 16-camera ring whose starting rotations are off by N(0, 0.8^2) per component: the
    # first step is accepted, the next three overshoot (points cross the image planes)
    from paper_2007_01941_gb300 import scenes
    return scenes.rotated_start(scene("ring", seed=0, n_cams=16, n_pts=800), 0.8, seed=11)


def test_lm_step_rejects_and_raises_lambda():
    """The reject branch: when the cost at x + delta exceeds the cost at x, the step is
    refused, x is unchanged, lambda is multiplied by nu and nu doubles (each rejection in
    a row doubles the factor)."""
    s = rejecting_scene()
    x, p, lam, nu = s.cams, s.pts, 1e-4, 2.0
    x, p, lam, nu, acc, *_ = lm.lm_step(x, p, s.cam_idx, s.pt_idx, s.obs, lam, nu, rtol=1e-10,
                                        coarse_max_nodes=4)
    assert acc
    for k in range(2):
        sch = schur.linearize(x, p, s.cam_idx, s.pt_idx, s.obs, lam)
        dc, dp, _, _ = lm.solve_step(sch, x, "mg", rtol=1e-10, coarse_max_nodes=4)
        cost_x = camera.cost(x, p, s.cam_idx, s.pt_idx, s.obs)
        cost_trial = camera.cost(x + dc.reshape(-1, 9), p + dp.reshape(-1, 3), s.cam_idx, s.pt_idx, s.obs)
        assert cost_trial > cost_x          # the step overshoots: the cost rises
        x1, p1, lam1, nu1, acc, cost0, cost1, info = lm.lm_step(x, p, s.cam_idx, s.pt_idx, s.obs, lam, nu,
                                                                rtol=1e-10, coarse_max_nodes=4)
        assert not acc
        assert info["rho"] < 0
        assert x1 is x and p1 is p
        assert lam1 == lam * nu and nu1 == 2.0 * nu
        assert cost0 == cost1 == cost_x
        lam, nu = lam1, nu1
    assert nu == 8.0


def _fd_loss(s, vbar, cams, pts, obs, lam):
    sch = schur.linearize(cams, pts, s.cam_idx, s.pt_idx, obs, lam)
    dc, dp = adjoint.solve_delta(sch)
    return vbar @ np.concatenate([dc, dp])


def test_adjoint_matches_central_differences():
    s = scene("ring", seed=5, n_cams=6, n_pts=40, kmin=2, kmax=4)
    lam = 1e-2
    rng = np.random.default_rng(0)
    vbar = rng.normal(size=9 * s.n_cams + 3 * s.n_pts)
    go, gc, gp, _ = adjoint.adjoint(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, lam, vbar)
    for (arr, grad, which) in ((s.obs, go, "obs"), (s.cams, gc, "cams"), (s.pts, gp, "pts")):
        for _ in range(6):
            i = rng.integers(arr.shape[0])
            j = rng.integers(arr.shape[1])
            # kappa(S) ~ 1e7 here: h = 1e-4 balances truncation against amplified rounding
            h = 1e-4 * max(1.0, abs(arr[i, j]))
            ap, am = arr.copy(), arr.copy()
            ap[i, j] += h
            am[i, j] -= h
            args = {"cams": s.cams, "pts": s.pts, "obs": s.obs}
            args[which] = ap
            lp = _fd_loss(s, vbar, args["cams"], args["pts"], args["obs"], lam)
            args[which] = am
            lm_ = _fd_loss(s, vbar, args["cams"], args["pts"], args["obs"], lam)
            fd = (lp - lm_) / (2 * h)
            scale = np.abs(grad).max()
            assert abs(fd - grad[i, j]) <= 1e-5 * max(abs(fd), 1e-3 * scale), (which, i, j, fd, grad[i, j])


def test_adjoint_is_linear_in_the_cotangent():
    s = scene("ring", seed=5, n_cams=6, n_pts=40, kmin=2, kmax=4)
    rng = np.random.default_rng(1)
    v1, v2 = rng.normal(size=(2, 9 * s.n_cams + 3 * s.n_pts))
    a = adjoint.adjoint(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 1e-3, v1)
    b = adjoint.adjoint(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 1e-3, v2)
    c = adjoint.adjoint(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 1e-3, 2 * v1 - v2)
    for k in range(3):
        assert np.allclose(c[k], 2 * a[k] - b[k], rtol=1e-9, atol=1e-9 * np.abs(a[k]).max())


def test_lm_step_with_a_failed_solve_is_a_rejection(monkeypatch):
    """A solve that fails (here: the coarsest factorisation raising, planted in the oracle)
    leaves x unchanged and grows lambda as a rejection does."""
    s = scene("ring", seed=0, n_cams=16, n_pts=800)

    def failing(*a, **k):
        raise np.linalg.LinAlgError("planted: not positive definite")
    monkeypatch.setattr(lm, "solve_step", failing)
    x1, p1, lam1, nu1, acc, cost0, cost1, info = lm.lm_step(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs, 1e-4, 4.0)
    assert not acc and x1 is s.cams and p1 is s.pts
    assert lam1 == 4e-4 and nu1 == 8.0
    assert cost0 == cost1 == camera.cost(s.cams, s.pts, s.cam_idx, s.pt_idx, s.obs)
