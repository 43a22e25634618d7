"""A full LM run on the loop-closure scene (10,000 cameras on a closed loop with cross-loop
links, 1,000,000 points, 8,189,552 observations, 2 % parameter perturbation): 50
iterations of ba_lm_step with multigrid-PCG solves to 1e-6 relative residual, in mixed
precision and in FP64.  The mixed run must end within 1e-6 relative of the FP64 run's
final cost (its FP32 V-cycle changes only how fast each solve converges; the outer
operator, residual and step control are FP64-valued), and both runs must decrease the
cost at every accepted step and leave it unchanged at every rejected one.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

STEPS = 50


def _run(s, gpu, precision):
    from paper_2007_01941_gb300 import api
    prob, cams, pts, obs = api.from_scene(s, device=gpu, precision=precision, rtol=1e-6, max_iters=2000,
                                          coarse_max_nodes=32)
    cost0 = prob.linearize(cams, pts, obs)
    lam, costs, accepted = s.lam, [cost0], []
    for _ in range(STEPS):
        lam, acc, cost = prob.lm_step(cams, pts, obs, lam)
        accepted.append(acc)
        costs.append(cost)
    prob.close()
    return np.array(costs), accepted


def test_loop_closure_lm_run_mixed_matches_fp64(gpu):
    from paper_2007_01941_gb300 import _ffi, scenes
    s = scenes.loop_closure()
    runs = {p: _run(s, gpu, code) for p, code in (("fp64", _ffi.BA_FP64), ("mixed", _ffi.BA_MIXED))}
    for name, (costs, acc) in runs.items():
        for k, a in enumerate(acc):
            if a:
                assert costs[k + 1] < costs[k], (name, k)
            else:
                # the cost at the unchanged point, evaluated again by this step's linearisation
                # (mixed: paired-FP32 sums, ~kappa u |obs| / |f| of the cost)
                assert abs(costs[k + 1] - costs[k]) <= (1e-12 if name == "fp64" else 1e-9) * costs[k], (name, k)
        assert costs[-1] < costs[0], name
    c64, c32 = runs["fp64"][0][-1], runs["mixed"][0][-1]
    assert abs(c32 - c64) <= 1e-6 * c64, (c32, c64)
