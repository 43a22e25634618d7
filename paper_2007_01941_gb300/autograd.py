"""torch.autograd wrapper of one LM step's linear solve.

``lm_step_delta(problem, cams, pts, obs, lam)`` returns delta = [delta_c; delta_p]
(9 n_cams + 3 n_pts), the solution of (J^T J + D) delta = -J^T f at (cams, pts)
(Section 2.1).  Its backward pass calls ``ba_adjoint``: a second PCG solve with S
on the same multigrid hierarchy plus the per-observation second-derivative
kernel, and returns gradients for obs, cams and pts (lambda is held fixed).

The problem keeps only the state of its last solve, so run the backward pass
before using the same Problem for another solve.
"""
from __future__ import annotations

import torch


class _LMStepDelta(torch.autograd.Function):
    @staticmethod
    def forward(ctx, obs, cams, pts, problem, lam):
        dc, dp, _, _ = problem.solve(cams.detach(), pts.detach(), obs.detach(), lam)
        ctx.problem = problem
        return torch.cat([dc.reshape(-1), dp.reshape(-1)])

    @staticmethod
    def backward(ctx, grad_delta):
        prob = ctx.problem
        want = ctx.needs_input_grad
        go, gc, gp = prob.adjoint(grad_delta.contiguous(), want_obs=want[0], want_cams=want[1],
                                  want_pts=want[2])
        return go, gc, gp, None, None


def lm_step_delta(problem, cams, pts, obs, lam: float):
    return _LMStepDelta.apply(obs, cams, pts, problem, lam)
