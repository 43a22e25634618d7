"""Huber loss of Section 5 (robust error metrics) for the LM step.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this module.

The paper's loss acts on s = |f_o|^2, the squared norm of an observation's
residual:  loss(s) = s for s <= 1 and 2 sqrt(s) - 1 beyond.  With a scale a
(the paper's a = 1) this reads loss(s) = s for s <= a^2 and 2 a sqrt(s) - a^2
beyond, and the objective is 1/2 sum_o loss(|f_o|^2).

Its use inside LM is delegated by the paper to Ceres.  The reading taken here is
Ceres' residual corrector (Triggs et al.): each residual and its Jacobian rows
are rescaled so that the Gauss-Newton model matches the robust objective to
first order, and since loss''(s) <= 0 everywhere for this loss the corrector
reduces to the scaling by w_o = sqrt(loss'(s_o)):

    f~_o = w_o f_o,   J~_o = w_o J_o,   loss'(s) = 1 (s <= a^2), a / sqrt(s) (s > a^2).

The gain ratio compares the change of the robust objective with the reduction of
the model built from f~ and J~.
"""
from __future__ import annotations

import numpy as np


def huber(s, a=1.0):
    """loss(s) and loss'(s) elementwise."""
    s = np.asarray(s, dtype=float)
    a2 = a * a
    inner = s <= a2
    root = np.sqrt(np.maximum(s, a2))
    rho = np.where(inner, s, 2.0 * a * root - a2)
    rho1 = np.where(inner, 1.0, a / root)
    return rho, rho1


def weights(f, a=1.0):
    """w_o = sqrt(loss'(|f_o|^2)) for residuals f [n_obs, 2]."""
    _, rho1 = huber(np.sum(f * f, axis=1), a)
    return np.sqrt(rho1)


def cost(f, a=1.0) -> float:
    """1/2 sum_o loss(|f_o|^2)."""
    rho, _ = huber(np.sum(f * f, axis=1), a)
    return 0.5 * float(np.sum(rho))
