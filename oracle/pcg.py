"""Preconditioned conjugate gradients on the reduced camera system.

CG needs only products with S (Section 3.6); the preconditioner is one
V-cycle (Algorithm 1), point-block Jacobi, or none.  Start x_0 = 0.  Two stopping
rules: the relative recursive residual |r_k| <= rtol |b| (the default reading, as
the target metric is quoted at a relative residual), or the Nash-Sofer forcing rule
of Section 2.1: with the quadratic model Q_i = 1/2 x_i^T S x_i - x_i^T b, stop at
the first iteration i with i (Q_i - Q_{i-1}) / Q_i <= tau (the printed Q_{n-1} is
read as Q_{i-1}; Q_0 = 0 at x_0 = 0).  The number of iterations is the number of
products with S.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this module.
"""
from __future__ import annotations

import numpy as np


def quadratic_model(matvec, b, x):
    """Q(x) = 1/2 x^T S x - x^T b, from its definition (one product with S)."""
    return 0.5 * float(x @ matvec(x)) - float(x @ b)


def pcg(matvec, b, precond=None, rtol=1e-8, max_iters=1000, stop="relres", tau=0.1):
    """Returns (x, iterations, |r|/|b| of the recursive residual, history).

    stop = "relres": |r_k| <= rtol |b|;  stop = "nash_sofer": i (Q_i - Q_{i-1}) / Q_i <= tau.
    """
    if stop not in ("relres", "nash_sofer"):
        raise ValueError(stop)
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0, []
    r = b.copy()
    z = precond(r) if precond is not None else r.copy()
    p = z.copy()
    rz = r @ z
    hist = []
    it = 0
    rel = 1.0
    q_prev = 0.0
    while it < max_iters:
        q = matvec(p)
        pq = p @ q
        if not pq > 0:
            raise FloatingPointError("PCG breakdown: p.Sp <= 0")
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        it += 1
        rel = np.linalg.norm(r) / nb
        hist.append(rel)
        if stop == "relres":
            if rel <= rtol:
                break
        else:
            q_i = quadratic_model(matvec, b, x)
            if q_i < 0.0 and it * (q_i - q_prev) / q_i <= tau:
                break
            q_prev = q_i
        z = precond(r) if precond is not None else r.copy()
        rz_new = r @ z
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    return x, it, rel, hist
