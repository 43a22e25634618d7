"""Preconditioned conjugate gradients on the reduced camera system.

CG needs only products with S (Section 3.6); the preconditioner is one
V-cycle (Algorithm 1), point-block Jacobi, or none.  Start x_0 = 0.  The paper
stops with the Nash-Sofer rule of Section 2.1; the reading taken here stops
when the recursive residual satisfies |r_k| <= rtol |b|, and the number of
iterations is the number of products with S.
"""
from __future__ import annotations

import numpy as np


def pcg(matvec, b, precond=None, rtol=1e-8, max_iters=1000):
    """Returns (x, iterations, |r|/|b| of the recursive residual, history)."""
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
        if rel <= rtol:
            break
        z = precond(r) if precond is not None else r.copy()
        rz_new = r @ z
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    return x, it, rel, hist
