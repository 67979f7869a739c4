"""Dense log-barrier interior-point solver for small SOCPs (test tool, not the oracle).

min ½xᵀPx + qᵀx  s.t.  ‖A_i x + b_i‖ ≤ c_iᵀx + d_i (second-order cones),  G x ≤ h.

Barrier method: minimize t·f(x) + Σ_i -log((c_iᵀx+d_i)² - ‖A_ix+b_i‖²) + Σ -log(h - Gx)
by damped Newton steps that keep the iterate strictly inside every cone, then t ← 10 t.
It is an independent method (no splitting, no projections) used to pin the fixed points
of the ADMM and DR iterations on tiny instances.  Needs a strictly feasible start.
"""
from __future__ import annotations

import numpy as np


def _feasible(x, socs, G, h):
    for (A, b, c, d) in socs:
        s = c @ x + d
        u = A @ x + b
        if not (s > 0 and s * s - u @ u > 0):
            return False
    if G is not None and np.any(G @ x >= h):
        return False
    return True


def _barrier(x, socs, G, h):
    val = 0.0
    n = x.shape[0]
    g = np.zeros(n)
    H = np.zeros((n, n))
    for (A, b, c, d) in socs:
        s = c @ x + d
        u = A @ x + b
        D = s * s - u @ u
        v = 2 * s * c - 2 * A.T @ u
        val -= np.log(D)
        g -= v / D
        H -= (2 * np.outer(c, c) - 2 * A.T @ A) / D
        H += np.outer(v, v) / (D * D)
    if G is not None:
        r = h - G @ x
        val -= np.sum(np.log(r))
        g += G.T @ (1.0 / r)
        H += G.T @ (G / (r * r)[:, None])
    return val, g, H


def solve(P, q, socs, G=None, h=None, x0=None, tol=1e-11, t0=1.0, mu=10.0, max_newton=200):
    x = np.array(x0, dtype=np.float64)
    assert _feasible(x, socs, G, h), "start point must be strictly feasible"
    m = len(socs) * 2 + (0 if G is None else G.shape[0])
    t = t0
    while True:
        for _ in range(max_newton):
            bv, bg, bH = _barrier(x, socs, G, h)
            fval = t * (0.5 * x @ P @ x + q @ x) + bv
            grad = t * (P @ x + q) + bg
            Hess = t * P + bH
            dx = -np.linalg.solve(Hess, grad)
            lam2 = -grad @ dx
            if lam2 / 2 <= 1e-14 * max(1.0, abs(fval)):
                break
            step = 1.0
            while not _feasible(x + step * dx, socs, G, h):
                step *= 0.5
            while True:
                xn = x + step * dx
                bv2, _, _ = _barrier(xn, socs, G, h)
                f2 = t * (0.5 * xn @ P @ xn + q @ xn) + bv2
                if f2 <= fval - 0.25 * step * lam2 or step < 1e-14:
                    break
                step *= 0.5
            x = xn
        if m / t < tol:
            return x
        t *= mu
