"""Second-order-cone projection (oracle; test infrastructure only).

Supplementary Sec. II-C, closed-form projection onto K_soc = {(t, η): ‖η‖₂ ≤ t}
(illustrated by the three cases of Fig. 3): with a = ‖r^η‖,
  a ≤ r^t        →  (r^t, r^η)                 (already in the cone)
  a ≤ -r^t       →  (0, 0)                     (in the polar cone)
  otherwise      →  ((r^t + a)/2, (r^t + a)/(2a) · r^η)
"""
from __future__ import annotations

import numpy as np


def project(rt, reta):
    """Project one cone block. rt scalar, reta 1-D array. Returns (t, eta)."""
    a = float(np.sqrt(np.sum(reta * reta)))
    if a <= rt:
        return float(rt), reta.copy()
    if a <= -rt:
        return 0.0, np.zeros_like(reta)
    c = (rt + a) / 2.0
    return c, (c / a) * reta


def project_rows(rt, reta):
    """Row-wise projection of n rows: rt (n,), reta (n, ...) → (t (n,), eta like reta)."""
    t = np.zeros_like(rt)
    eta = np.zeros_like(reta)
    for j in range(rt.shape[0]):
        t[j], e = project(rt[j], reta[j].reshape(-1))
        eta[j] = e.reshape(reta[j].shape)
    return t, eta


def project_ball(v, r):
    """Euclidean projection onto {‖e‖₂ ≤ r} (trust region of Problem 2)."""
    n = float(np.sqrt(np.sum(v * v)))
    if n <= r:
        return v.copy()
    return (r / n) * v
