"""Successive-linearization outer loop (oracle; test infrastructure only).

Fig. 1 / Sec. II-B: linearize Problem 1 around the nominal (x̂, û) to get Problem 2, solve it
with the inner loop, then accept or reject the candidate and adapt the trust radius.  The
acceptance rule and trust-radius schedule are defined only in prior work; the reading used
here is: merit φ(ū, K) = J(ū, K) + w_p Σ_j max(0, g_j(x̄) + b_jᵀ·0 + ‖Â_j k_v + b̂_j‖) evaluated
with the linearization at the candidate itself; accept iff φ decreases; on accept
r ← min(1.5 r, r_0), on reject r ← max(0.8 r, r_min).  J is the Problem 1 cost
Σ_k (ū_k - u_ref)ᵀR_u(·) + ‖R_K K_k‖_F² plus the state-tracking term Σ_{t≥1}(x̄_t - x_goal)ᵀQ_x(·).
Parity status: pinned on a convex case (linear dynamics and linear constraints, where every
linearization is exact and the loop must end at the optimum of Problem 1, which an independent
barrier solve gives); the schedule's constants are not given in the paper and stay a reading.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import dr
from . import fulladmm
from . import problem as P


@dataclass
class OuterOptions:
    n_outer: int = 10
    r0: float = 2.0
    r_min: float = 1e-3
    w_p: float = 10.0
    solver: str = "fulladmm"          # or "dr"
    # FullADMM only: start every inner solve after the first from the state the previous inner
    # solve ended in (fulladmm.carry_state); the paper re-initializes each inner solve.
    carry: bool = False
    # FullADMM only: iteration cap of the last outer step's inner solve (0: the same cap as the
    # others), so that the inner solves during the successive linearization can stay inexact (the
    # paper's 40 iterations) while the returned step's subproblem is solved to tolerance.
    max_inner_final: int = 0


def cost(inst, lin, K):
    """Problem 1 objective at the nominal of `lin` with gains K."""
    ud = lin.u_hat - inst.u_ref[None, :]
    xd = lin.x_hat[1:] - inst.x_goal[None, :]
    RK = inst.RK[None, :, None] * K
    return float(np.sum(ud * ud * inst.Ru[None, :]) + np.sum(xd * xd * inst.Qx[None, :]) + np.sum(RK * RK))


def robust_violation(lin, K):
    """Per-row robust constraint of Problem 2 at δû = 0: g_j(x̂) + ‖Â_j k_v + b̂_j‖ (≤ 0 when the
    constraint holds for every disturbance of the ellipsoid, to first order around x̂)."""
    return lin.g0 + np.sqrt(np.sum((P.Ahat_apply(lin, K) + lin.bhat) ** 2, axis=(1, 2)))


def merit(inst, lin, K, w_p):
    viol = robust_violation(lin, K)
    return cost(inst, lin, K) + w_p * float(np.sum(np.maximum(viol, 0.0)))


@dataclass
class OuterResult:
    u_bar: np.ndarray
    K: np.ndarray
    phi: float
    accepted: list = field(default_factory=list)
    inner_iters: list = field(default_factory=list)
    inner_converged: list = field(default_factory=list)
    radii: list = field(default_factory=list)
    max_violation: float = np.inf      # max_j of robust_violation at the accepted iterate
    accepted_inner_converged: bool = False   # the inner solve of the last accepted step converged


def solve(inst, opts: OuterOptions, admm: fulladmm.FullADMMOptions | None = None,
          dropts: dr.DROptions | None = None) -> OuterResult:
    admm = admm or fulladmm.FullADMMOptions()
    dropts = dropts or dr.DROptions()
    u_hat = np.array(inst.u_init, dtype=np.float64)
    K = np.zeros((inst.T, inst.nu, inst.nx))
    lin = P.linearize(inst, u_hat)
    phi = merit(inst, lin, K, opts.w_p)
    r = opts.r0
    res = OuterResult(u_bar=u_hat, K=K, phi=phi)
    res.max_violation = float(np.max(robust_violation(lin, K))) if lin.g0.size else -np.inf
    prev = None
    moved = False          # the nominal changed since the previous inner solve
    for step in range(opts.n_outer):
        res.radii.append(r)
        if opts.solver == "fulladmm":
            a = fulladmm.FullADMMOptions(**{**admm.__dict__, "r_trust": r})
            if opts.max_inner_final > 0 and step == opts.n_outer - 1:
                a.max_iter = opts.max_inner_final
            if opts.carry and prev is not None and np.isfinite(prev.r_p) and np.isfinite(prev.r_d):
                st0, rho0 = fulladmm.carry_state(lin, prev, a, shifted=moved)
                s = fulladmm.iterate(inst, lin, a, st0, rho0=rho0)
            else:
                s = fulladmm.iterate(inst, lin, a)
            prev = s
            du, K_c, n_it, conv = s.du, s.K, s.iters, s.converged
        else:
            o = dr.DROptions(**{**dropts.__dict__, "r_trust": r})
            s = dr.solve(inst, lin, o)
            du, K_c, n_it, conv = s.du, s.K, s.admm_iters, s.converged
        res.inner_iters.append(n_it)
        res.inner_converged.append(conv)
        u_c = u_hat + du
        lin_c = P.linearize(inst, u_c)
        phi_c = merit(inst, lin_c, K_c, opts.w_p)
        if phi_c < phi:
            u_hat, K, lin, phi = u_c, K_c, lin_c, phi_c
            res.max_violation = float(np.max(robust_violation(lin, K))) if lin.g0.size else -np.inf
            res.accepted_inner_converged = bool(conv)
            r = min(1.5 * r, opts.r0)
            res.accepted.append(True)
            moved = True
        else:
            moved = False
            r = max(0.8 * r, opts.r_min)
            res.accepted.append(False)
    res.u_bar, res.K, res.phi = u_hat, K, phi
    return res
