"""NRTO-FullADMM inner loop (oracle; test infrastructure only).

Sec. IV ("NRTO-FullADMM Framework"), Algorithm 1 and Supplementary Sec. III.

Problem (12): min Q_û(δû) + Q̃(k_v)  s.t.  g^{lin,1}(δû, p) ≤ 0,  ‖F_u δû‖ ≤ r,
‖ν_j‖ ≤ p̃_j,  p = p̃,  Â_j k_v + b̂_j = ν_j,
solved by scaled ADMM with block 1 = (ν, p̃) and block 2 = (δû, p, k_v).

Reading used for the Block-2 (δû, p) update (the paper solves it with Jacobi-PCG, which
cannot carry inequality constraints): the two inequality sets of (12a) are moved into
block 1 with slack variables,
    g_j(x̂) + b_jᵀ δû + p_j + w_j = 0,  w ≥ 0          (scaled dual λ_w)
    F_u δû = e,  ‖e‖ ≤ r                             (scaled dual λ_e)
so block 1 also projects w onto the orthant and e onto the ball, and block 2 becomes an
unconstrained quadratic in (δû, p) whose Hessian is fixed per outer step.  The fixed
point is the same Problem (12) optimum.  The k_v update uses the direct form
k_v = M ρ Σ_j Â_jᵀ(ν_j - b̂_j - λ_ν,j), M = (Q_v + ρ Σ_j Â_jᵀÂ_j)^{-1}, which equals the
paper's q + 𝓜 k_v^{prev} + 𝓜̄ ν under the dual invariant it assumes (zero initialization).

The cost Q_û(δû) = Σ_k (û_k+δû_k-u_ref)ᵀ R_u (·) is extended with the state-tracking term
Σ_{t=1}^T (x̂_t+δx_t-x_goal)ᵀ Q_x (·), δx = F_u δû.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import math

import numpy as np

from . import dr
from . import problem as P
from . import soc


@dataclass
class FullADMMOptions:
    rho: float = 10.0
    r_trust: float = 2.0
    eps_p: float = 1e-4
    eps_d: float = 1e-4
    max_iter: int = 500
    check: bool = True          # stop at the first iteration meeting both tolerances
    # Residual balancing (standard ADMM penalty adaptation; the paper keeps ρ fixed): at the start
    # of iteration l with (l-1) % adapt_every == 0 and l > adapt_every, look at the residuals of
    # iteration l-2; ρ ← min(τρ, ρ_max) if r_p > μ r_d, ρ ← max(ρ/τ, ρ_min) if r_d > μ r_p, and the
    # scaled duals are multiplied by ρ_old/ρ_new.  adapt_every = 0 disables it.
    adapt_every: int = 0
    adapt_mu: float = 10.0
    adapt_tau: float = 2.0
    rho_min: float = 1e-3
    rho_max: float = 1e3
    # Stall stop: at iterations l that are multiples of stall_every (l >= 2·stall_every), stop when
    # r_p^l > ε_p and r_p^l > stall_ratio · r_p^{l-stall_every} (and the tolerances are not met): a
    # primal residual that is above its tolerance and no longer falls marks an infeasible
    # linearization.  0 disables it.
    stall_every: int = 0
    stall_ratio: float = 0.9
    # Budget stop (a scheduling rule of the library; the paper runs a fixed budget): at the same
    # checkpoints, when r_p^l > ε_p fell by at least stall_ratio, the geometric rate
    # q = r_p^l / r_p^{l-stall_every} needs n = stall_every · log(ε_p / r_p^l) / log q more
    # iterations to reach ε_p; stop (as stalled) when l + stall_budget · n exceeds the iteration cap.
    # 0 disables it.
    stall_budget: float = 0.0
    # k_v update by matrix-free Jacobi-preconditioned CG (problem.gain_solve_pcg) from the previous
    # gains, with this iteration cap and relative tolerance; 0 iterations: the exact per-step solve.
    kv_pcg_iters: int = 0
    kv_pcg_tol: float = 0.05


@dataclass
class FullADMMState:
    K: np.ndarray
    du: np.ndarray
    dx: np.ndarray
    p: np.ndarray
    pt: np.ndarray
    lam_p: np.ndarray
    lam_nu: np.ndarray
    w: np.ndarray
    lam_w: np.ndarray
    e: np.ndarray
    lam_e: np.ndarray
    nu: np.ndarray = None
    iters: int = 0
    r_p: float = np.inf
    r_d: float = np.inf
    r_p_paper: float = np.inf
    r_d_paper: float = np.inf
    converged: bool = False
    stalled: bool = False
    rho: float = np.nan
    history: list = field(default_factory=list)
    pcg_iters: int = 0            # PCG iterations summed over the solve (kv_pcg_iters > 0)


def zero_state(lin) -> FullADMMState:
    """Algorithm 1 initialization: λ_p, λ_ν, k_v, p ← 0 (and δû, w, λ_w, e, λ_e ← 0)."""
    n_g, T, nu = lin.bvec.shape
    nx = lin.Psi.shape[1]
    return FullADMMState(
        K=np.zeros((T, nu, nx)), du=np.zeros((T, nu)), dx=np.zeros((T + 1, nx)),
        p=np.zeros(n_g), pt=np.zeros(n_g), lam_p=np.zeros(n_g),
        lam_nu=np.zeros((n_g, T + 1, nx)), w=np.zeros(n_g), lam_w=np.zeros(n_g),
        e=np.zeros((T, nx)), lam_e=np.zeros((T, nx)))


def warm_state(lin, K0, pt0, lam_p0) -> FullADMMState:
    """Warm start from a predicted (K, p̃, λ_p): k_v^0 = K0, p^0 = p̃0, λ_p^0 = λ_p0, λ_ν = 0."""
    s = zero_state(lin)
    s.K = np.array(K0, dtype=np.float64)
    s.p = np.array(pt0, dtype=np.float64)
    s.pt = np.array(pt0, dtype=np.float64)
    s.lam_p = np.array(lam_p0, dtype=np.float64)
    return s


def warm_state_lifted(lin, K0, pt0, lam_p0, theta0, du0, lam_w0, lam_e0) -> FullADMMState:
    """Warm start of the lifted iteration (reading R8) from a predicted
    (K, p̃, λ_p, θ, δû, λ_w, λ_e): warm_state plus
      λ_ν,j^0 = θ_j (Â_j k^0 + b̂_j)   (at a fixed point ν_j = Â_j k + b̂_j = s_j(ν_j/s_j) with
                                       ν_j = Π(Â_j k + b̂_j + λ_ν,j), so λ_ν,j = (1/s_j - 1)(Â_j k + b̂_j):
                                       one scalar per row θ_j = 1/s_j - 1 ≥ 0 fixes the S-length dual),
      δû^0 = du0 with δx^0 = F_u δû^0 (its linearized trajectory),
      λ_w^0 = lam_w0 (orthant coupling) and λ_e^0 = lam_e0 (trust-region coupling, rows t = 1..T).
    At a solution's values and the penalty its scaled duals belong to, the first iteration is at the
    fixed point."""
    s = warm_state(lin, K0, pt0, lam_p0)
    s.lam_nu = np.asarray(theta0, dtype=np.float64)[:, None, None] * (P.Ahat_apply(lin, s.K) + lin.bhat)
    s.du = np.array(du0, dtype=np.float64)
    s.dx = P.delta_x(lin, s.du)
    s.lam_w = np.array(lam_w0, dtype=np.float64)
    s.lam_e = np.array(lam_e0, dtype=np.float64)
    return s


def block2_matrices(inst, lin, rho):
    """Hessian of the Block-2 (δû) quadratic after eliminating p (fixed per outer step):
    2R̄ + F̃ᵀ(2Q̄ + ρI)F̃ + (ρ/2) Σ_j b_j b_jᵀ, F̃ = rows t = 1..T of F_u."""
    T, nu, nx = inst.T, inst.nu, inst.nx
    Ft = lin.Fu[nx:, :]
    Rbar = np.diag(np.tile(inst.Ru, T))
    Qbar = np.diag(np.tile(inst.Qx, T))
    Bm = lin.bvec.reshape(lin.bvec.shape[0], T * nu)
    H = 2.0 * Rbar + Ft.T @ (2.0 * Qbar + rho * np.eye(T * nx)) @ Ft + 0.5 * rho * Bm.T @ Bm
    return H, Ft, Rbar, Qbar, Bm


def block2_solve(inst, lin, rho, mats, pt, lam_p, w, lam_w, e, lam_e):
    """Block-2 (δû, p) update: argmin_{δû,p} Q_û(δû) + ρ/2‖p - p̃ + λ_p‖²
    + ρ/2‖g + b_jᵀδû + p + w + λ_w‖² + ρ/2‖F̃δû - e + λ_e‖².
    p_j is eliminated in closed form, p_j = ½[(p̃_j - λ_p,j) - (g_j + b_jᵀδû + w_j + λ_w,j)],
    which leaves (ρ/4)(b_jᵀδû + d_j)² with d_j = p̃_j - λ_p,j + g_j + w_j + λ_w,j."""
    H, Ft, Rbar, Qbar, Bm = mats
    T, nu, nx = inst.T, inst.nu, inst.nx
    d = pt - lam_p + lin.g0 + w + lam_w
    xdev = (lin.x_hat[1:] - inst.x_goal[None, :]).reshape(-1)
    udev = (lin.u_hat - inst.u_ref[None, :]).reshape(-1)
    grad = 2.0 * Rbar @ udev + Ft.T @ (2.0 * Qbar @ xdev - rho * (e - lam_e).reshape(-1)) + 0.5 * rho * Bm.T @ d
    du = -np.linalg.solve(H, grad).reshape(T, nu)
    dx = P.delta_x(lin, du)
    l = P.ell(lin, du)
    p = 0.5 * ((pt - lam_p) - (lin.g0 + l + w + lam_w))
    return du, dx, p


def iterate(inst, lin, opts: FullADMMOptions, state: FullADMMState | None = None,
            n_iter: int | None = None, rho0: float | None = None) -> FullADMMState:
    """Run Algorithm 1 for up to n_iter (default opts.max_iter) iterations, starting from `state`
    (default: the zero initialization) with penalty rho0 (default opts.rho)."""
    rho = opts.rho if rho0 is None else rho0
    s = zero_state(lin) if state is None else state
    H = P.gain_hessian_blocks(lin, inst, coef=rho)
    mats = block2_matrices(inst, lin, rho)
    L = opts.max_iter if n_iter is None else n_iter
    Y_prev = P.Ahat_apply(lin, s.K) + lin.bhat
    rp_mark = np.inf
    for it in range(1, L + 1):
        A = opts.adapt_every
        if A > 0 and it >= 3 and it > A and (it - 1) % A == 0:
            rp2, rd2 = s.history[it - 3]
            rho_new = rho
            if rp2 > opts.adapt_mu * rd2:
                rho_new = min(rho * opts.adapt_tau, opts.rho_max)
            elif rd2 > opts.adapt_mu * rp2:
                rho_new = max(rho / opts.adapt_tau, opts.rho_min)
            if rho_new != rho:
                f = rho / rho_new
                s.lam_p, s.lam_nu, s.lam_w, s.lam_e = s.lam_p * f, s.lam_nu * f, s.lam_w * f, s.lam_e * f
                rho = rho_new
                H = P.gain_hessian_blocks(lin, inst, coef=rho)
                mats = block2_matrices(inst, lin, rho)
        # Block 1 (13): per-row SOC projection of (Â_j k + b̂_j + λ_ν,j, p_j + λ_p,j);
        # lifted slacks: orthant for w, ball for e.
        Y = Y_prev
        pt_new, nu = soc.project_rows(s.p + s.lam_p, Y + s.lam_nu)
        l_prev = P.ell(lin, s.du)
        w = np.maximum(0.0, -(lin.g0 + l_prev + s.p + s.lam_w))
        e = soc.project_ball((s.dx[1:] + s.lam_e).reshape(-1), opts.r_trust).reshape(s.e.shape)
        # Block 2b (14b), direct form: k = M ρ Σ_j Â_jᵀ(ν_j - b̂_j - λ_ν,j), exactly or by PCG.
        rhs = rho * P.Ahat_T_apply(lin, nu - lin.bhat - s.lam_nu)
        n_cg = 0
        if opts.kv_pcg_iters > 0:
            K_new, n_cg = P.gain_solve_pcg(lin, inst, rho, rhs, s.K, opts.kv_pcg_tol, opts.kv_pcg_iters)
        else:
            K_new = P.gain_solve(H, rhs)
        # Block 2a (14a): (δû, p).
        du, dx, p = block2_solve(inst, lin, rho, mats, pt_new, s.lam_p, w, s.lam_w, e, s.lam_e)
        l_new = P.ell(lin, du)
        Y_new = P.Ahat_apply(lin, K_new) + lin.bhat
        # Dual updates (15) plus the lifted couplings.
        lam_p = s.lam_p + (p - pt_new)
        lam_nu = s.lam_nu + (Y_new - nu)
        lam_w = s.lam_w + (lin.g0 + l_new + p + w)
        lam_e = s.lam_e + (dx[1:] - e)
        # Residuals: every coupling (primal) and the block-2 change mapped through the
        # couplings (dual); the paper's r_p = ‖p - p̃‖, r_d = ρ‖Δp̃‖ are kept alongside.
        r_p = np.sqrt(np.sum((p - pt_new) ** 2) + np.sum((Y_new - nu) ** 2)
                      + np.sum((lin.g0 + l_new + p + w) ** 2) + np.sum((dx[1:] - e) ** 2))
        dp = p - s.p
        r_d = rho * np.sqrt(np.sum(dp ** 2) + np.sum((Y_new - Y) ** 2)
                            + np.sum((l_new - l_prev + dp) ** 2) + np.sum((dx - s.dx) ** 2))
        r_p_paper = float(np.linalg.norm(p - pt_new))
        r_d_paper = float(rho * np.linalg.norm(pt_new - s.pt))
        s = FullADMMState(K=K_new, du=du, dx=dx, p=p, pt=pt_new, lam_p=lam_p, lam_nu=lam_nu,
                          w=w, lam_w=lam_w, e=e, lam_e=lam_e, nu=nu, iters=s.iters + 1,
                          r_p=float(r_p), r_d=float(r_d), r_p_paper=r_p_paper, r_d_paper=r_d_paper,
                          rho=rho, history=s.history + [(float(r_p), float(r_d))],
                          pcg_iters=s.pcg_iters + n_cg)
        Y_prev = Y_new
        if opts.check and r_p <= opts.eps_p and r_d <= opts.eps_d:
            s.converged = True
            break
        S_ = opts.stall_every
        if opts.check and S_ > 0 and it % S_ == 0:
            if it >= 2 * S_ and r_p > opts.eps_p and r_p > opts.stall_ratio * rp_mark:
                s.stalled = True
                break
            if it >= 2 * S_ and r_p > opts.eps_p and opts.stall_budget > 0:
                need = S_ * math.log(opts.eps_p / r_p) / math.log(r_p / rp_mark)
                if it + opts.stall_budget * need > L:
                    s.stalled = True
                    break
            rp_mark = r_p
    return s


def solve_warm_with_fallback(inst, lin, opts: FullADMMOptions, K0, pt0, lam_p0):
    """Learned-warm-start solve with its fallback: iterate from warm_state(K0, p̃0, λ_p0); if that
    run stops on the stall rule, run the cold solve (zero_state, Algorithm 1 initialization) with
    the full iteration budget, so the outcome is never worse than without the warm start.
    Returns (state, fell_back); state.iters counts both runs."""
    s = iterate(inst, lin, opts, warm_state(lin, K0, pt0, lam_p0))
    if not s.stalled:
        return s, False
    c = iterate(inst, lin, opts, zero_state(lin))
    c.iters = s.iters + c.iters
    return c, True


def carry_state(lin, prev: FullADMMState, opts: FullADMMOptions, shifted: bool):
    """Start of the next inner solve from the state the previous one ended in (the library's
    inner-state carry across successive-linearization steps; the paper re-initializes each inner
    solve).  Carried: k_v (K), p, p̃ and the scaled duals λ_p, λ_ν, λ_w, λ_e, with the penalty
    they are scaled for.  δû, δx and e are measured from the nominal: `shifted` means the nominal
    moved to û + δû (an accepted outer step), so in the new coordinates the previous solution is
    δû = 0 and they restart at zero; otherwise (same nominal, e.g. a rejected step that only
    shrinks the trust radius) they are carried too.  The solver state at the end of a solve is
    the one at the start of its next iteration, so a residual-balancing update scheduled there
    (same rule as in `iterate`, with the residuals of the iteration before last) is applied first.
    Any state is a valid ADMM start, so the fixed point is the same as the cold solve's.
    Returns (state, rho)."""
    rho = prev.rho
    f = 1.0
    it = prev.iters + 1
    A = opts.adapt_every
    # A solve that ran to its iteration cap has no next iteration; one that stopped at its
    # tolerance or on the stall rule stopped before the iteration cap.
    if (A > 0 and (prev.converged or prev.stalled) and it >= 3 and it > A and (it - 1) % A == 0):
        rp2, rd2 = prev.history[it - 3]
        rho_new = rho
        if rp2 > opts.adapt_mu * rd2:
            rho_new = min(rho * opts.adapt_tau, opts.rho_max)
        elif rd2 > opts.adapt_mu * rp2:
            rho_new = max(rho / opts.adapt_tau, opts.rho_min)
        f = rho / rho_new
        rho = rho_new
    s = zero_state(lin)
    s.K = prev.K.copy()
    s.p = prev.p.copy()
    s.pt = prev.pt.copy()
    s.lam_p = prev.lam_p * f
    s.lam_nu = prev.lam_nu * f
    s.lam_w = prev.lam_w * f
    s.lam_e = prev.lam_e * f
    if not shifted:
        s.du = prev.du.copy()
        s.dx = prev.dx.copy()
        s.e = prev.e.copy()
    return s, rho


def iterate_as_written(inst, lin, opts: FullADMMOptions, state: FullADMMState | None = None,
                       n_iter: int | None = None) -> FullADMMState:
    """Algorithm 1 with block 2a as the paper states it (Sec. IV): (δû, p) is the exact minimizer of
    Q_û(δû) + ρ/2‖p - p̃ + λ_p‖² subject to the linearized robust constraints
    g_j(x̂) + b_jᵀδû + p_j ≤ 0 and the trust region ‖F_u δû‖ ≤ r, with no slack variables.  That QP
    is NRTO-DR's subproblem 2 with v = p̃ - λ_p (scaled dual), solved exactly by dr.sub2_solve.
    Block 1 and the k_v update are those of `iterate`; duals λ_p, λ_ν only.  Residuals: every
    coupling, r_p = ‖(p - p̃, Â_jk + b̂_j - ν_j)‖, and the block-2 change mapped through them,
    r_d = ρ‖(Δp, Δ(Â_jk + b̂_j))‖; the paper's r_p, r_d are kept alongside.  The lifted form of
    `iterate` has the same Problem (12) fixed point."""
    rho = opts.rho
    s = zero_state(lin) if state is None else state
    H = P.gain_hessian_blocks(lin, inst, coef=rho)
    L = opts.max_iter if n_iter is None else n_iter
    Y_prev = P.Ahat_apply(lin, s.K) + lin.bhat
    for it in range(1, L + 1):
        Y = Y_prev
        # Block 1: per-row SOC projection of (Â_j k + b̂_j + λ_ν,j, p_j + λ_p,j).
        pt_new, nu = soc.project_rows(s.p + s.lam_p, Y + s.lam_nu)
        # Block 2b, direct form.
        K_new = P.gain_solve(H, rho * P.Ahat_T_apply(lin, nu - lin.bhat - s.lam_nu))
        # Block 2a: the constrained (δû, p) QP (λ_p is scaled: the unscaled dual is ρ λ_p).
        du, dx, p, _ = dr.sub2_solve(inst, lin, rho, pt_new, rho * s.lam_p, opts.r_trust)
        Y_new = P.Ahat_apply(lin, K_new) + lin.bhat
        lam_p = s.lam_p + (p - pt_new)
        lam_nu = s.lam_nu + (Y_new - nu)
        r_p = np.sqrt(np.sum((p - pt_new) ** 2) + np.sum((Y_new - nu) ** 2))
        r_d = rho * np.sqrt(np.sum((p - s.p) ** 2) + np.sum((Y_new - Y) ** 2))
        r_p_paper = float(np.linalg.norm(p - pt_new))
        r_d_paper = float(rho * np.linalg.norm(pt_new - s.pt))
        s = FullADMMState(K=K_new, du=du, dx=dx, p=p, pt=pt_new, lam_p=lam_p, lam_nu=lam_nu,
                          w=s.w, lam_w=s.lam_w, e=s.e, lam_e=s.lam_e, nu=nu, iters=s.iters + 1,
                          r_p=float(r_p), r_d=float(r_d), r_p_paper=r_p_paper, r_d_paper=r_d_paper,
                          rho=rho, history=s.history + [(float(r_p), float(r_d))])
        Y_prev = Y_new
        if opts.check and r_p <= opts.eps_p and r_d <= opts.eps_d:
            s.converged = True
            break
    return s
