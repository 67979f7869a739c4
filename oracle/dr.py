"""NRTO-DR (oracle; test infrastructure only).

Sec. II-B (the NRTO ADMM on Problem 3, steps (4a)-(4c)), Sec. III (relaxed Douglas–Rachford
on subproblem (7)) and Supplementary Sec. II (standard conic form, KKT system, cone
projection).

Subproblem (7):  min_{k_v, p̃}  Q̃(k_v) + ρ/2‖p̃ - p - λ/ρ‖²  s.t. ‖Â_j k_v + b̂_j‖ ≤ p̃_j.
Standard form (Supplementary Sec. II-A): χ = [k_v; p̃], P = blkdiag(Q_v, ρI),
q = [0; -ρ(p + λ/ρ)], A_j χ + s_j = b_j with s_j = (t_j, η_j) ∈ K_j, t_j = p̃_j,
η_j = Â_j k_v + b̂_j.

DR step 1 (affine prox, Supplementary Sec. II-B) with R_χ = r_χ I and R_s = σ I: the KKT
system is solved through its reduced normal equations (eliminating the multiplier y gives
s = b - Aχ, and (P + R_χ + σAᵀA)χ = R_χ χ̃ - q + σAᵀ(b - s̃)); since AᵀA is
blkdiag(Σ_j Â_jᵀÂ_j, I) the k_v and p̃ parts decouple.  Steps 2-3: reflection, cone
projection of s_ref, relaxation with α.  Termination on r_dr = ‖s̃^l - s̃^{l-1}‖₂.

Subproblem 2 (step (4b), defined in prior work): the exact minimizer of
Q_û(δû) + λᵀ(p - p̃) + ρ/2‖p - p̃‖² s.t. g_j + b_jᵀδû + p_j ≤ 0, ‖F_u δû‖ ≤ r.  With
v = p̃ - λ/ρ, p_j = min(v_j, -g_j - b_jᵀδû), which leaves a strongly convex squared-hinge
objective in δû; it is minimized by semismooth Newton (active-set Newton steps with an
Armijo backtracking safeguard) and the trust region is enforced by a multiplier μ ≥ 0, the
root of ‖F̃ δû(μ)‖² = r² found by bracketing (growth by 4) and Illinois regula falsi.
Dual update (4c) uses the current iterates: λ ← λ + ρ(p - p̃).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import problem as P
from . import soc


@dataclass
class DROptions:
    rho: float = 40.0          # NRTO ADMM penalty
    alpha: float = 0.9         # DR relaxation, α ∈ (0, 1)
    r_chi: float = 1.0         # R_χ = r_χ I
    sigma: float = 1.0         # R_s = σ I
    eps_dr: float = 1e-4       # absolute ‖Δs̃‖ tolerance
    max_dr: int = 500
    r_trust: float = 2.0
    eps_p: float = 1e-4
    eps_d: float = 1e-4
    max_admm: int = 40


@dataclass
class DRState:
    """DR iterate ξ̃ = [χ̃; s̃] with χ̃ = (k̃, p̃̃), s̃_j = (t̃_j, η̃_j)."""
    Kt: np.ndarray
    ptt: np.ndarray
    tt: np.ndarray
    etat: np.ndarray


def zero_dr_state(lin):
    n_g, T, nu = lin.bvec.shape
    nx = lin.Psi.shape[1]
    return DRState(Kt=np.zeros((T, nu, nx)), ptt=np.zeros(n_g), tt=np.zeros(n_g),
                   etat=np.zeros((n_g, T + 1, nx)))


def dr_solve(inst, lin, p, lam, opts: DROptions, state: DRState | None = None, n_iter=None,
             check=True):
    """Relaxed DR on subproblem (7). Returns (K, p̃, state, iterations, r_dr)."""
    rho, a, rc, sg = opts.rho, opts.alpha, opts.r_chi, opts.sigma
    st = zero_dr_state(lin) if state is None else state
    H = P.gain_hessian_blocks(lin, inst, coef=sg, shift=rc)
    L = opts.max_dr if n_iter is None else n_iter
    K = st.Kt.copy()
    pt = st.ptt.copy()
    r_dr = np.inf
    it = 0
    for it in range(1, L + 1):
        # Step 1: χ = Prox_J(ξ̃), s = b - Aχ.
        K = P.gain_solve(H, rc * st.Kt + sg * P.Ahat_T_apply(lin, st.etat - lin.bhat))
        pt = (rc * st.ptt + rho * p + lam + sg * st.tt) / (rho + rc + sg)
        t_s = pt
        eta_s = P.Ahat_apply(lin, K) + lin.bhat
        # Step 2: reflection.
        t_ref = 2.0 * t_s - st.tt
        eta_ref = 2.0 * eta_s - st.etat
        # Step 3: Prox of the cone indicator on s_ref (identity on χ_ref), relaxation.
        t_pi, eta_pi = soc.project_rows(t_ref, eta_ref)
        tt_new = st.tt + a * (t_pi - t_s)
        etat_new = st.etat + a * (eta_pi - eta_s)
        r_dr = float(np.sqrt(np.sum((tt_new - st.tt) ** 2) + np.sum((etat_new - st.etat) ** 2)))
        st = DRState(Kt=st.Kt + a * (K - st.Kt), ptt=st.ptt + a * (pt - st.ptt), tt=tt_new, etat=etat_new)
        if check and r_dr <= opts.eps_dr:
            break
    return K, pt, st, it, r_dr


def sub2_objective(inst, lin, rho, v, du, Hc, c):
    """½δûᵀHcδû + cᵀδû + ρ/2 Σ_j max(0, v_j + g_j + b_jᵀδû)² (constant dropped)."""
    z = v + lin.g0 + P.ell(lin, du)
    x = du.reshape(-1)
    return 0.5 * x @ Hc @ x + c @ x + 0.5 * rho * np.sum(np.maximum(z, 0.0) ** 2)


def _ssn(inst, lin, rho, v, Hc, c, Bm, x0, max_newton=100):
    """Semismooth Newton for min ½xᵀHc x + cᵀx + ρ/2 Σ max(0, v+g+Bx)²."""
    x = x0.copy()
    base = v + lin.g0

    def obj(y):
        z = base + Bm @ y
        return 0.5 * y @ Hc @ y + c @ y + 0.5 * rho * np.sum(np.maximum(z, 0.0) ** 2)

    for _ in range(max_newton):
        z = base + Bm @ x
        act = z > 0
        grad = Hc @ x + c + rho * Bm[act].T @ z[act]
        Hn = Hc + rho * Bm[act].T @ Bm[act]
        dx = -np.linalg.solve(Hn, grad)
        if np.linalg.norm(grad) <= 1e-13 * (1.0 + np.linalg.norm(c)):
            break
        f0 = obj(x)
        step = 1.0
        while obj(x + step * dx) > f0 + 1e-4 * step * (grad @ dx) and step > 1e-12:
            step *= 0.5
        x_new = x + step * dx
        z_new = base + Bm @ x_new
        x = x_new
        if step == 1.0 and np.array_equal(z_new > 0, act):
            break
    return x


def sub2_solve(inst, lin, rho, pt, lam, r_trust):
    """Exact subproblem 2. Returns (δû, δx, p, μ)."""
    T, nu, nx = inst.T, inst.nu, inst.nx
    Ft = lin.Fu[nx:, :]
    Rbar = np.diag(np.tile(inst.Ru, T))
    Qbar = np.diag(np.tile(inst.Qx, T))
    Bm = lin.bvec.reshape(lin.bvec.shape[0], T * nu)
    H0 = 2.0 * Rbar + 2.0 * Ft.T @ Qbar @ Ft
    xdev = (lin.x_hat[1:] - inst.x_goal[None, :]).reshape(-1)
    udev = (lin.u_hat - inst.u_ref[None, :]).reshape(-1)
    c = 2.0 * Rbar @ udev + 2.0 * Ft.T @ Qbar @ xdev
    v = pt - lam / rho
    FtF = Ft.T @ Ft

    def solve_mu(mu, x0):
        return _ssn(inst, lin, rho, v, H0 + mu * FtF, c, Bm, x0)

    def phi(y):
        """‖F̃ δû‖² - r²: decreasing in μ; the multiplier μ > 0 is its root."""
        return float(np.sum((Ft @ y) ** 2)) - r_trust * r_trust

    x = solve_mu(0.0, np.zeros(T * nu))
    mu = 0.0
    if phi(x) > 0.0:
        # bracket [lo, hi] with phi(lo) > 0 >= phi(hi), growing hi by 4
        lo, hi = 0.0, 1.0
        fa = phi(x)
        xh = solve_mu(hi, x)
        fb = phi(xh)
        while fb > 0.0:
            lo, fa = hi, fb
            hi *= 4.0
            xh = solve_mu(hi, xh)
            fb = phi(xh)
        # Illinois regula falsi on phi (a bracketing secant: the endpoint kept twice in a row has
        # its phi halved), each point solved from the feasible end's solution; the feasible end is
        # returned once the bracket is 1e-14 relative
        side = 0
        for _ in range(200):
            mc = hi - fb * (hi - lo) / (fb - fa)
            if not (lo < mc < hi):
                mc = 0.5 * (lo + hi)
            xc = solve_mu(mc, xh)
            fc = phi(xc)
            if fc > 0.0:
                lo, fa = mc, fc
                if side == -1:
                    fb *= 0.5
                side = -1
            else:
                hi, fb, xh = mc, fc, xc
                if side == 1:
                    fa *= 0.5
                side = 1
            if hi - lo <= 1e-14 * hi or fc == 0.0:
                break
        mu, x = hi, xh
    du = x.reshape(T, nu)
    dx = P.delta_x(lin, du)
    p = np.minimum(v, -lin.g0 - P.ell(lin, du))
    return du, dx, p, mu


@dataclass
class NRTODRResult:
    K: np.ndarray
    du: np.ndarray
    dx: np.ndarray
    p: np.ndarray
    pt: np.ndarray
    lam: np.ndarray
    admm_iters: int
    dr_iters: list = field(default_factory=list)
    r_p: float = np.inf
    r_d: float = np.inf
    converged: bool = False
    dr_state: DRState = None


def solve(inst, lin, opts: DROptions, n_admm=None, n_dr=None, check=True) -> NRTODRResult:
    """NRTO ADMM (4a)-(4c) with subproblem 1 by DR (warm-started across ADMM iterations)
    and subproblem 2 exact.  r_p = ‖p - p̃‖, r_d = ρ‖p^l - p^{l-1}‖."""
    n_g, T, nu = lin.bvec.shape
    nx = lin.Psi.shape[1]
    p = np.zeros(n_g)
    lam = np.zeros(n_g)
    du = np.zeros((T, nu))
    dx = np.zeros((T + 1, nx))
    st = zero_dr_state(lin)
    res = NRTODRResult(K=np.zeros((T, nu, nx)), du=du, dx=dx, p=p, pt=np.zeros(n_g), lam=lam,
                       admm_iters=0)
    L = opts.max_admm if n_admm is None else n_admm
    for it in range(1, L + 1):
        K, pt, st, n_it, r_dr = dr_solve(inst, lin, p, lam, opts, st, n_iter=n_dr, check=check)
        du, dx, p_new, mu = sub2_solve(inst, lin, opts.rho, pt, lam, opts.r_trust)
        lam = lam + opts.rho * (p_new - pt)
        r_p = float(np.linalg.norm(p_new - pt))
        r_d = float(opts.rho * np.linalg.norm(p_new - p))
        p = p_new
        res = NRTODRResult(K=K, du=du, dx=dx, p=p, pt=pt, lam=lam, admm_iters=it,
                           dr_iters=res.dr_iters + [n_it], r_p=r_p, r_d=r_d, dr_state=st)
        if check and r_p <= opts.eps_p and r_d <= opts.eps_d:
            res.converged = True
            break
    return res
