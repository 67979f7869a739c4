"""Pins for the oracle's NRTO-FullADMM loop (Sec. IV, Algorithm 1, Supplementary Sec. III)."""
import numpy as np
import pytest
import torch

from oracle import fulladmm as F, models, problem as P
from paper_2603_02642_b300 import workloads as W

from . import ipsolver

RNG = np.random.default_rng(5)


def tiny_unicycle(T=6, tau=1.0):
    inst = W.unicycle(0, T=T, n_obs=1)
    inst.obs_center = np.array([[0.75, 0.55]])
    inst.obs_radius = np.array([0.3])
    inst.u_init = np.tile([1.0, 0.0], (T, 1))
    inst.tau = tau
    return inst


def problem2_ip(inst, lin, r):
    """Problem 2 (with the tracking term) as a dense SOCP for the barrier solver."""
    T, nu, nx = inst.T, inst.nu, inst.nx
    n1, n2, ng = T * nu, T * nu * nx, lin.g0.shape[0]
    n = n1 + n2 + ng
    H, Ft, Rbar, Qbar, Bm = F.block2_matrices(inst, lin, 0.0)
    Pm = np.zeros((n, n))
    Pm[:n1, :n1] = H
    Pm[n1:n1 + n2, n1:n1 + n2] = 2 * np.kron(np.eye(T * nx), np.diag(inst.RK ** 2))
    q = np.zeros(n)
    xdev = (lin.x_hat[1:] - inst.x_goal).reshape(-1)
    udev = (lin.u_hat - inst.u_ref).reshape(-1)
    q[:n1] = 2 * Rbar @ udev + 2 * Ft.T @ Qbar @ xdev
    socs = []
    for j in range(ng):
        A = np.zeros(((T + 1) * nx, n))
        A[:, n1:n1 + n2] = P.dense_Ahat(lin, j)
        c = np.zeros(n)
        c[n1 + n2 + j] = 1.0
        socs.append((A, lin.bhat[j].reshape(-1), c, 0.0))
    At = np.zeros((Ft.shape[0], n))
    At[:, :n1] = Ft
    socs.append((At, np.zeros(Ft.shape[0]), np.zeros(n), r))
    G = np.zeros((ng, n))
    G[:, :n1] = Bm
    G[:, n1 + n2:] = np.eye(ng)
    h = -lin.g0
    x0 = np.zeros(n)
    x0[n1 + n2:] = np.linalg.norm(lin.bhat.reshape(ng, -1), axis=1) + 1e-3
    x = ipsolver.solve(Pm, q, socs, G, h, x0)
    return x[:n1].reshape(T, nu), P.K_from_kv(x[n1:n1 + n2], T, nu, nx)


def test_fixed_point_matches_interior_point():
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    du_ip, K_ip = problem2_ip(inst, lin, r=0.5)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=0.5, eps_p=1e-9, eps_d=1e-9, max_iter=30000))
    assert s.converged
    assert np.allclose(s.du, du_ip, atol=2e-6)
    assert np.allclose(s.K, K_ip, atol=2e-6)
    # The solution touches constraints (otherwise the pin would be weak).
    act = lin.g0 + P.ell(lin, s.du) + s.p
    assert np.max(act) > -1e-6


def test_block2_stationarity_by_autograd():
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    rho = 7.0
    ng, T = lin.g0.shape[0], inst.T
    pt, lam_p, w, lam_w = RNG.normal(size=ng), RNG.normal(size=ng), np.abs(RNG.normal(size=ng)), RNG.normal(size=ng)
    e, lam_e = RNG.normal(size=(T, inst.nx)), RNG.normal(size=(T, inst.nx))
    mats = F.block2_matrices(inst, lin, rho)
    du, dx, p = F.block2_solve(inst, lin, rho, mats, pt, lam_p, w, lam_w, e, lam_e)
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    du_t = t(du).requires_grad_(True)
    p_t = t(p).requires_grad_(True)
    Fu = t(lin.Fu)
    dxv = (Fu @ du_t.reshape(-1)).reshape(T + 1, inst.nx)
    ubar = t(lin.u_hat) + du_t - t(inst.u_ref)
    xbar = t(lin.x_hat[1:]) + dxv[1:] - t(inst.x_goal)
    ellv = torch.einsum("jku,ku->j", t(lin.bvec), du_t)
    obj = (torch.sum(ubar * ubar * t(inst.Ru)) + torch.sum(xbar * xbar * t(inst.Qx))
           + rho / 2 * torch.sum((p_t - t(pt) + t(lam_p)) ** 2)
           + rho / 2 * torch.sum((t(lin.g0) + ellv + p_t + t(w) + t(lam_w)) ** 2)
           + rho / 2 * torch.sum((dxv[1:] - t(e) + t(lam_e)) ** 2))
    gdu, gp = torch.autograd.grad(obj, [du_t, p_t])
    assert gdu.abs().max().item() < 1e-9 and gp.abs().max().item() < 1e-9


def test_direct_form_equals_paper_closed_form_under_zero_init():
    """k^l = q + 𝓜 k^{l-1} + 𝓜̄ ν^l (Supplementary Sec. III) vs the direct form used by the loop."""
    inst = tiny_unicycle(T=4)
    lin = P.linearize(inst, inst.u_init)
    rho = 10.0
    T, nu, nx = inst.T, inst.nu, inst.nx
    ng = lin.g0.shape[0]
    Ad = [P.dense_Ahat(lin, j) for j in range(ng)]
    Qv = 2 * np.kron(np.eye(T * nx), np.diag(inst.RK ** 2))
    M = np.linalg.inv(Qv + rho * sum(a.T @ a for a in Ad))
    q = -rho * M @ sum(a.T @ lin.bhat[j].reshape(-1) for j, a in enumerate(Ad))
    opts = F.FullADMMOptions(rho=rho, r_trust=0.5, check=False)
    s = F.zero_state(lin)
    for _ in range(8):
        k_prev = P.kv_from_K(s.K)
        s = F.iterate(inst, lin, opts, s, n_iter=1)
        k_cf = q + M @ Qv @ k_prev + sum(rho * M @ a.T @ s.nu[j].reshape(-1) for j, a in enumerate(Ad))
        assert np.allclose(k_cf, P.kv_from_K(s.K), atol=1e-11)
        # The invariant Σ_j ρ Â_jᵀ λ_ν,j + Q_v k = 0 holds at every iterate.
        inv = rho * sum(a.T @ s.lam_nu[j].reshape(-1) for j, a in enumerate(Ad)) + Qv @ P.kv_from_K(s.K)
        assert np.abs(inv).max() < 1e-10


def test_no_constraints_reduces_to_lqr_tracking():
    """n_g = 0, trust radius inactive: K = 0 and δû is the finite-horizon LQ tracking
    solution, computed here by an independent backward Riccati recursion."""
    inst = W.quadcopter(1, T=8, n_obs=0)
    inst.u_lo = np.full(4, -np.inf)
    inst.u_hi = np.full(4, np.inf)
    u = inst.u_init + 0.05 * RNG.normal(size=inst.u_init.shape)
    lin = P.linearize(inst, u)
    assert lin.g0.shape[0] == 0
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=1.0, r_trust=1e6, eps_p=1e-12, eps_d=1e-12, max_iter=2000))
    assert np.abs(s.K).max() == 0.0
    T, nx, nu = inst.T, inst.nx, inst.nu
    Q = 2 * np.diag(inst.Qx)
    R = 2 * np.diag(inst.Ru)
    qv = [Q @ (lin.x_hat[t] - inst.x_goal) for t in range(T + 1)]
    rv = [R @ (lin.u_hat[k] - inst.u_ref) for k in range(T)]
    Pn, pn = Q.copy(), qv[T].copy()
    Ks, ks = [None] * T, [None] * T
    for k in range(T - 1, -1, -1):
        A, B = lin.A[k], lin.B[k]
        Huu = R + B.T @ Pn @ B
        Hux = B.T @ Pn @ A
        hu = rv[k] + B.T @ pn
        Ks[k] = -np.linalg.solve(Huu, Hux)
        ks[k] = -np.linalg.solve(Huu, hu)
        Qk = Q if k > 0 else np.zeros_like(Q)
        qk = qv[k] if k > 0 else np.zeros(nx)
        Pn = Qk + A.T @ Pn @ A + Hux.T @ Ks[k]
        pn = qk + A.T @ pn + Hux.T @ ks[k]
    dx = np.zeros(nx)
    du = np.zeros((T, nu))
    for k in range(T):
        du[k] = Ks[k] @ dx + ks[k]
        dx = lin.A[k] @ dx + lin.B[k] @ du[k]
    assert np.allclose(s.du, du, atol=1e-8)


def test_iterates_are_deterministic_and_warm_start_shapes():
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    o = F.FullADMMOptions(check=False)
    a = F.iterate(inst, lin, o, n_iter=5)
    b = F.iterate(inst, lin, o, n_iter=5)
    assert np.array_equal(a.K, b.K) and np.array_equal(a.lam_nu, b.lam_nu)
    ws = F.warm_state(lin, a.K, a.pt, a.lam_p)
    c = F.iterate(inst, lin, o, ws, n_iter=1)
    assert c.iters == 1 and np.isfinite(c.r_p)


def test_adaptive_rho_reaches_the_same_fixed_point():
    """Residual balancing changes the path, not the solution: the adaptive loop converges to the
    interior-point solution of Problem 2 as the fixed-ρ loop does."""
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    du_ip, K_ip = problem2_ip(inst, lin, r=0.5)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=100.0, r_trust=0.5, eps_p=1e-9, eps_d=1e-9, max_iter=30000,
                                               adapt_every=25))
    assert s.converged and s.rho < 100.0
    assert np.allclose(s.du, du_ip, atol=2e-6) and np.allclose(s.K, K_ip, atol=2e-6)


def test_stall_stop_on_infeasible_linearization():
    """A trust radius too small to clear an obstacle that the nominal crosses makes Problem 2
    infeasible: the primal residual plateaus and the stall rule stops the loop."""
    inst = tiny_unicycle()
    inst.obs_center = np.array([[0.5, 0.0]])           # on the nominal path
    inst.obs_radius = np.array([0.3])
    lin = P.linearize(inst, inst.u_init)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=1.0, r_trust=0.01, max_iter=5000, stall_every=100))
    assert s.stalled and not s.converged and s.iters < 5000 and s.r_p > 1e-3


def test_budget_stop_cuts_only_a_solve_that_misses_its_cap():
    """The budget stop ends a solve at the first stall checkpoint where r_p, at the geometric rate it
    fell over the last period, would reach ε_p only after the cap.  On this case (ε = 1e-9 with a
    600-iteration cap) the solve without the rule indeed runs to the cap unconverged, so the early
    stop gives up nothing; up to the stop both runs take the same path, and a vanishing factor only
    stops at the cap itself."""
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    base = dict(rho=10.0, r_trust=0.5, eps_p=1e-9, eps_d=1e-9, max_iter=600, stall_every=50)
    full = F.iterate(inst, lin, F.FullADMMOptions(**base))
    cut = F.iterate(inst, lin, F.FullADMMOptions(**base, stall_budget=1.0))
    assert not full.converged and not full.stalled and full.iters == 600
    assert cut.stalled and not cut.converged and 100 <= cut.iters < 600 and cut.iters % 50 == 0
    assert cut.history == full.history[:cut.iters]
    h = [x[0] for x in full.history]
    reach = lambda l: l + 50 * np.log(1e-9 / h[l - 1]) / np.log(h[l - 1] / h[l - 51])
    assert reach(cut.iters) > 600 and all(reach(l) <= 600 for l in range(100, cut.iters, 50))
    assert all(h[l - 1] <= 0.9 * h[l - 51] for l in range(100, cut.iters + 1, 50))   # not the ratio rule
    late = F.iterate(inst, lin, F.FullADMMOptions(**base, stall_budget=1e-9))
    assert late.iters == 600 and late.history == full.history


def test_warm_start_fallback_runs_the_cold_solve():
    """A warm start on an infeasible linearization stalls; the fallback then equals the cold solve
    with the full budget.  On a feasible problem, a warm start at the solution's (k_v, p̃, λ_p)
    needs no fallback and converges (λ_ν restarts at zero, so it is not immediate)."""
    inst = tiny_unicycle()
    inst.obs_center = np.array([[0.5, 0.0]])
    inst.obs_radius = np.array([0.3])
    lin = P.linearize(inst, inst.u_init)
    o = F.FullADMMOptions(rho=1.0, r_trust=0.01, max_iter=2000, stall_every=100)
    w = F.iterate(inst, lin, F.FullADMMOptions(rho=1.0, r_trust=0.01, check=False), n_iter=5)
    s, fell = F.solve_warm_with_fallback(inst, lin, o, w.K, w.pt, w.lam_p)
    first = F.iterate(inst, lin, o, F.warm_state(lin, w.K, w.pt, w.lam_p))
    cold = F.iterate(inst, lin, o, F.zero_state(lin))
    assert fell and first.stalled
    assert s.iters == first.iters + cold.iters
    assert np.array_equal(s.K, cold.K) and np.array_equal(s.du, cold.du)
    feas = tiny_unicycle()
    linf = P.linearize(feas, feas.u_init)
    of = F.FullADMMOptions(rho=10.0, r_trust=0.5, eps_p=1e-6, eps_d=1e-6, max_iter=30000, stall_every=100)
    ref = F.iterate(feas, linf, of)
    s2, fell2 = F.solve_warm_with_fallback(feas, linf, of, ref.K, ref.pt, ref.lam_p)
    assert not fell2 and s2.converged and np.allclose(s2.du, ref.du, atol=1e-5)


def test_carried_start_reaches_the_interior_point_solution_of_the_next_linearization():
    """The inner-state carry starts the next inner solve from the previous one's final state.  Any
    ADMM start converges to the same fixed point, so after an accepted step (new nominal û + δû,
    new linearization) the carried solve must reach the interior-point solution of the new
    Problem 2, like a cold solve."""
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    o = F.FullADMMOptions(rho=10.0, r_trust=0.5, eps_p=1e-9, eps_d=1e-9, max_iter=30000)
    s1 = F.iterate(inst, lin, o)
    assert s1.converged
    # half of the step: a new nominal whose every row is still strictly feasible at δû = 0 (the
    # barrier solver needs a strictly feasible start), so the new solution is interior-pinned
    lin2 = P.linearize(inst, inst.u_init + 0.5 * s1.du)
    assert np.max(lin2.g0 + np.linalg.norm(lin2.bhat.reshape(lin2.g0.shape[0], -1), axis=1)) < -1e-3
    du_ip, K_ip = problem2_ip(inst, lin2, r=0.4)
    o2 = F.FullADMMOptions(rho=10.0, r_trust=0.4, eps_p=1e-9, eps_d=1e-9, max_iter=30000)
    st, rho0 = F.carry_state(lin2, s1, o2, shifted=True)
    assert rho0 == 10.0
    assert np.array_equal(st.K, s1.K) and np.array_equal(st.lam_nu, s1.lam_nu)
    assert not st.du.any() and not st.dx.any() and not st.e.any()
    s2 = F.iterate(inst, lin2, o2, st, rho0=rho0)
    assert s2.converged
    assert np.allclose(s2.du, du_ip, atol=2e-6) and np.allclose(s2.K, K_ip, atol=2e-6)


def test_carry_into_the_same_problem_is_immediately_converged():
    """Carrying a converged state into the same linearization and trust radius (a rejected step
    whose radius did not change) leaves nothing to do: the first iteration already meets the
    tolerances.  A dropped or mis-scaled dual would restart the transient instead."""
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    o = F.FullADMMOptions(rho=10.0, r_trust=0.5, eps_p=1e-7, eps_d=1e-7, max_iter=30000)
    s1 = F.iterate(inst, lin, o)
    assert s1.converged and s1.iters > 20
    st, rho0 = F.carry_state(lin, s1, o, shifted=False)
    s2 = F.iterate(inst, lin, o, st, rho0=rho0)
    assert s2.converged and s2.iters <= 2
    assert np.allclose(s2.du, s1.du, atol=1e-6) and np.allclose(s2.K, s1.K, atol=1e-6)


def test_carry_applies_the_pending_penalty_update_and_keeps_unscaled_duals():
    """With residual balancing, the state at the end of a solve is the one at the start of its next
    iteration, where a scheduled penalty change rescales the scaled duals (λ ← λ ρ_old / ρ_new).
    The unscaled duals ρλ are unchanged by that rescale, and the carried solve still reaches the
    interior-point solution."""
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    found = None
    for eps in (1e-4, 3e-5, 1e-5, 3e-6, 1e-6, 3e-7, 1e-7):
        o = F.FullADMMOptions(rho=100.0, r_trust=0.5, eps_p=eps, eps_d=eps, max_iter=30000, adapt_every=1,
                              adapt_mu=1.5)
        s1 = F.iterate(inst, lin, o)
        st, rho0 = F.carry_state(lin, s1, o, shifted=False)
        if s1.converged and rho0 != s1.rho:
            found = (o, s1, st, rho0)
            break
    assert found is not None, "no tolerance ended on an iteration with a pending penalty change"
    o, s1, st, rho0 = found
    assert np.allclose(rho0 * st.lam_nu, s1.rho * s1.lam_nu, rtol=1e-14, atol=0)
    assert np.allclose(rho0 * st.lam_p, s1.rho * s1.lam_p, rtol=1e-14, atol=0)
    du_ip, K_ip = problem2_ip(inst, lin, r=0.5)
    o2 = F.FullADMMOptions(rho=100.0, r_trust=0.5, eps_p=1e-9, eps_d=1e-9, max_iter=30000, adapt_every=25)
    s2 = F.iterate(inst, lin, o2, st, rho0=rho0)
    assert s2.converged
    assert np.allclose(s2.du, du_ip, atol=2e-6) and np.allclose(s2.K, K_ip, atol=2e-6)


def test_as_written_block2_reaches_the_interior_point_solution():
    """The as-written block 2a (exact constrained (δû, p) QP every iteration, no slacks) converges to
    the interior-point solution of Problem 2, as the lifted split does: both are ADMM splittings of
    the same problem, and their iteration counts differ."""
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    du_ip, K_ip = problem2_ip(inst, lin, r=0.5)
    o = F.FullADMMOptions(rho=10.0, r_trust=0.5, eps_p=1e-8, eps_d=1e-8, max_iter=30000)
    aw = F.iterate_as_written(inst, lin, o)
    lifted = F.iterate(inst, lin, o)
    assert aw.converged and lifted.converged
    assert np.allclose(aw.du, du_ip, atol=2e-6) and np.allclose(aw.K, K_ip, atol=2e-6)
    assert aw.iters != lifted.iters
    # every iterate of the as-written form satisfies the linearized constraints and the trust region
    # exactly (block 2a is feasible by construction): g + bᵀδû + p ≤ 0 and ‖F_u δû‖ ≤ r
    assert np.max(lin.g0 + P.ell(lin, aw.du) + aw.p) <= 1e-10
    assert np.linalg.norm(aw.dx[1:]) <= 0.5 * (1 + 1e-12)


def test_as_written_block2_is_the_dr_subproblem_2_minimizer():
    """One as-written iteration from a given state: its (δû, p) is the KKT point of the block-2a QP,
    checked independently: p = min(p̃ - λ_p, -g - bᵀδû), and the gradient of the squared-hinge
    objective in δû vanishes (trust region inactive at this radius)."""
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    o = F.FullADMMOptions(rho=7.0, r_trust=100.0, check=False)
    s0 = F.iterate(inst, lin, o, n_iter=3)
    s1 = F.iterate_as_written(inst, lin, o, s0, n_iter=1)
    v = s1.pt - s0.lam_p
    assert np.allclose(s1.p, np.minimum(v, -lin.g0 - P.ell(lin, s1.du)), atol=1e-12)
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    du_t = t(s1.du).requires_grad_(True)
    dxv = (t(lin.Fu) @ du_t.reshape(-1)).reshape(inst.T + 1, inst.nx)
    ub = t(lin.u_hat) + du_t - t(inst.u_ref)
    xb = t(lin.x_hat[1:]) + dxv[1:] - t(inst.x_goal)
    z = t(v + lin.g0) + torch.einsum("jku,ku->j", t(lin.bvec), du_t)
    f = torch.sum(ub * ub * t(inst.Ru)) + torch.sum(xb * xb * t(inst.Qx)) + 0.5 * 7.0 * torch.sum(torch.clamp(z, min=0) ** 2)
    g, = torch.autograd.grad(f, [du_t])
    assert g.abs().max().item() < 1e-9


def test_fixed_point_with_singular_sigma_matches_interior_point():
    """Disturbance through a per-step input map Γ_i that misses the heading (Σ_i = Γ_i S_i^{-1} Γ_iᵀ of
    rank 2): the FullADMM fixed point is still the interior-point solution of Problem 2."""
    inst = tiny_unicycle()
    inst.Sigma = np.stack([np.diag([0.02 ** 2, 0.02 ** 2, 0.0])] * (inst.T + 1))
    lin = P.linearize(inst, inst.u_init)
    du_ip, K_ip = problem2_ip(inst, lin, r=0.5)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=0.5, eps_p=1e-9, eps_d=1e-9, max_iter=30000))
    assert s.converged
    assert np.allclose(s.du, du_ip, atol=2e-6) and np.allclose(s.K, K_ip, atol=2e-6)
    assert np.abs(s.K[:, :, 2]).max() < 1e-12        # no disturbance on θ: its feedback column is zero


def test_pcg_gain_solve_matches_the_exact_solve_and_meets_its_tolerance():
    """The PCG k_v update converges to the exact per-step (Kronecker) solve, and at a loose
    tolerance returns an x whose residual meets it; the operator it applies without forming is the
    assembled Q_v + ρ Σ_j Â_jᵀÂ_j (checked against the dense Â_j)."""
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    rho = 7.0
    T, nu, nx = inst.T, inst.nu, inst.nx
    R = RNG.normal(size=(T, nu, nx))
    H = P.gain_hessian_blocks(lin, inst, coef=rho)
    exact = P.gain_solve(H, R)
    x, it = P.gain_solve_pcg(lin, inst, rho, R, np.zeros_like(R), 1e-13, 500)
    assert np.allclose(x, exact, atol=1e-11 * np.abs(exact).max())
    assert it <= T * nu * nx
    # dense operator check: Q_v + ρ Σ Â_jᵀÂ_j applied to a random gain vs the exact solve's inverse
    Ad = [P.dense_Ahat(lin, j) for j in range(lin.g0.shape[0])]
    Hd = 2 * np.kron(np.eye(T * nx), np.diag(inst.RK ** 2)) + rho * sum(a.T @ a for a in Ad)
    kv = np.linalg.solve(Hd, P.kv_from_K(R))
    assert np.allclose(P.K_from_kv(kv, T, nu, nx), exact, atol=1e-10 * np.abs(exact).max())
    x2, it2 = P.gain_solve_pcg(lin, inst, rho, R, np.zeros_like(R), 0.05, 500)
    res = np.linalg.norm(P.kv_from_K(R) - Hd @ P.kv_from_K(x2))
    assert res <= 0.05 * np.linalg.norm(R) and 0 < it2 < it
    # warm start at the solution: nothing to do
    _, it3 = P.gain_solve_pcg(lin, inst, rho, R, exact, 1e-8, 500)
    assert it3 == 0


def test_fulladmm_with_tight_pcg_equals_the_exact_gain_update():
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    a = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=0.5, check=False), n_iter=30)
    b = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=0.5, check=False, kv_pcg_iters=500,
                                               kv_pcg_tol=1e-13), n_iter=30)
    assert np.allclose(a.K, b.K, atol=1e-10 * np.abs(a.K).max()) and np.allclose(a.du, b.du, atol=1e-10)
    assert b.pcg_iters > 0


def test_lifted_warm_start_at_a_solution_is_its_fixed_point():
    """At a converged solution the scaled dual λ_ν,j of a row whose cone is not projected to zero is
    a non-negative multiple of Â_j k + b̂_j (the SOC fixed point), so one scalar per row rebuilds it;
    from the solution's (k_v, p̃, λ_p, θ, δû, λ_w, λ_e) at the penalty its scaled duals belong to, the
    first iteration meets the tolerances and returns the same solution.  With θ clipped at zero (rows
    projected to zero, whose SOC vector vanishes, restart λ_ν at zero) it takes at most one more.
    The plain (k_v, p̃, λ_p) warm start, which restarts the rest at zero, does not."""
    inst = W.quadcopter(1, T=12, n_obs=3)
    lin = P.linearize(inst, inst.u_init)
    o = F.FullADMMOptions(rho=10.0, r_trust=2.0, max_iter=20000, eps_p=1e-8, eps_d=1e-8, adapt_every=25)
    ref = F.iterate(inst, lin, o)
    assert ref.converged and ref.iters > 20 and ref.rho != 10.0
    Y = P.Ahat_apply(lin, ref.K) + lin.bhat
    yy = np.sum(Y * Y, axis=(1, 2))
    theta = np.where(yy > 0, np.sum(ref.lam_nu * Y, axis=(1, 2)) / np.where(yy > 0, yy, 1.0), 0.0)
    resid = ref.lam_nu - theta[:, None, None] * Y
    assert np.max(np.abs(resid)) < 1e-6 * max(1.0, np.max(np.abs(ref.lam_nu)))
    live = yy > 1e-12                 # rows whose SOC vector does not vanish at the solution
    assert live.sum() > 10 and np.all(theta[live] > -1e-6)
    st = F.warm_state_lifted(lin, ref.K, ref.pt, ref.lam_p, theta, ref.du, ref.lam_w, ref.lam_e)
    assert np.allclose(st.dx, ref.dx, atol=1e-9)          # δx = F_u δû of the solution
    s1 = F.iterate(inst, lin, o, st, rho0=ref.rho)
    assert s1.converged and s1.iters == 1
    assert np.allclose(s1.du, ref.du, rtol=1e-6, atol=1e-8) and np.allclose(s1.K, ref.K, rtol=1e-3, atol=1e-8)
    st0 = F.warm_state_lifted(lin, ref.K, ref.pt, ref.lam_p, np.maximum(theta, 0.0), ref.du, ref.lam_w, ref.lam_e)
    s2 = F.iterate(inst, lin, o, st0, rho0=ref.rho)
    assert s2.converged and s2.iters <= 2 and np.allclose(s2.du, ref.du, rtol=1e-6, atol=1e-8)
    plain = F.iterate(inst, lin, o, F.warm_state(lin, ref.K, ref.pt, ref.lam_p), rho0=ref.rho)
    assert plain.iters > 10
