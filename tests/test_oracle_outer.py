"""Checks of the oracle's successive-linearization loop: against its stated definition (the
acceptance rule and the radius schedule's constants come from prior work) and, independently of
that rule, on a convex case where the loop's end point is fixed by the mathematics."""
import numpy as np

from oracle import fulladmm as F, outer as O, problem as P
from paper_2603_02642_b300 import workloads as W

from .test_oracle_fulladmm import problem2_ip, tiny_unicycle


def test_cost_definition():
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    K = np.ones((inst.T, inst.nu, inst.nx))
    c = O.cost(inst, lin, K)
    ud = inst.u_init - inst.u_ref
    xd = lin.x_hat[1:] - inst.x_goal
    expect = (ud * ud * inst.Ru).sum() + (xd * xd * inst.Qx).sum() + inst.T * inst.nx * (inst.RK ** 2).sum()
    assert np.isclose(c, expect)


def test_accepted_steps_decrease_merit_and_radius_schedule():
    inst = tiny_unicycle()
    res = O.solve(inst, O.OuterOptions(n_outer=5), F.FullADMMOptions(max_iter=400))
    assert len(res.accepted) == 5
    for i in range(1, 5):
        r_prev, r = res.radii[i - 1], res.radii[i]
        expect = min(1.5 * r_prev, 2.0) if res.accepted[i - 1] else max(0.8 * r_prev, 1e-3)
        assert np.isclose(r, expect)
    lin0 = P.linearize(inst, inst.u_init)
    assert res.phi <= O.merit(inst, lin0, np.zeros((inst.T, inst.nu, inst.nx)), 10.0)


def test_carry_changes_the_path_not_the_outer_iterates():
    """With every inner solve converged tightly, each outer step's candidate is the unique
    (δû, k_v) solution of its Problem 2 whatever the inner start, so the carried and the
    re-initialized outer loops accept the same steps and end at the same (ū, K); the carried
    one needs fewer inner iterations after the first step."""
    inst = tiny_unicycle()
    a = F.FullADMMOptions(rho=10.0, eps_p=1e-10, eps_d=1e-10, max_iter=40000)
    cold = O.solve(inst, O.OuterOptions(n_outer=4), a)
    warm = O.solve(inst, O.OuterOptions(n_outer=4, carry=True), a)
    assert cold.accepted == warm.accepted
    assert all(cold.inner_converged) and all(warm.inner_converged)
    assert np.allclose(cold.u_bar, warm.u_bar, atol=1e-7) and np.allclose(cold.K, warm.K, atol=1e-7)
    assert warm.inner_iters[0] == cold.inner_iters[0]
    assert sum(warm.inner_iters[1:]) < sum(cold.inner_iters[1:])
    lin = P.linearize(inst, warm.u_bar)
    assert np.isclose(warm.max_violation, np.max(O.robust_violation(lin, warm.K)))
    assert warm.accepted_inner_converged


def test_final_step_cap_applies_to_the_last_inner_solve_only():
    inst = tiny_unicycle()
    a = F.FullADMMOptions(rho=10.0, max_iter=5)
    res = O.solve(inst, O.OuterOptions(n_outer=3, carry=True, max_inner_final=3000), a)
    assert res.inner_iters[:2] == [5, 5]
    assert res.inner_iters[2] > 5 and res.inner_converged[2]


def linear_arm(T=3):
    """A convex case: the arm's double integrator (linear dynamics) with velocity limits on two
    joints as the only constraints (linear), a light control weight and a wider disturbance, so
    that two robust constraints are active at the optimum and the gains are not zero there."""
    inst = W.arm(3, T=T, n_link=1, n_static=0)
    lo, hi = np.full(14, -np.inf), np.full(14, np.inf)
    lo[7:9], hi[7:9] = -0.08, 0.08
    inst.x_lo, inst.x_hi = lo, hi
    inst.Ru = 1e-3 * np.ones(7)
    inst.Sigma = 10.0 * inst.Sigma
    return inst


def test_outer_loop_reaches_the_convex_optimum_for_linear_dynamics():
    """With linear dynamics and linear constraints, Problem 2 at any nominal is Problem 1 itself
    (the first-order robust reformulation is exact), so successive linearization must end at
    Problem 1's optimum: the barrier solution of Problem 2 around the initial nominal with an
    inactive trust region.  In one step when the trust radius does not bind; in several accepted
    steps when it does, each one truncated to the ball."""
    inst = linear_arm()
    lin0 = P.linearize(inst, inst.u_init)
    du_ip, K_ip = problem2_ip(inst, lin0, r=1e3)
    viol = O.robust_violation(lin0, K_ip) + P.ell(lin0, du_ip)
    assert np.sum(viol > -1e-6) >= 2 and np.abs(K_ip).max() > 1e-5      # active rows, gains not zero
    admm = F.FullADMMOptions(rho=10.0, eps_p=1e-10, eps_d=1e-10, max_iter=40000)
    res = O.solve(inst, O.OuterOptions(n_outer=3, r0=1e3), admm)
    assert res.accepted[0] and all(res.inner_converged)
    np.testing.assert_allclose(res.u_bar, inst.u_init + du_ip, rtol=0, atol=1e-8)
    np.testing.assert_allclose(res.K, K_ip, rtol=0, atol=1e-11)
    # trust radius a third of the optimal step: the first accepted steps are truncated
    r_star = np.linalg.norm(lin0.Fu @ du_ip.reshape(-1))
    res = O.solve(inst, O.OuterOptions(n_outer=10, r0=r_star / 3), admm)
    assert res.accepted[:4] == [True] * 4 and all(res.inner_converged)
    np.testing.assert_allclose(res.u_bar, inst.u_init + du_ip, rtol=0, atol=1e-8)
    np.testing.assert_allclose(res.K, K_ip, rtol=0, atol=1e-11)
