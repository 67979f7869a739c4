"""Checks of the oracle's successive-linearization loop against its stated definition
(parity unpinned against the paper: the acceptance constants come from prior work)."""
import numpy as np

from oracle import fulladmm as F, outer as O, problem as P

from .test_oracle_fulladmm import tiny_unicycle


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
