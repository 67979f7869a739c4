"""GPU parity of the FullADMM inner-state carry (each inner solve after the first starts from the
previous one's final state) against oracle/fulladmm.carry_state and oracle/outer.solve(carry=True)
in FP64, and of the per-instance statistics (nrto_get_stats) including the robust-constraint value
of the accepted iterate."""
import numpy as np
import pytest

from oracle import fulladmm as F, outer as O, problem as P
from paper_2603_02642_b300 import nrto, workloads as W

from .gpu_common import RTOL64, assert_close, ragged_from_dense

pytestmark = pytest.mark.gpu

# (instance, residual-balancing period): each mixes converged and capped inner solves, accepted
# and rejected outer steps (rejected: carried into the same nominal; accepted: shifted to û + δû),
# and penalty updates pending at the end of a converged solve.
# The last case keeps the inner solves inexact (40 iterations) during the linearization steps and
# solves the last step's subproblem with a larger cap (max_inner_final).
OUTER_CASES = {
    "uni_T12_o1_adapt5": (lambda: W.unicycle(1, T=12, n_obs=1), 5, 400, 0),
    "quad_T16_o2_adapt5": (lambda: W.quadcopter(5, T=16, n_obs=2), 5, 400, 0),
    "uni_T20_o3_fixed": (lambda: W.unicycle(0, T=20, n_obs=3), 0, 400, 0),
    "quad_T16_o2_adapt5_cap40_final400": (lambda: W.quadcopter(5, T=16, n_obs=2), 5, 40, 400),
}


@pytest.mark.parametrize("name", list(OUTER_CASES))
def test_outer_loop_with_carry_parity_fp64(name):
    make, adapt, cap, cap_final = OUTER_CASES[name]
    inst = make()
    res = O.solve(inst, O.OuterOptions(n_outer=6, r0=2.0, r_min=1e-3, w_p=10.0, carry=True, max_inner_final=cap_final),
                  admm=F.FullADMMOptions(rho=10.0, max_iter=cap, eps_p=1e-4, eps_d=1e-4, adapt_every=adapt))
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    out = prob.solve(nrto.Options(rho=10.0, max_inner=cap, eps_p=1e-4, eps_d=1e-4, check=1, r0=2.0, r_min=1e-3,
                                  w_p=10.0, adapt_every=adapt, carry=1, max_inner_final=cap_final), n_outer=6)
    st = prob.stats()
    assert st["n_accepted"][0] == sum(res.accepted)
    assert st["cum_iters"][0] == sum(res.inner_iters), (st["cum_iters"][0], res.inner_iters)
    assert_close(out["u_bar"][0], res.u_bar, RTOL64, "u_bar")
    assert_close(out["K"][0], res.K, RTOL64, "K")
    assert abs(out["merit"][0] - res.phi) <= RTOL64 * abs(res.phi)
    assert abs(st["max_violation"][0] - res.max_violation) <= RTOL64 * max(1.0, abs(res.max_violation))
    assert (st["accepted_status"][0] == 1) == res.accepted_inner_converged
    prob.close()


@pytest.mark.parametrize("prec_tol", [(nrto.PREC_FP64, RTOL64)])
def test_carry_into_the_same_linearization_iterates_parity(prec_tol):
    """Two inner solves on one linearization with carry: the second continues from the first's
    final state (δû, δx, e included, as the nominal did not move); iterates after 7 + 5
    iterations at fixed counts."""
    prec, tol = prec_tol
    inst = W.quadcopter(4, T=40, n_obs=5)
    lin = P.linearize(inst, inst.u_init)
    o = F.FullADMMOptions(rho=10.0, r_trust=0.5, check=False)
    s1 = F.iterate(inst, lin, o, n_iter=7)
    st0, rho0 = F.carry_state(lin, s1, o, shifted=False)
    s2 = F.iterate(inst, lin, o, st0, n_iter=5, rho0=rho0)
    prob = nrto.Problem([inst], prec)
    prob.linearize()
    prob.set_trust_radius(0.5)
    prob.solve_socp(nrto.Options(rho=10.0, max_inner=7, check=0, carry=1))
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=5, check=0, carry=1))
    assert out["iters"][0] == 5
    assert_close(out["K"][0], s2.K, tol, "K")
    assert_close(out["du"][0], s2.du, tol, "du")
    assert_close(out["p"][0], s2.p, tol, "p")
    assert_close(out["pt"][0], s2.pt, tol, "p~")
    assert_close(prob.export(nrto.F_LAMP, 0), s2.lam_p, tol, "lambda_p")
    assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, s2.lam_nu), tol, "lambda_nu")
    assert_close(prob.export(nrto.F_DX, 0), s2.dx, tol, "dx")
    sc = prob.export(nrto.F_SCAL, 0)
    assert abs(sc[0] - s2.r_p) <= tol * s2.r_p and abs(sc[1] - s2.r_d) <= tol * s2.r_d
    prob.close()


def test_carry_off_and_reset_start_cold():
    """carry = 0, and the first inner solve after a reset, are the cold solves of Algorithm 1."""
    inst = W.unicycle(3, T=30, n_obs=2)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(0.5)
    a = prob.solve_socp(nrto.Options(rho=10.0, max_inner=9, check=0, carry=0))
    b = prob.solve_socp(nrto.Options(rho=10.0, max_inner=9, check=0, carry=0))
    assert np.array_equal(a["K"][0], b["K"][0]) and np.array_equal(a["du"][0], b["du"][0])
    prob.linearize(inst.u_init.reshape(1, -1))   # a new nominal from the caller: the next solve is cold
    c = prob.solve_socp(nrto.Options(rho=10.0, max_inner=9, check=0, carry=1))
    assert np.array_equal(a["K"][0], c["K"][0]) and np.array_equal(a["du"][0], c["du"][0])
    prob.close()


def test_stats_agree_with_exports():
    insts = [W.unicycle(0, T=20, n_obs=3), W.quadcopter(5, T=16, n_obs=2)]
    prob = nrto.Problem(insts, nrto.PREC_FP64)
    prob.solve(nrto.Options(rho=10.0, max_inner=60, check=1, adapt_every=5, carry=1), n_outer=3)
    st = prob.stats()
    for i in range(len(insts)):
        e = prob.export(nrto.F_STATS, i)
        sc = prob.export(nrto.F_SCAL, i)
        assert [st[k][i] for k in ("cum_iters", "iters", "status", "n_accepted", "rho", "dr_iters", "fallback")] \
            == list(e)
        assert st["merit"][i] == sc[4] and st["trust_radius"][i] == sc[7]
        assert st["r_p"][i] == sc[0] and st["r_d"][i] == sc[1]
        assert np.isfinite(st["max_violation"][i]) and np.isfinite(st["cost"][i])
    prob.close()
