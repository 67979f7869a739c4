"""GPU parity of FullADMM with block 2a as the paper states it (the constrained (δû, p) QP solved
exactly each iteration, NRTO_SOLVER_FULLADMM_AW) against oracle/fulladmm.iterate_as_written in FP64,
and its fixed point and iteration count against the lifted form."""
import numpy as np
import pytest

from oracle import fulladmm as F, problem as P
from paper_2603_02642_b300 import nrto, workloads as W

from .gpu_common import RTOL64, assert_close, ragged_from_dense, relerr

pytestmark = pytest.mark.gpu

CASES = {
    "uni_T20_o3_r05": (lambda: W.unicycle(0, T=20, n_obs=3), 0.5),      # trust region active
    "uni_T40_o6_r50": (lambda: W.unicycle(11, T=40, n_obs=6), 50.0),    # several chunks, inactive
    "quad_T16_o3_r05": (lambda: W.quadcopter(12, T=16, n_obs=3), 0.5),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("n_iter", [1, 2, 10])
def test_as_written_iterates_parity_fp64(name, n_iter):
    make, r = CASES[name]
    inst = make()
    lin = P.linearize(inst, inst.u_init)
    s = F.iterate_as_written(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=r, check=False), n_iter=n_iter)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(r)
    out = prob.solve_socp(nrto.Options(solver=nrto.SOLVER_FULLADMM_AW, rho=10.0, max_inner=n_iter, check=0))
    assert out["iters"][0] == n_iter
    assert_close(out["K"][0], s.K, RTOL64, "K")
    assert_close(out["du"][0], s.du, RTOL64, "du")
    assert_close(out["p"][0], s.p, RTOL64, "p")
    assert_close(out["pt"][0], s.pt, RTOL64, "p~")
    assert_close(prob.export(nrto.F_LAMP, 0), s.lam_p, RTOL64, "lambda_p")
    assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, s.lam_nu), RTOL64, "lambda_nu")
    assert_close(prob.export(nrto.F_DX, 0), s.dx, RTOL64, "dx")
    # r_p, r_d are norms of differences of iterates that each carry a 1e-8 relative error, so their
    # bound scales with the iterates' norms (ρ for r_d), not with the residuals themselves
    sc = prob.export(nrto.F_SCAL, 0)
    scale = np.linalg.norm(s.p) + np.linalg.norm(s.pt) + np.linalg.norm(s.lam_nu)
    assert abs(sc[0] - s.r_p) <= RTOL64 * 2 * scale
    assert abs(sc[1] - s.r_d) <= RTOL64 * 10.0 * 2 * scale
    prob.close()


def test_as_written_and_lifted_reach_the_same_solution_with_different_counts():
    """Both splittings converge to the Problem 2 solution (δû, k_v are unique); the iteration
    counts to the full residuals ≤ 1e-4 equal the oracle's for each form."""
    from .test_oracle_fulladmm import tiny_unicycle
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    o = F.FullADMMOptions(rho=10.0, r_trust=0.5, eps_p=1e-6, eps_d=1e-6, max_iter=20000)
    aw = F.iterate_as_written(inst, lin, o)
    li = F.iterate(inst, lin, o)
    res = {}
    for solver in (nrto.SOLVER_FULLADMM_AW, nrto.SOLVER_FULLADMM):
        prob = nrto.Problem([inst], nrto.PREC_FP64)
        prob.linearize()
        prob.set_trust_radius(0.5)
        res[solver] = prob.solve_socp(nrto.Options(solver=solver, rho=10.0, max_inner=20000, eps_p=1e-6,
                                                   eps_d=1e-6, check=1))
        prob.close()
    ga, gl = res[nrto.SOLVER_FULLADMM_AW], res[nrto.SOLVER_FULLADMM]
    assert ga["status"][0] == 1 and gl["status"][0] == 1
    assert ga["iters"][0] == aw.iters and gl["iters"][0] == li.iters
    assert aw.iters != li.iters
    # at this case the gains are small (‖K‖ ~ 1e-5), so they agree to the tolerance in absolute terms
    assert relerr(ga["du"][0], gl["du"][0]) < 1e-4 and np.abs(ga["K"][0] - gl["K"][0]).max() < 1e-4


def test_as_written_mixed_precision_bounds():
    """Mixed precision after 10 iterations, on the unicycle case whose gains are well away from zero
    (the quadcopter case's gains are ~1e-9 there, below the FP32 resolution of the sums that form them)."""
    make, r = CASES["uni_T20_o3_r05"]
    inst = make()
    lin = P.linearize(inst, inst.u_init)
    s = F.iterate_as_written(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=r, check=False), n_iter=10)
    prob = nrto.Problem([inst], nrto.PREC_MIXED)
    prob.linearize()
    prob.set_trust_radius(r)
    out = prob.solve_socp(nrto.Options(solver=nrto.SOLVER_FULLADMM_AW, rho=10.0, max_inner=10, check=0))
    assert relerr(out["K"][0], s.K) < 5e-4 and relerr(out["du"][0], s.du) < 5e-5 and relerr(out["pt"][0], s.pt) < 5e-5
    prob.close()
