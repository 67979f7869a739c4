"""GPU parity on the degenerate and extreme inputs the library accepts: an instance with no state
rows (no obstacles and no state bounds, so the row pass has no chunks and only control rows carry
cones), the shortest horizon T = 1, the longest horizon of the unicycle and the quadcopter kernels,
and batches that mix such instances with ordinary ones.  FullADMM and NRTO-DR inner solves and the
outer loop, FP64, with the tolerances of the other parity tests; batches bitwise equal to
single-instance solves."""
import numpy as np
import pytest

from oracle import dr as DRO, fulladmm as F, outer as O, problem as P
from paper_2603_02642_b300 import nrto, workloads as W

from .gpu_common import RTOL64, assert_close, ragged_from_dense

pytestmark = pytest.mark.gpu

CASES = {
    "quad_T10_no_state_rows": lambda: W.quadcopter(11, T=10, n_obs=0),
    "uni_T1": lambda: W.unicycle(12, T=1, n_obs=2),
    "uni_T256_longest": lambda: W.unicycle(13, T=256, n_obs=1),
    "quad_T160_longest": lambda: W.quadcopter(14, T=160, n_obs=1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_degenerate_and_extreme_iterates_parity_fp64(name):
    inst = CASES[name]()
    n_iter, r = 3, 0.5
    lin = P.linearize(inst, inst.u_init)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=r, check=False), n_iter=n_iter)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(r)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=n_iter, check=0))
    assert prob.info[0].n_state_rows == lin.n_state
    if name == "quad_T10_no_state_rows":
        assert prob.info[0].n_entries_state == 0 and prob.info[0].n_control_rows > 0
    assert out["iters"][0] == n_iter
    assert_close(prob.export(nrto.F_XHAT, 0), lin.x_hat, 1e-12, "x_hat")
    assert_close(out["K"][0], s.K, RTOL64, "K")
    assert_close(out["du"][0], s.du, RTOL64, "du")
    assert_close(out["p"][0], s.p, RTOL64, "p")
    assert_close(out["pt"][0], s.pt, RTOL64, "p~")
    assert_close(prob.export(nrto.F_LAMP, 0), s.lam_p, RTOL64, "lambda_p")
    assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, s.lam_nu), RTOL64, "lambda_nu")
    assert_close(prob.export(nrto.F_DX, 0), s.dx, RTOL64, "dx")
    sc = prob.export(nrto.F_SCAL, 0)
    assert abs(sc[0] - s.r_p) <= RTOL64 * max(s.r_p, 1e-300) + 1e-14
    assert abs(sc[1] - s.r_d) <= RTOL64 * max(s.r_d, 1e-300) + 1e-14
    prob.close()


@pytest.mark.parametrize("prec", [nrto.PREC_FP64, nrto.PREC_MIXED])
def test_batch_with_degenerate_members_equals_single_instances(prec):
    """Instances without state rows and with T = 1 beside ordinary ones: every instance of the batch
    gets the iterates it gets when solved alone."""
    insts = [W.unicycle(12, T=1, n_obs=2), W.quadcopter(11, T=10, n_obs=0), W.quadcopter(15, T=20, n_obs=2),
             W.unicycle(16, T=30, n_obs=3), W.unicycle(17, T=1, n_obs=0)]
    opts = nrto.Options(rho=10.0, max_inner=12, check=0)
    batch = nrto.Problem(insts, prec)
    batch.linearize()
    batch.set_trust_radius(0.5)
    ob = batch.solve_socp(opts)
    for i, inst in enumerate(insts):
        single = nrto.Problem([inst], prec)
        single.linearize()
        single.set_trust_radius(0.5)
        os_ = single.solve_socp(opts)
        assert np.all(np.isfinite(ob["K"][i])) and np.all(np.isfinite(ob["du"][i]))
        assert np.array_equal(ob["K"][i], os_["K"][0]) and np.array_equal(ob["du"][i], os_["du"][0])
        assert np.array_equal(ob["p"][i], os_["p"][0])
        single.close()
    batch.close()


DEGENERATE = ["quad_T10_no_state_rows", "uni_T1"]


@pytest.mark.parametrize("name", DEGENERATE)
def test_degenerate_dr_iterates_parity_fp64(name):
    inst = CASES[name]()
    n_admm, n_dr, r = 2, 3, 0.5
    lin = P.linearize(inst, inst.u_init)
    o = DRO.DROptions(rho=40.0, alpha=0.9, r_chi=1.0, sigma=1.0, r_trust=r, max_admm=n_admm, max_dr=n_dr)
    res = DRO.solve(inst, lin, o, n_admm=n_admm, n_dr=n_dr, check=False)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(r)
    out = prob.solve_socp(nrto.Options(solver=nrto.SOLVER_DR, rho=40.0, alpha=0.9, r_chi=1.0, sigma=1.0,
                                       max_inner=n_admm, max_dr=n_dr, check=0))
    assert out["iters"][0] == n_admm
    assert_close(out["K"][0], res.K, RTOL64, "K")
    assert_close(out["du"][0], res.du, RTOL64, "du")
    assert_close(out["p"][0], res.p, RTOL64, "p")
    assert_close(out["pt"][0], res.pt, RTOL64, "p~")
    assert_close(prob.export(nrto.F_LAMP, 0), res.lam, RTOL64, "lambda")
    assert_close(prob.export(nrto.F_DX, 0), res.dx, RTOL64, "dx")
    assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, res.dr_state.etat), RTOL64, "eta~")
    prob.close()


@pytest.mark.parametrize("name", DEGENERATE)
def test_degenerate_outer_loop_parity_fp64(name):
    inst = CASES[name]()
    res = O.solve(inst, O.OuterOptions(n_outer=3, r0=2.0, r_min=1e-3, w_p=10.0),
                  admm=F.FullADMMOptions(rho=10.0, max_iter=40, eps_p=1e-4, eps_d=1e-4))
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    out = prob.solve(nrto.Options(rho=10.0, max_inner=40, eps_p=1e-4, eps_d=1e-4, check=1, r0=2.0, r_min=1e-3,
                                  w_p=10.0), n_outer=3)
    st = prob.export(nrto.F_STATS, 0)
    assert st[3] == sum(res.accepted)
    assert_close(out["u_bar"][0], res.u_bar, RTOL64, "u_bar")
    assert_close(out["K"][0], res.K, RTOL64, "K")
    assert abs(out["merit"][0] - res.phi) <= RTOL64 * abs(res.phi)
    prob.close()
