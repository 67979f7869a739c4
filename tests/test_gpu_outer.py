"""GPU parity of the successive-linearization outer loop (Fig. 1, Problem 2; accept/reject and
trust-radius reading of the oracle) against oracle/outer.py in FP64: the accepted nominal ū,
the accepted gains K and the merit after n_outer steps, with FullADMM and with NRTO-DR inside."""
import numpy as np
import pytest

from oracle import dr as DRO, fulladmm as F, outer as O
from paper_2603_02642_b300 import nrto, workloads as W

from .gpu_common import RTOL64, assert_close

pytestmark = pytest.mark.gpu

CASES = {
    "uni_T20_o3": lambda: W.unicycle(0, T=20, n_obs=3),
    "quad_T16_o2": lambda: W.quadcopter(5, T=16, n_obs=2),
}


@pytest.mark.parametrize("name", list(CASES))
def test_outer_loop_fulladmm_parity_fp64(name):
    inst = CASES[name]()
    res = O.solve(inst, O.OuterOptions(n_outer=4, r0=2.0, r_min=1e-3, w_p=10.0),
                  admm=F.FullADMMOptions(rho=10.0, max_iter=40, eps_p=1e-4, eps_d=1e-4))
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    out = prob.solve(nrto.Options(rho=10.0, max_inner=40, eps_p=1e-4, eps_d=1e-4, check=1, r0=2.0, r_min=1e-3,
                                  w_p=10.0), n_outer=4)
    st = prob.export(nrto.F_STATS, 0)
    assert st[3] == sum(res.accepted)
    assert_close(out["u_bar"][0], res.u_bar, RTOL64, "u_bar")
    assert_close(out["K"][0], res.K, RTOL64, "K")
    assert abs(out["merit"][0] - res.phi) <= RTOL64 * abs(res.phi)
    prob.close()


def test_outer_loop_dr_parity_fp64():
    inst = CASES["uni_T20_o3"]()
    res = O.solve(inst, O.OuterOptions(n_outer=2, r0=2.0, r_min=1e-3, w_p=10.0, solver="dr"),
                  dropts=DRO.DROptions(rho=40.0, max_admm=5, max_dr=50, eps_dr=1e-4, eps_p=1e-4, eps_d=1e-4))
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    out = prob.solve(nrto.Options(solver=nrto.SOLVER_DR, rho=40.0, max_inner=5, max_dr=50, eps_dr=1e-4, eps_p=1e-4,
                                  eps_d=1e-4, check=1, r0=2.0, r_min=1e-3, w_p=10.0), n_outer=2)
    st = prob.export(nrto.F_STATS, 0)
    assert st[3] == sum(res.accepted)
    assert_close(out["u_bar"][0], res.u_bar, 1e-7, "u_bar")
    assert_close(out["K"][0], res.K, 1e-7, "K")
    assert abs(out["merit"][0] - res.phi) <= 1e-7 * abs(res.phi)
    prob.close()


def test_outer_loop_mixed_precision_merit_close():
    """Mixed precision (FP32 rows, merit row norms in FP32): merit within 1e-4 of the FP64 run."""
    inst = CASES["quad_T16_o2"]()
    o = nrto.Options(rho=10.0, max_inner=40, eps_p=1e-4, eps_d=1e-4, check=1, r0=2.0, r_min=1e-3, w_p=10.0)
    p64 = nrto.Problem([inst], nrto.PREC_FP64)
    m64 = p64.solve(o, n_outer=3)["merit"][0]
    p32 = nrto.Problem([inst], nrto.PREC_MIXED)
    m32 = p32.solve(o, n_outer=3)["merit"][0]
    assert abs(m32 - m64) <= 1e-4 * abs(m64)
    p64.close()
    p32.close()
