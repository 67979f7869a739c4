"""GPU parity of the FullADMM k_v update by matrix-free Jacobi-PCG (Sec. IV, GPU implementation;
Supplementary Tables VI-VIII: iteration cap 100, relative tolerance 0.05) against
oracle/fulladmm.iterate(kv_pcg_iters > 0) in FP64: iterates at fixed counts, the PCG iteration count,
and, with a tolerance far below the solve's own, the exact per-step solve's iterates."""
import numpy as np
import pytest

from oracle import fulladmm as F, problem as P
from paper_2603_02642_b300 import nrto, workloads as W

from .gpu_common import RTOL64, assert_close, ragged_from_dense

pytestmark = pytest.mark.gpu

CASES = {
    "uni_T30_o3": lambda: W.unicycle(2, T=30, n_obs=3),
    "quad_T40_o5": lambda: W.quadcopter(4, T=40, n_obs=5),
    "arm_T20": lambda: W.franka(3, T=20),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("cap_tol", [(100, 0.05), (3, 0.01)])
def test_pcg_iterates_parity_fp64(name, cap_tol):
    cap, tol = cap_tol
    inst = CASES[name]()
    lin = P.linearize(inst, inst.u_init)
    o = F.FullADMMOptions(rho=10.0, r_trust=0.5, check=False, kv_pcg_iters=cap, kv_pcg_tol=tol)
    s = F.iterate(inst, lin, o, n_iter=9)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(0.5)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=9, check=0, kv_pcg_iters=cap, kv_pcg_tol=tol))
    assert out["iters"][0] == 9
    assert prob.stats()["pcg_iters"][0] == s.pcg_iters
    assert_close(out["K"][0], s.K, RTOL64, "K")
    assert_close(out["du"][0], s.du, RTOL64, "du")
    assert_close(out["p"][0], s.p, RTOL64, "p")
    assert_close(out["pt"][0], s.pt, RTOL64, "p~")
    assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, s.lam_nu), RTOL64, "lambda_nu")
    sc = prob.export(nrto.F_SCAL, 0)
    assert abs(sc[0] - s.r_p) <= RTOL64 * s.r_p and abs(sc[1] - s.r_d) <= RTOL64 * s.r_d
    prob.close()


def test_pcg_at_tight_tolerance_matches_the_exact_solve():
    """tol 1e-13 with a generous cap: the PCG gains are the exact per-step solve's to ~1e-10."""
    inst = W.quadcopter(6, T=24, n_obs=3)
    lin = P.linearize(inst, inst.u_init)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=0.5, check=False), n_iter=6)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(0.5)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=6, check=0, kv_pcg_iters=5000, kv_pcg_tol=1e-13))
    assert prob.stats()["pcg_iters"][0] > 0
    assert_close(out["K"][0], s.K, 1e-8, "K")
    assert_close(out["du"][0], s.du, 1e-8, "du")
    prob.close()


def test_pcg_solve_in_mixed_precision_converges():
    """The whole outer loop with PCG gain updates in the mixed-precision solver: under the same
    schedule as the exact-solve run, about as many instances end on a converged accepted step, at a
    merit within a few percent of the exact-solve run's."""
    insts = [W.unicycle(s, T=40, n_obs=4) for s in range(3)] + [W.quadcopter(s, T=40, n_obs=4) for s in range(3)]
    opts = dict(rho=10.0, max_inner=2000, check=1, adapt_every=25, eps_p=1e-4, eps_d=1e-4)
    res = {}
    for cap in (0, 100):
        prob = nrto.Problem(insts, nrto.PREC_MIXED)
        prob.solve(nrto.Options(kv_pcg_iters=cap, kv_pcg_tol=0.05, **opts), n_outer=6)
        res[cap] = prob.stats()
        prob.close()
    assert np.all(res[100]["pcg_iters"] > 0) and np.all(res[0]["pcg_iters"] == 0)
    ok = {c: res[c]["accepted_status"] == 1 for c in res}
    assert ok[100].sum() >= ok[0].sum() - 1
    both = ok[0] & ok[100]
    assert np.all(np.abs(res[100]["merit"][both] - res[0]["merit"][both]) <= 0.05 * np.abs(res[0]["merit"][both]))


def test_pcg_option_rejected_for_other_solvers():
    inst = W.unicycle(0, T=12, n_obs=1)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    with pytest.raises(nrto.NrtoError):
        prob.solve_socp(nrto.Options(solver=nrto.SOLVER_DR, kv_pcg_iters=10))
    with pytest.raises(nrto.NrtoError):
        prob.solve_socp(nrto.Options(kv_pcg_iters=10, kv_pcg_tol=1.5))
    prob.close()
