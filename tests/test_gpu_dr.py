"""GPU parity of the NRTO-DR inner solve (Sec. II-B, Sec. III, Supplementary Sec. II) against the
oracle, through the C ABI: FP64 element-wise within 1e-8 relative at fixed ADMM / DR iteration
counts, termination counts with the tolerances on, and mixed-precision error bounds."""
import numpy as np
import pytest

from oracle import dr as DRO, problem as P
from paper_2603_02642_b300 import nrto, workloads as W

from .gpu_common import RTOL64, assert_close, ragged_from_dense, relerr

pytestmark = pytest.mark.gpu

# Small horizons: subproblem 2 runs a bisection of semismooth-Newton solves in FP64.  The unicycle
# case spans several solver chunks with a ragged tail; the trust radius of 0.5 is active.
CASES = {
    "uni_T20_o3": lambda: W.unicycle(0, T=20, n_obs=3),
    "uni_T40_o6": lambda: W.unicycle(11, T=40, n_obs=6),
    "quad_T16_o3": lambda: W.quadcopter(12, T=16, n_obs=3),
    "arm_T8": lambda: W.arm(13, T=8),
}


@pytest.fixture(scope="module")
def cases():
    return {k: f() for k, f in CASES.items()}


def _opts(n_admm, n_dr, check, r):
    o = DRO.DROptions(rho=40.0, alpha=0.9, r_chi=1.0, sigma=1.0, r_trust=r, max_admm=n_admm, max_dr=n_dr)
    g = nrto.Options(solver=nrto.SOLVER_DR, rho=40.0, alpha=0.9, r_chi=1.0, sigma=1.0, max_inner=n_admm,
                     max_dr=n_dr, check=check)
    return o, g


def _run(inst, n_admm, n_dr, r, prec=nrto.PREC_FP64, check=0):
    lin = P.linearize(inst, inst.u_init)
    o, g = _opts(n_admm, n_dr, check, r)
    res = DRO.solve(inst, lin, o, n_admm=None if check else n_admm, n_dr=None if check else n_dr,
                    check=bool(check))
    prob = nrto.Problem([inst], prec)
    prob.linearize()
    prob.set_trust_radius(r)
    out = prob.solve_socp(g)
    return lin, res, prob, out


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("n_admm,n_dr", [(1, 1), (2, 3), (3, 8)])
def test_dr_iterates_parity_fp64(cases, name, n_admm, n_dr):
    inst = cases[name]
    lin, res, prob, out = _run(inst, n_admm, n_dr, r=0.5)
    assert out["iters"][0] == n_admm
    assert_close(out["K"][0], res.K, RTOL64, "K")
    assert_close(out["du"][0], res.du, RTOL64, "du")
    assert_close(out["p"][0], res.p, RTOL64, "p")
    assert_close(out["pt"][0], res.pt, RTOL64, "p~")
    assert_close(prob.export(nrto.F_LAMP, 0), res.lam, RTOL64, "lambda")
    assert_close(prob.export(nrto.F_DX, 0), res.dx, RTOL64, "dx")
    assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, res.dr_state.etat), RTOL64, "eta~")
    # r_p = ‖p - p̃‖ and r_d = ρ‖Δp‖ are differences of O(‖p‖) vectors that each carry a 1e-8
    # relative error, so their bound scales with those norms rather than with the residuals.
    scale = np.linalg.norm(res.p) + np.linalg.norm(res.pt)
    assert abs(out["r_p"][0] - res.r_p) <= RTOL64 * scale
    assert abs(out["r_d"][0] - res.r_d) <= RTOL64 * 40.0 * 2 * scale
    assert prob.export(nrto.F_STATS, 0)[5] == n_admm * n_dr
    prob.close()


@pytest.mark.parametrize("r", [0.05, 50.0])
def test_dr_trust_region_active_and_inactive(cases, r):
    """Subproblem 2 with the trust multiplier at work (r small) and without it (r large: the
    unconstrained ‖F_u δû‖ of this case is about 6.4)."""
    lin, res, prob, out = _run(cases["uni_T20_o3"], 2, 4, r=r)
    assert_close(out["du"][0], res.du, RTOL64, "du")
    assert_close(out["p"][0], res.p, RTOL64, "p")
    dxn = np.linalg.norm(prob.export(nrto.F_DX, 0)[cases["uni_T20_o3"].nx:])
    if r < 1:
        assert abs(dxn - r) <= 1e-9 * r
    else:
        assert dxn < r
    prob.close()


def test_dr_termination_counts_match_oracle(cases):
    """With the tolerances on, ADMM and DR iteration counts equal the oracle's."""
    inst = cases["uni_T20_o3"]
    lin = P.linearize(inst, inst.u_init)
    o = DRO.DROptions(rho=40.0, r_trust=2.0, eps_dr=1e-4, max_dr=500, eps_p=1e-4, eps_d=1e-4, max_admm=40)
    res = DRO.solve(inst, lin, o)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(2.0)
    out = prob.solve_socp(nrto.Options(solver=nrto.SOLVER_DR, rho=40.0, max_inner=40, max_dr=500, eps_dr=1e-4,
                                       eps_p=1e-4, eps_d=1e-4, check=1))
    st = prob.export(nrto.F_STATS, 0)
    assert out["iters"][0] == res.admm_iters
    assert st[5] == sum(res.dr_iters)
    assert out["status"][0] == (1 if res.converged else 2)
    assert_close(out["K"][0], res.K, 1e-7, "K at termination")
    assert_close(out["du"][0], res.du, 1e-7, "du at termination")
    prob.close()


def test_dr_batch_equals_single_instances(cases):
    insts = [cases["uni_T20_o3"], cases["quad_T16_o3"], cases["uni_T40_o6"]]
    g = _opts(2, 3, 0, 0.5)[1]
    batch = nrto.Problem(insts, nrto.PREC_FP64)
    batch.linearize()
    batch.set_trust_radius(0.5)
    ob = batch.solve_socp(g)
    for i, inst in enumerate(insts):
        single = nrto.Problem([inst], nrto.PREC_FP64)
        single.linearize()
        single.set_trust_radius(0.5)
        os_ = single.solve_socp(g)
        assert np.array_equal(ob["K"][i], os_["K"][0]) and np.array_equal(ob["du"][i], os_["du"][0])
        single.close()
    batch.close()


@pytest.mark.parametrize("name", ["uni_T40_o6", "quad_T16_o3"])
def test_dr_mixed_precision_error_bounds(cases, name):
    """Mixed mode (FP32 rows, cones and gain products; FP64 factorizations and subproblem 2) after
    3 ADMM × 8 DR iterations: error against the FP64 oracle within the FP32 rounding budget."""
    lin, res, prob, out = _run(cases[name], 3, 8, r=0.5, prec=nrto.PREC_MIXED)
    assert relerr(out["K"][0], res.K) < 5e-4
    assert relerr(out["du"][0], res.du) < 5e-5
    assert relerr(out["pt"][0], res.pt) < 5e-5
    prob.close()
