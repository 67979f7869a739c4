"""GPU parity of the linearization prologue and the FullADMM inner loop against the oracle,
through the C ABI (libnrto.so).  FP64 mode: element-wise within 1e-8 relative at fixed
iteration counts; mixed mode: stated per-result bounds."""
import numpy as np
import pytest

from oracle import fulladmm as F, problem as P
from paper_2603_02642_b300 import nrto, workloads as W

from .gpu_common import RTOL64, assert_close, bvec_ragged, ragged_from_dense, relerr

pytestmark = pytest.mark.gpu

# Sizes: several solver chunks per instance (chunks hold ~8k row entries) and a ragged tail.
CASES = {
    "uni_T50_o4": lambda: W.unicycle(3, T=50, n_obs=4),
    "quad_T40_o5": lambda: W.quadcopter(4, T=40, n_obs=5),
    "arm_T12": lambda: W.arm(5, T=12),
}


def _lin_oracle(inst):
    return P.linearize(inst, inst.u_init)


@pytest.fixture(scope="module")
def cases():
    return {k: f() for k, f in CASES.items()}


@pytest.mark.parametrize("name", list(CASES))
def test_linearization_parity_fp64(cases, name):
    inst = cases[name]
    lin = _lin_oracle(inst)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    assert_close(prob.export(nrto.F_XHAT, 0), lin.x_hat, 1e-12, "x_hat")
    assert_close(prob.export(nrto.F_A, 0), lin.A, 1e-12, "A")
    assert_close(prob.export(nrto.F_B, 0), lin.B, 1e-12, "B")
    assert_close(prob.export(nrto.F_G0, 0), lin.g0, 1e-12, "g0")
    assert_close(prob.export(nrto.F_BHAT, 0), ragged_from_dense(lin, lin.bhat)[:prob.info[0].n_entries_state], 1e-10, "bhat")
    assert_close(prob.export(nrto.F_BVEC, 0), bvec_ragged(lin), 1e-10, "bvec")
    G = np.einsum("jmu,jmv->muv", lin.bvec, lin.bvec)
    assert_close(prob.export(nrto.F_GM, 0), G, 1e-10, "G_m")
    prob.close()


def _run_both(inst, n_iter, prec, rho=10.0, r=0.5):
    lin = _lin_oracle(inst)
    o = F.FullADMMOptions(rho=rho, r_trust=r, check=False)
    s = F.iterate(inst, lin, o, n_iter=n_iter)
    prob = nrto.Problem([inst], prec)
    prob.linearize()
    prob.set_trust_radius(r)
    out = prob.solve_socp(nrto.Options(rho=rho, max_inner=n_iter, check=0))
    return lin, s, prob, out


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("n_iter", [1, 2, 25])
def test_fulladmm_iterates_parity_fp64(cases, name, n_iter):
    inst = cases[name]
    lin, s, prob, out = _run_both(inst, n_iter, nrto.PREC_FP64)
    assert out["iters"][0] == n_iter
    assert_close(out["K"][0], s.K, RTOL64, "K")
    assert_close(out["du"][0], s.du, RTOL64, "du")
    assert_close(out["p"][0], s.p, RTOL64, "p")
    assert_close(out["pt"][0], s.pt, RTOL64, "p~")
    assert_close(prob.export(nrto.F_LAMP, 0), s.lam_p, RTOL64, "lambda_p")
    assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, s.lam_nu), RTOL64, "lambda_nu")
    assert_close(prob.export(nrto.F_DX, 0), s.dx, RTOL64, "dx")
    sc = prob.export(nrto.F_SCAL, 0)
    assert abs(sc[0] - s.r_p) <= RTOL64 * s.r_p and abs(sc[1] - s.r_d) <= RTOL64 * s.r_d
    assert abs(sc[2] - s.r_p_paper) <= RTOL64 * max(s.r_p_paper, 1e-300)
    prob.close()


def test_fulladmm_termination_matches_oracle():
    inst = W.unicycle(0)
    lin = _lin_oracle(inst)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=2.0, eps_p=1e-4, eps_d=1e-4, max_iter=2000))
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(2.0)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=2000, eps_p=1e-4, eps_d=1e-4, check=1))
    assert out["status"][0] == 1 and s.converged
    assert out["iters"][0] == s.iters
    assert_close(out["K"][0], s.K, 1e-7, "K at termination")
    assert_close(out["du"][0], s.du, 1e-7, "du at termination")
    prob.close()


def test_batch_equals_single_instances():
    """Instances are independent: a mixed batch gives the same iterates as solving each alone."""
    insts = [W.unicycle(7, T=30, n_obs=3), W.quadcopter(8, T=25, n_obs=2), W.unicycle(9, T=22, n_obs=5)]
    opts = nrto.Options(rho=10.0, max_inner=15, check=0)
    batch = nrto.Problem(insts, nrto.PREC_FP64)
    batch.linearize()
    ob = batch.solve_socp(opts)
    for i, inst in enumerate(insts):
        single = nrto.Problem([inst], nrto.PREC_FP64)
        single.linearize()
        os_ = single.solve_socp(opts)
        assert np.array_equal(ob["K"][i], os_["K"][0]) and np.array_equal(ob["du"][i], os_["du"][0])
        single.close()
    batch.close()


@pytest.mark.parametrize("name", ["uni_T50_o4", "quad_T40_o5"])
def test_mixed_precision_error_bounds(cases, name):
    """Mixed mode (FP32 rows, cones and gain products; FP64 factorizations) after 25 iterations:
    per-result error against the FP64 oracle stays within the FP32 rounding budget."""
    inst = cases[name]
    lin, s, prob, out = _run_both(inst, 25, nrto.PREC_MIXED)
    assert relerr(out["K"][0], s.K) < 5e-4
    assert relerr(out["du"][0], s.du) < 5e-5
    assert relerr(out["pt"][0], s.pt) < 5e-5
    prob.close()


@pytest.mark.parametrize("name", ["uni_T50_o4", "quad_T40_o5"])
def test_residual_balancing_iterates_parity_fp64(cases, name):
    """Iterates with ρ adapted every 5 iterations (starting far from balance) match the oracle's."""
    inst = cases[name]
    lin = _lin_oracle(inst)
    o = F.FullADMMOptions(rho=200.0, r_trust=0.5, check=False, adapt_every=5)
    s = F.iterate(inst, lin, o, n_iter=40)
    assert s.rho != 200.0
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(0.5)
    out = prob.solve_socp(nrto.Options(rho=200.0, max_inner=40, check=0, adapt_every=5))
    st = prob.export(nrto.F_STATS, 0)
    assert st[4] == s.rho
    assert_close(out["K"][0], s.K, RTOL64, "K")
    assert_close(out["du"][0], s.du, RTOL64, "du")
    assert_close(out["pt"][0], s.pt, RTOL64, "p~")
    assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, s.lam_nu), RTOL64, "lambda_nu")
    assert_close(prob.export(nrto.F_LAMP, 0), s.lam_p, RTOL64, "lambda_p")
    prob.close()


def test_stall_stop_matches_oracle():
    from .test_oracle_fulladmm import tiny_unicycle
    inst = tiny_unicycle()
    inst.obs_center = np.array([[0.5, 0.0]])
    inst.obs_radius = np.array([0.3])
    lin = _lin_oracle(inst)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=1.0, r_trust=0.01, max_iter=5000, stall_every=100))
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(0.01)
    out = prob.solve_socp(nrto.Options(rho=1.0, max_inner=5000, check=1, stall_every=100))
    assert s.stalled and out["status"][0] == 5 and out["iters"][0] == s.iters


def test_budget_stop_matches_oracle():
    """The budget stop (stall_budget) ends the solve at the same checkpoint as the oracle's, with
    status 5, on a case where the cap cannot reach the tolerance."""
    from .test_oracle_fulladmm import tiny_unicycle
    inst = tiny_unicycle()
    lin = _lin_oracle(inst)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=0.5, eps_p=1e-9, eps_d=1e-9, max_iter=600,
                                               stall_every=50, stall_budget=1.0))
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(0.5)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=600, check=1, eps_p=1e-9, eps_d=1e-9, stall_every=50,
                                       stall_budget=1.0))
    assert s.stalled and s.iters < 600
    assert out["status"][0] == 5 and out["iters"][0] == s.iters
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=600, check=1, eps_p=1e-9, eps_d=1e-9, stall_every=50))
    assert out["status"][0] == 2 and out["iters"][0] == 600
    prob.close()


def test_warm_start_iterates_parity_fp64(cases):
    """nrto_set_warm_start (k_v, p̃, λ_p; λ_ν = 0) then 25 iterations: same iterates as the oracle
    started from warm_state."""
    inst = cases["quad_T40_o5"]
    lin = _lin_oracle(inst)
    w = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=0.5, check=False), n_iter=7)
    o = F.FullADMMOptions(rho=10.0, r_trust=0.5, check=False)
    s = F.iterate(inst, lin, o, F.warm_state(lin, w.K, w.pt, w.lam_p), n_iter=25)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(0.5)
    prob.set_warm_start([w.K], [w.pt], [w.lam_p])
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=25, check=0))
    assert_close(out["K"][0], s.K, RTOL64, "K")
    assert_close(out["du"][0], s.du, RTOL64, "du")
    assert_close(out["pt"][0], s.pt, RTOL64, "p~")
    assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, s.lam_nu), RTOL64, "lambda_nu")
    prob.close()


def test_warm_start_fallback_matches_oracle():
    from .test_oracle_fulladmm import tiny_unicycle
    inst = tiny_unicycle()
    inst.obs_center = np.array([[0.5, 0.0]])
    inst.obs_radius = np.array([0.3])
    lin = _lin_oracle(inst)
    w = F.iterate(inst, lin, F.FullADMMOptions(rho=1.0, r_trust=0.01, check=False), n_iter=5)
    # residual balancing on: the cold rerun must start again from ρ = 1 with matching factors
    o = F.FullADMMOptions(rho=1.0, r_trust=0.01, max_iter=2000, stall_every=100, adapt_every=25)
    s, fell = F.solve_warm_with_fallback(inst, lin, o, w.K, w.pt, w.lam_p)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(0.01)
    prob.set_warm_start([w.K], [w.pt], [w.lam_p])
    out = prob.solve_socp(nrto.Options(rho=1.0, max_inner=2000, check=1, stall_every=100, adapt_every=25,
                                       warm_fallback=1))
    st = prob.export(nrto.F_STATS, 0)
    assert fell and st[6] == 1
    assert out["iters"][0] == s.iters
    # The linearization is infeasible on purpose (that is what makes the warm start stall), so the
    # iterates drift without bound and only the discrete outcome is compared.
    assert out["status"][0] == (5 if s.stalled else (1 if s.converged else 2))
    prob.close()
