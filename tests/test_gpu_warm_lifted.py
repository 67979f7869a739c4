"""GPU parity of the lifted warm start (nrto_set_warm_start_lifted: K, p̃, λ_p plus the per-row
λ_ν factor θ, λ_w, δû, λ_e and the penalty) against oracle/fulladmm.warm_state_lifted in FP64,
its fixed-point property at a solution, and the network path's scatter against the host path."""
import numpy as np
import pytest

from oracle import fulladmm as F, problem as P
from paper_2603_02642_b300 import nrto, warmstart as WS, workloads as W

from .gpu_common import RTOL64, assert_close, ragged_from_dense

pytestmark = pytest.mark.gpu


def _solution(kind, eps=1e-8):
    inst = W.quadcopter(1, T=12, n_obs=3) if kind == "quad" else W.unicycle(2, T=20, n_obs=3)
    lin = P.linearize(inst, inst.u_init)
    o = F.FullADMMOptions(rho=10.0, r_trust=2.0, max_iter=20000, eps_p=eps, eps_d=eps, adapt_every=25)
    ref = F.iterate(inst, lin, o)
    assert ref.converged
    Y = P.Ahat_apply(lin, ref.K) + lin.bhat
    yy = np.sum(Y * Y, axis=(1, 2))
    theta = np.where(yy > 0, np.sum(ref.lam_nu * Y, axis=(1, 2)) / np.where(yy > 0, yy, 1.0), 0.0)
    return inst, lin, ref, np.maximum(theta, 0.0)


def _gpu(inst, ref, theta, theta_scale=1.0, du_scale=1.0):
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(2.0)
    prob.set_warm_start([ref.K], [ref.pt], [ref.lam_p])
    prob.set_warm_start_lifted([theta * theta_scale], [ref.lam_w], [ref.du * du_scale], [ref.lam_e], rho=ref.rho)
    return prob


@pytest.mark.parametrize("kind", ["quad", "uni"])
def test_lifted_warm_start_iterates_parity_fp64(kind):
    """Perturbed values (so that the iterates move): θ and δû scaled by 0.9, 5 iterations."""
    inst, lin, ref, theta = _solution(kind)
    o = F.FullADMMOptions(rho=10.0, r_trust=2.0, check=False)
    st = F.warm_state_lifted(lin, ref.K, ref.pt, ref.lam_p, 0.9 * theta, 0.9 * ref.du, ref.lam_w, ref.lam_e)
    s = F.iterate(inst, lin, o, st, n_iter=5, rho0=ref.rho)
    prob = _gpu(inst, ref, theta, 0.9, 0.9)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=5, check=0))
    assert out["iters"][0] == 5
    assert_close(out["K"][0], s.K, RTOL64, "K")
    assert_close(out["du"][0], s.du, RTOL64, "du")
    assert_close(out["p"][0], s.p, RTOL64, "p")
    assert_close(out["pt"][0], s.pt, RTOL64, "p~")
    assert_close(prob.export(nrto.F_LAMP, 0), s.lam_p, RTOL64, "lambda_p")
    assert_close(prob.export(nrto.F_LAMW, 0), s.lam_w, RTOL64, "lambda_w")
    assert_close(prob.export(nrto.F_LAME, 0)[inst.nx:], s.lam_e.reshape(-1), RTOL64, "lambda_e")
    assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, s.lam_nu), RTOL64, "lambda_nu")
    assert_close(prob.export(nrto.F_DX, 0), s.dx, RTOL64, "dx")
    assert prob.stats()["rho"][0] == ref.rho
    prob.close()


def test_lifted_warm_start_at_a_solution_converges_at_once():
    inst, lin, ref, theta = _solution("quad")
    o = F.FullADMMOptions(rho=10.0, r_trust=2.0, max_iter=20000, eps_p=1e-8, eps_d=1e-8, adapt_every=25)
    s = F.iterate(inst, lin, o, F.warm_state_lifted(lin, ref.K, ref.pt, ref.lam_p, theta, ref.du, ref.lam_w,
                                                    ref.lam_e), rho0=ref.rho)
    prob = _gpu(inst, ref, theta)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=20000, eps_p=1e-8, eps_d=1e-8, check=1, adapt_every=25))
    assert out["iters"][0] == s.iters <= 2 and out["status"][0] == 1
    assert_close(out["du"][0], ref.du, 1e-6, "du")
    # the next solve is cold again (the lifted start is consumed)
    out2 = prob.solve_socp(nrto.Options(rho=10.0, max_inner=20000, eps_p=1e-8, eps_d=1e-8, check=1, adapt_every=25))
    assert out2["iters"][0] > 10
    prob.close()


def test_lifted_warm_start_argument_and_state_checks():
    inst, lin, ref, theta = _solution("uni", eps=1e-4)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    with pytest.raises(nrto.NrtoError):      # needs the plain warm start first
        prob.set_warm_start_lifted([theta], [ref.lam_w], [ref.du], [ref.lam_e])
    prob.set_warm_start([ref.K], [ref.pt], [ref.lam_p])
    with pytest.raises(nrto.NrtoError):
        prob.set_warm_start_lifted([theta], [ref.lam_w], [ref.du], [ref.lam_e], rho=-1.0)
    prob.set_warm_start_lifted([theta], [ref.lam_w], [ref.du], [ref.lam_e])
    with pytest.raises(nrto.NrtoError):      # only the lifted FullADMM iteration takes it
        prob.solve_socp(nrto.Options(solver=nrto.SOLVER_DR, max_inner=2, check=0))
    prob.close()


def test_device_lifted_warm_start_equals_host_path():
    """nrto_set_warm_start_from_network_lifted installs exactly what predict + the two host calls do."""
    insts = [W.warmstart_quad(3_000_000 + s) for s in range(8)]
    ws = WS.WarmStart(max_batch=64, seed=4, lifted=True)
    ws.deployed = True          # untrained network: the mapping, not the values, is under test
    outs = []
    parts = ("th", "lw", "du", "le", "rho")
    for apply in (ws.apply, ws.apply_host):
        prob = nrto.Problem(insts, nrto.PREC_FP64)
        prob.linearize()
        apply(prob, insts, parts=parts)
        prob.solve_socp(nrto.Options(rho=10.0, max_inner=1, check=0))
        outs.append([(prob.export(nrto.F_K, i), prob.export(nrto.F_LAMW, i), prob.export(nrto.F_LAME, i),
                      prob.export(nrto.F_DU, i), prob.export(nrto.F_LAMNU, i), prob.stats()["rho"][i])
                     for i in range(len(insts))])
        prob.close()
    for a, b in zip(*outs):
        for x, y in zip(a, b):
            assert np.allclose(x, y, rtol=1e-12, atol=1e-13)
    ws.net.close()


def test_device_lifted_warm_start_with_absent_parts_equals_host_path():
    """The default lifted parts (δû only): the absent parts start at zero on both paths."""
    insts = [W.warmstart_quad(3_100_000 + s) for s in range(8)]
    ws = WS.WarmStart(max_batch=64, seed=5, lifted=True)
    ws.deployed = True
    outs = []
    for apply in (ws.apply, ws.apply_host):
        prob = nrto.Problem(insts, nrto.PREC_FP64)
        prob.linearize()
        apply(prob, insts)
        prob.solve_socp(nrto.Options(rho=10.0, max_inner=2, check=0))
        outs.append([(prob.export(nrto.F_K, i), prob.export(nrto.F_DU, i), prob.export(nrto.F_LAMNU, i),
                      prob.export(nrto.F_LAMW, i), prob.stats()["rho"][i]) for i in range(len(insts))])
        prob.close()
    for a, b in zip(*outs):
        for x, y in zip(a, b):
            assert np.allclose(x, y, rtol=1e-12, atol=1e-13)
    ws.net.close()
