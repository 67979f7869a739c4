"""GPU parity of the paper's Franka model (Supplementary Sec. IV-A: damping, unit inertia, velocity
and position limits clamped after each Euler step, torque bounds; the Panda's published kinematics)
against the oracle in FP64: the linearization, FullADMM iterates and the outer loop, on nominal
trajectories that drive joints into their clamped limits."""
import numpy as np
import pytest

from oracle import fulladmm as F, models, outer as O, problem as P
from paper_2603_02642_b300 import nrto, workloads as W

from .gpu_common import RTOL64, assert_close, bvec_ragged, ragged_from_dense

pytestmark = pytest.mark.gpu


def _franka(seed, T):
    inst = W.franka(seed, T=T)
    # a nominal that saturates: joint 1 torqued to its velocity limit within two steps, joint 4
    # driven towards its position limit
    u = np.zeros((T, 7))
    u[: T // 2, 0] = 80.0
    u[: T // 3, 3] = 60.0
    inst.u_init = u
    return inst


@pytest.mark.parametrize("seed,T", [(3, 12), (4, 60)])
def test_franka_linearization_parity_fp64(seed, T):
    inst = _franka(seed, T)
    lin = P.linearize(inst, inst.u_init)
    # the clamp is active on the nominal (otherwise the test would not exercise it)
    assert np.any(np.abs(lin.x_hat[:, 7:]) >= inst.x_hi[7:] - 1e-12)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    assert_close(prob.export(nrto.F_XHAT, 0), lin.x_hat, 1e-12, "x_hat")
    assert_close(prob.export(nrto.F_A, 0), lin.A, 1e-12, "A")
    assert_close(prob.export(nrto.F_B, 0), lin.B, 1e-12, "B")
    assert_close(prob.export(nrto.F_G0, 0), lin.g0, 1e-12, "g0")
    assert_close(prob.export(nrto.F_BHAT, 0), ragged_from_dense(lin, lin.bhat)[:prob.info[0].n_entries_state], 1e-10,
                 "bhat")
    assert_close(prob.export(nrto.F_BVEC, 0), bvec_ragged(lin), 1e-10, "bvec")
    prob.close()


@pytest.mark.parametrize("n_iter", [1, 2, 25])
def test_franka_fulladmm_iterates_parity_fp64(n_iter):
    inst = _franka(5, 20)
    lin = P.linearize(inst, inst.u_init)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=0.5, check=False), n_iter=n_iter)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(0.5)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=n_iter, check=0))
    assert_close(out["K"][0], s.K, RTOL64, "K")
    assert_close(out["du"][0], s.du, RTOL64, "du")
    assert_close(out["pt"][0], s.pt, RTOL64, "p~")
    assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, s.lam_nu), RTOL64, "lambda_nu")
    prob.close()


def test_franka_outer_loop_parity_fp64():
    inst = _franka(6, 16)
    res = O.solve(inst, O.OuterOptions(n_outer=4, r0=2.0, r_min=1e-3, w_p=10.0, carry=True),
                  admm=F.FullADMMOptions(rho=10.0, max_iter=60, eps_p=1e-4, eps_d=1e-4, adapt_every=10))
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    out = prob.solve(nrto.Options(rho=10.0, max_inner=60, eps_p=1e-4, eps_d=1e-4, check=1, r0=2.0, r_min=1e-3,
                                  w_p=10.0, adapt_every=10, carry=1), n_outer=4)
    st = prob.stats()
    assert st["n_accepted"][0] == sum(res.accepted)
    assert_close(out["u_bar"][0], res.u_bar, RTOL64, "u_bar")
    assert_close(out["K"][0], res.K, RTOL64, "K")
    assert abs(out["merit"][0] - res.phi) <= RTOL64 * abs(res.phi)
    prob.close()


def test_franka_mixed_precision_bounds():
    inst = _franka(7, 40)
    lin = P.linearize(inst, inst.u_init)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=0.5, check=False), n_iter=25)
    prob = nrto.Problem([inst], nrto.PREC_MIXED)
    prob.linearize()
    prob.set_trust_radius(0.5)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=25, check=0))
    from .gpu_common import relerr
    assert relerr(out["K"][0], s.K) < 5e-4 and relerr(out["du"][0], s.du) < 5e-5 and relerr(out["pt"][0], s.pt) < 5e-5
    prob.close()
