"""GPU parity of the Monte Carlo robust-constraint satisfaction check (nrto_monte_carlo; Sec. V,
Methodology) against oracle/montecarlo.py on the same seeded inputs: per-sample worst constraint
values (FP64, rounding-level agreement) and the satisfied-rollout counts, which are integers
decided by floating point: compared exactly except for samples whose worst value lies within the
comparison tolerance of the threshold."""
import numpy as np
import pytest

from oracle import fulladmm as F, montecarlo as MC, outer as O
from paper_2603_02642_b300 import nrto, workloads as W

pytestmark = pytest.mark.gpu

TOL_W = 1e-9


def _batch(seed=11):
    rng = np.random.default_rng(seed)
    insts = [W.unicycle(seed, T=12, n_obs=2), W.quadcopter(seed, T=10, n_obs=2), W.franka(seed, T=8)]
    us, Ks = [], []
    for inst in insts:
        for i in range(inst.T + 1):
            M = rng.normal(size=(inst.nx, inst.nx)) * 0.01
            inst.Sigma[i] = inst.Sigma[i] + M @ M.T
        inst.tau = 0.9
        us.append(inst.u_init + 0.05 * rng.normal(size=inst.u_init.shape))
        Ks.append(0.2 * rng.normal(size=(inst.T, inst.nu, inst.nx)))
    return insts, us, Ks


def _compare(gw, ow, gok, ook, tol=0.0, tw=TOL_W):
    diff = np.abs(gw - ow)
    assert np.all(diff <= tw * np.maximum(1.0, np.abs(ow))), (diff.max(), np.argmax(diff))
    near = int(np.sum(np.abs(ow - tol) <= tw * np.maximum(1.0, np.abs(ow))))
    assert abs(int(gok) - int(ook)) <= near


@pytest.mark.parametrize("n_int_edge", [(40, 40), (7, 23)])
def test_monte_carlo_parity_fp64(n_int_edge):
    n_int, n_edge = n_int_edge
    insts, us, Ks = _batch()
    prob = nrto.Problem(insts, nrto.PREC_FP64)
    prob.linearize(us)
    ok, worst = prob.monte_carlo(n_int, n_edge, seed=123, K=Ks, per_sample=True)
    for i, inst in enumerate(insts):
        ook, ow = MC.check(inst, us[i], Ks[i], 123, i, n_int, n_edge)
        _compare(worst[i], ow, ok[i], ook)
    # a threshold between the samples' values splits them the same way on both sides
    tol = float(np.median(worst[0]))
    ok2, _ = prob.monte_carlo(n_int, n_edge, seed=123, K=Ks, tol=tol, per_sample=True)
    ook2, ow0 = MC.check(insts[0], us[0], Ks[0], 123, 0, n_int, n_edge, tol=tol)
    _compare(worst[0], ow0, ok2[0], ook2, tol=tol)
    prob.close()


def test_monte_carlo_of_the_accepted_iterate_fp64():
    """After nrto_solve the check runs at the accepted nominal with the accepted gains: the oracle's
    own outer loop reaches the same iterate (to the solver's FP64 parity), so the samples agree."""
    inst = W.unicycle(1, T=12, n_obs=1)
    res = O.solve(inst, O.OuterOptions(n_outer=4, r0=2.0, r_min=1e-3, w_p=10.0),
                  admm=F.FullADMMOptions(rho=10.0, max_iter=300, eps_p=1e-4, eps_d=1e-4))
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.solve(nrto.Options(rho=10.0, max_inner=300, eps_p=1e-4, eps_d=1e-4, check=1, r0=2.0, r_min=1e-3,
                            w_p=10.0), n_outer=4)
    ok, worst = prob.monte_carlo(30, 30, seed=5, per_sample=True)
    ook, ow = MC.check(inst, res.u_bar, res.K, 5, 0, 30, 30)
    _compare(worst[0], ow, ok[0], ook, tw=1e-6)
    prob.close()


def test_monte_carlo_mixed_precision_within_bound():
    """The mixed-precision problem stores b̂ and b in FP32, which perturbs the edge directions only."""
    insts, us, Ks = _batch(seed=4)
    res = {}
    for prec in (nrto.PREC_FP64, nrto.PREC_MIXED):
        prob = nrto.Problem(insts, prec)
        prob.linearize(us)
        res[prec] = prob.monte_carlo(20, 20, seed=9, K=Ks, per_sample=True)
        prob.close()
    w64, wm = res[nrto.PREC_FP64][1], res[nrto.PREC_MIXED][1]
    # interior samples use no stored row data
    assert np.allclose(w64[:, :20], wm[:, :20], rtol=1e-12, atol=1e-14)
    assert np.all(np.abs(w64 - wm) <= 1e-4 * np.maximum(1.0, np.abs(w64)))


def test_monte_carlo_argument_checks():
    insts, us, Ks = _batch()
    prob = nrto.Problem(insts[:1], nrto.PREC_FP64)
    with pytest.raises(nrto.NrtoError):
        prob.monte_carlo(4, 4)                  # no linearization yet
    prob.linearize(us[:1])
    with pytest.raises(nrto.NrtoError):
        prob.monte_carlo(-1, 4)
    ok = prob.monte_carlo(0, 0)
    assert ok[0] == 0
    prob.close()


def test_monte_carlo_parity_at_workload_sizes_fp64():
    """The largest horizons of the batched workload (unicycle T = 200 with 20 obstacles, quadcopter
    T = 150 with 15), seeded nominal and gains given to both sides: the per-sample worst values of
    interior and edge samples at 1e-9."""
    rng = np.random.default_rng(21)
    insts = [W.unicycle(5, T=200, n_obs=20), W.quadcopter(6, T=150, n_obs=15)]
    us = [x.u_init + 0.02 * rng.normal(size=x.u_init.shape) for x in insts]
    Ks = [0.05 * rng.normal(size=(x.T, x.nu, x.nx)) for x in insts]
    prob = nrto.Problem(insts, nrto.PREC_FP64)
    prob.linearize(us)
    ok, worst = prob.monte_carlo(4, 5, seed=77, K=Ks, per_sample=True)
    for i, inst in enumerate(insts):
        ook, ow = MC.check(inst, us[i], Ks[i], 77, i, 4, 5)
        _compare(worst[i], ow, ok[i], ook)
    prob.close()
