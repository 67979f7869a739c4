"""The device-side watchdog of the solver kernels, exercised without a fault: the bounded wait that
guards every bulk copy gives up on a barrier that nothing completes, reports status 4 once its cycle
limit has passed, and the device stays usable (a solve afterwards still matches the oracle)."""
import pytest

from oracle import fulladmm as F, problem as P
from paper_2603_02642_b300 import nrto, workloads as W

from .gpu_common import RTOL64, assert_close

pytestmark = pytest.mark.gpu

WAIT_LIMIT_CYCLES = 1 << 32   # the solver kernels' bound on a copy wait


def test_bounded_wait_gives_up_and_device_stays_usable():
    status, cycles = nrto.selftest_bounded_wait()
    assert status == 4
    assert WAIT_LIMIT_CYCLES < cycles < 2 * WAIT_LIMIT_CYCLES   # gave up at its limit, not before or long after
    inst = W.unicycle(3, T=12, n_obs=2)
    lin = P.linearize(inst, inst.u_init)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=0.5, check=False), n_iter=5)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(0.5)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=5, check=0))
    assert out["iters"][0] == 5
    assert_close(out["K"][0], s.K, RTOL64, "K")
    assert_close(out["du"][0], s.du, RTOL64, "du")
    prob.close()
