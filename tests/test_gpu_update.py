"""nrto_problem_update on a resident batch: the host validates and packs the instances on several
threads, so a failure must still name the lowest failing instance, and an updated problem must solve
exactly like one created from the same data."""
import dataclasses

import numpy as np
import pytest

from paper_2603_02642_b300 import nrto, workloads as W

pytestmark = pytest.mark.gpu


def _batch(n, seed0):
    return [W.unicycle(seed0 + i, T=20, n_obs=3) for i in range(n)]


def test_update_reports_the_lowest_failing_instance():
    insts = _batch(300, 0)
    prob = nrto.Problem(insts, nrto.PREC_MIXED)
    bad = list(insts)
    for i in (250, 70, 181):
        u = bad[i].u_init.copy()
        u[3] = np.nan
        bad[i] = dataclasses.replace(bad[i], u_init=u)
    with pytest.raises(nrto.NrtoError) as e:
        prob.update(bad)
    assert "instance 70:" in str(e.value)
    prob.close()


def test_updated_problem_solves_like_a_fresh_one():
    a, b = _batch(200, 0), _batch(200, 1000)
    opts = nrto.Options(rho=10.0, max_inner=20, eps_p=1e-4, eps_d=1e-4, check=1, r0=2.0)
    fresh = nrto.Problem(b, nrto.PREC_FP64)
    ref = fresh.solve(opts, n_outer=2)
    fresh.close()
    prob = nrto.Problem(a, nrto.PREC_FP64)
    prob.solve(opts, n_outer=1)
    prob.update(b)
    out = prob.solve(opts, n_outer=2)
    for i in range(len(b)):
        np.testing.assert_array_equal(out["u_bar"][i], ref["u_bar"][i])
        np.testing.assert_array_equal(out["K"][i], ref["K"][i])
    np.testing.assert_array_equal(out["merit"], ref["merit"])
    prob.close()
