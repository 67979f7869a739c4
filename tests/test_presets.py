"""The paper's settings as presets (Supplementary Sec. IV hyperparameter tables): each preset holds
the tables' values (the first of a listed set) and marshals into the C options struct."""
import pytest

from paper_2603_02642_b300 import nrto, presets


@pytest.mark.parametrize("system,solver,n_outer,r0,w_p,rho,iters", [
    ("unicycle", "fulladmm", 200, 1.5, 1.0, 10.0, 40),
    ("unicycle", "dr", 200, 1.5, 1.0, 40.0, 40),
    ("quadcopter", "fulladmm", 200, 1.5, 10.0, 10.0, 40),
    ("quadcopter", "dr", 200, 1.5, 10.0, 40.0, 40),
    ("franka", "fulladmm", 80, 2.0, 250.0, 10.0, 50),
])
def test_presets_hold_the_tables_values(system, solver, n_outer, r0, w_p, rho, iters):
    o, n = presets.paper_options(system, solver)
    assert n == n_outer and o.r0 == r0 and o.r_min == 1e-3 and o.w_p == w_p and o.rho == rho
    assert o.max_inner == iters and o.check == 1
    if solver == "fulladmm":
        assert o.solver == nrto.SOLVER_FULLADMM and o.eps_p == o.eps_d == 1e-3 and o.kv_pcg_iters == 100
        assert o.kv_pcg_tol == (0.01 if system == "unicycle" else 0.05)
    else:
        assert o.solver == nrto.SOLVER_DR and o.eps_dr == 1e-4 and o.max_dr == 100
    c = o.c()
    assert c.max_inner == iters and c.rho == rho


def test_unknown_preset_is_refused():
    with pytest.raises(KeyError):
        presets.paper_options("franka", "dr")
