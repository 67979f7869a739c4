"""The paper's solver settings as named presets (Supplementary Sec. IV, the hyperparameter tables of
the unicycle, quadcopter and Franka experiments).

`paper_options(system, solver)` returns `(Options, n_outer)` for system "unicycle", "quadcopter" or
"franka" and solver "fulladmm" or "dr" (the Franka table covers FullADMM only).  Where a table lists
a set of values for one setting, the preset takes the first one listed.  Settings of the tables
that have no counterpart in the library's options are named in `OMITTED` and left at the library's
defaults: the outer loop's acceptance constants (η₁, η₂), its termination thresholds (ε_u, ε_p) and
c_ε, and the penalty ceiling ρ_max of the NRTO ADMM.  The library's outer loop runs a fixed number of
steps with the trust-radius schedule min(β r, r₀) on acceptance and max(α r, r_min) on rejection,
(α, β) = (0.8, 1.5) fixed: the quadcopter and Franka tables' values, and one of the pairs the unicycle
table lists.  The penalty ρ₀ = 40 of the outer-loop tables is the NRTO-DR ADMM penalty (the
quadcopter's NRTO-DR row names none; NRTO's is taken); FullADMM runs its own ρ = 10 from the solver
tables.  The FullADMM tables give one threshold ε_p; the presets apply it to
both the primal and the dual residual.
"""
from __future__ import annotations

from . import nrto

OMITTED = ("acceptance eta1, eta2", "outer termination eps_u, eps_p", "c_eps", "ADMM penalty ceiling rho_max",
           "trust-radius factors alpha, beta (fixed at 0.8, 1.5)")

# (system, solver) -> settings of the tables, in the tables' names
_TABLES = {
    ("unicycle", "fulladmm"): dict(n_outer=200, r0=1.5, r_min=1e-3, w_p=1.0, rho=10.0, iters=40, eps=1e-3,
                                   pcg_iters=100, pcg_tol=0.01),
    ("unicycle", "dr"): dict(n_outer=200, r0=1.5, r_min=1e-3, w_p=1.0, rho=40.0, iters=40, dr_eps=1e-4,
                             dr_iters=100),
    ("quadcopter", "fulladmm"): dict(n_outer=200, r0=1.5, r_min=1e-3, w_p=10.0, rho=10.0, iters=40, eps=1e-3,
                                     pcg_iters=100, pcg_tol=0.05),
    ("quadcopter", "dr"): dict(n_outer=200, r0=1.5, r_min=1e-3, w_p=10.0, rho=40.0, iters=40, dr_eps=1e-4,
                               dr_iters=100),
    ("franka", "fulladmm"): dict(n_outer=80, r0=2.0, r_min=1e-3, w_p=250.0, rho=10.0, iters=50, eps=1e-3,
                                 pcg_iters=100, pcg_tol=0.05),
}

SYSTEMS = sorted({s for s, _ in _TABLES})


def paper_options(system: str, solver: str = "fulladmm"):
    """(Options, n_outer) with the paper's settings for `system` and `solver`; KeyError otherwise."""
    t = _TABLES[(system, solver)]
    o = nrto.Options(r0=t["r0"], r_min=t["r_min"], w_p=t["w_p"], rho=t["rho"], max_inner=t["iters"], check=1)
    if solver == "fulladmm":
        o.solver = nrto.SOLVER_FULLADMM
        o.eps_p = o.eps_d = t["eps"]
        o.kv_pcg_iters, o.kv_pcg_tol = t["pcg_iters"], t["pcg_tol"]
    else:
        o.solver = nrto.SOLVER_DR
        o.eps_dr, o.max_dr = t["dr_eps"], t["dr_iters"]
    return o, t["n_outer"]
