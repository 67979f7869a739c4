"""GPU parity at the sizes the benchmark runs, so that every thread mapping the solver kernel picks
there is executed against the oracle.  The FullADMM row pass splits a CTA's threads into row groups
by horizon: 512 / roundup32(⌈(T+1)/2⌉·n_x / W) groups, so a quadcopter takes two groups for
T < 84 and one from T = 84 on; the unicycle and the arm at their longest horizons run one group
with the most column pairs per thread.  FP64: iterates within 1e-8 relative (norm-wise and
element-wise) after 1, 2 and 25 iterations.  Mixed precision: per-result bounds after 25 and 200
iterations, and on instances of the 2048-instance batched workload solved together."""
import numpy as np
import pytest

from oracle import dr as DRO, fulladmm as F, problem as P
from paper_2603_02642_b300 import nrto, workloads as W

from .gpu_common import RTOL64, assert_close, ragged_from_dense, relerr

pytestmark = pytest.mark.gpu

CASES = {
    "quad_T60_o4": lambda: W.quadcopter(7, T=60, n_obs=4),       # two row groups
    "quad_T100_o3": lambda: W.quadcopter(8, T=100, n_obs=3),     # one row group
    "quad_T150_o2": lambda: W.quadcopter(9, T=150, n_obs=2),     # one row group, longest horizon
    "uni_T200_o15": lambda: W.unicycle(10, T=200, n_obs=15),     # entry-major pass, many rows per chunk
    "arm_T100": lambda: W.arm(11, T=100),                        # n_x = 14, one row group
}
COUNTS = (1, 2, 25)
R_TRUST = 0.5


@pytest.fixture(scope="module")
def oracle_runs():
    """Per case: linearization and the oracle iterates after each count (one continued run)."""
    out = {}
    for name, make in CASES.items():
        inst = make()
        lin = P.linearize(inst, inst.u_init)
        o = F.FullADMMOptions(rho=10.0, r_trust=R_TRUST, check=False)
        states, s, done = {}, None, 0
        for n in COUNTS:
            s = F.iterate(inst, lin, o, s, n_iter=n - done)
            done = n
            states[n] = s
        out[name] = (inst, lin, states)
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_fullsize_fulladmm_iterates_parity_fp64(oracle_runs, name):
    inst, lin, states = oracle_runs[name]
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(R_TRUST)
    for n in COUNTS:
        s = states[n]
        out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=n, check=0))
        assert out["iters"][0] == n
        what = f"{name} after {n}"
        assert_close(out["K"][0], s.K, RTOL64, f"K {what}")
        assert_close(out["du"][0], s.du, RTOL64, f"du {what}")
        assert_close(out["p"][0], s.p, RTOL64, f"p {what}")
        assert_close(out["pt"][0], s.pt, RTOL64, f"p~ {what}")
        assert_close(prob.export(nrto.F_LAMP, 0), s.lam_p, RTOL64, f"lambda_p {what}")
        assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, s.lam_nu), RTOL64, f"lambda_nu {what}")
        assert_close(prob.export(nrto.F_DX, 0), s.dx, RTOL64, f"dx {what}")
        sc = prob.export(nrto.F_SCAL, 0)
        assert abs(sc[0] - s.r_p) <= RTOL64 * s.r_p and abs(sc[1] - s.r_d) <= RTOL64 * s.r_d
    prob.close()


# Mixed precision (FP32 rows, cones and gain products; FP64 factorizations and residual sums):
# the bounds of the small cases, which follow from FP32 rounding of the S-length accumulations
# into Z' (relative 2^-24 · √S growth, S up to ~1e6 row entries: ~1e-4 on K before the Kronecker
# solve damps it) and hold at any iteration count because each ADMM step is non-expansive.
MIXED_BOUNDS = {"K": 5e-4, "du": 5e-5, "pt": 5e-5}


@pytest.mark.parametrize("name", ["quad_T100_o3", "uni_T200_o15"])
@pytest.mark.parametrize("n_iter", [25, 200])
def test_fullsize_mixed_precision_error_bounds(oracle_runs, name, n_iter):
    inst, lin, states = oracle_runs[name]
    s = states[25] if n_iter == 25 else F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=R_TRUST,
                                                                                check=False),
                                                  states[25], n_iter=n_iter - 25)
    prob = nrto.Problem([inst], nrto.PREC_MIXED)
    prob.linearize()
    prob.set_trust_radius(R_TRUST)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=n_iter, check=0))
    errs = {"K": relerr(out["K"][0], s.K), "du": relerr(out["du"][0], s.du), "pt": relerr(out["pt"][0], s.pt)}
    for k, b in MIXED_BOUNDS.items():
        assert errs[k] < b, f"{name} after {n_iter}: {k} relative error {errs[k]:.2e} >= {b:.0e}"
    prob.close()


def test_batched_workload_sample_mixed_precision():
    """Eight instances drawn (seeded) from the 2048-instance batched workload itself, solved as one
    batch in mixed precision, each within the mixed bounds of its own FP64 oracle run."""
    allw = W.batched_mix(2048, base_seed=10000)
    idx = sorted(np.random.default_rng(2024).choice(len(allw), size=8, replace=False).tolist())
    insts = [allw[i] for i in idx]
    prob = nrto.Problem(insts, nrto.PREC_MIXED)
    prob.linearize()
    prob.set_trust_radius(R_TRUST)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=25, check=0))
    for i, inst in enumerate(insts):
        lin = P.linearize(inst, inst.u_init)
        s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=R_TRUST, check=False), n_iter=25)
        for k, g, o in (("K", out["K"][i], s.K), ("du", out["du"][i], s.du), ("pt", out["pt"][i], s.pt)):
            e = relerr(g, o)
            assert e < MIXED_BOUNDS[k], f"instance {idx[i]} (kind {inst.kind}, T {inst.T}): {k} {e:.2e}"
    prob.close()


def test_fullsize_dr_iterates_parity_fp64():
    """NRTO-DR on a quadcopter past the one-row-group threshold (T = 90): 2 ADMM × 3 DR iterations."""
    inst = W.quadcopter(14, T=90, n_obs=2)
    lin = P.linearize(inst, inst.u_init)
    o = DRO.DROptions(rho=40.0, alpha=0.9, r_chi=1.0, sigma=1.0, r_trust=R_TRUST, max_admm=2, max_dr=3)
    res = DRO.solve(inst, lin, o, n_admm=2, n_dr=3, check=False)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(R_TRUST)
    out = prob.solve_socp(nrto.Options(solver=nrto.SOLVER_DR, rho=40.0, alpha=0.9, r_chi=1.0, sigma=1.0,
                                       max_inner=2, max_dr=3, check=0))
    assert out["iters"][0] == 2
    assert_close(out["K"][0], res.K, RTOL64, "K")
    assert_close(out["du"][0], res.du, RTOL64, "du")
    assert_close(out["pt"][0], res.pt, RTOL64, "p~")
    assert_close(prob.export(nrto.F_LAMP, 0), res.lam, RTOL64, "lambda")
    assert_close(prob.export(nrto.F_LAMNU, 0), ragged_from_dense(lin, res.dr_state.etat), RTOL64, "eta~")
    prob.close()
