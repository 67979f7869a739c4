"""GPU parity with a general block-diagonal Γ: the disturbance of step i enters through Γ_i of lower
rank, Σ_i = Γ_i S_i^{-1} Γ_iᵀ is singular and Ψ_i = Λ^{1/2}Vᵀ.  Ψ_i is unique only up to an orthogonal
factor (the library's and the oracle's eigensolvers may pick different eigenvector bases), and the
method's gains, controls, p, p̃ and residuals are invariant to that factor (the cone projection is
rotation-equivariant), so those are compared, with the per-row norms of b̂."""
import numpy as np
import pytest

from oracle import fulladmm as F, problem as P
from paper_2603_02642_b300 import nrto, workloads as W

from .gpu_common import RTOL64, assert_close

pytestmark = pytest.mark.gpu


def _uni():
    inst = W.unicycle(0, T=20, n_obs=3)
    inst.Sigma = np.stack([np.diag([0.02 ** 2, 0.02 ** 2, 0.0])] * (inst.T + 1))   # no heading disturbance
    return inst


def _quad():
    inst = W.quadcopter(5, T=16, n_obs=2)
    G = np.zeros((12, 3))
    G[3:6, :] = np.eye(3)                                # wind on the velocities only
    Sinv = np.diag([4e-4, 1e-4, 9e-4])
    inst.Sigma = np.stack([G @ Sinv @ G.T] * (inst.T + 1))
    return inst


@pytest.mark.parametrize("make", [_uni, _quad])
@pytest.mark.parametrize("n_iter", [1, 2, 25])
def test_singular_sigma_iterates_parity_fp64(make, n_iter):
    inst = make()
    lin = P.linearize(inst, inst.u_init)
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=0.5, check=False), n_iter=n_iter)
    prob = nrto.Problem([inst], nrto.PREC_FP64)
    prob.linearize()
    prob.set_trust_radius(0.5)
    out = prob.solve_socp(nrto.Options(rho=10.0, max_inner=n_iter, check=0))
    assert_close(out["K"][0], s.K, RTOL64, "K")
    assert_close(out["du"][0], s.du, RTOL64, "du")
    assert_close(out["p"][0], s.p, RTOL64, "p")
    assert_close(out["pt"][0], s.pt, RTOL64, "p~")
    sc = prob.export(nrto.F_SCAL, 0)
    assert abs(sc[0] - s.r_p) <= RTOL64 * s.r_p and abs(sc[1] - s.r_d) <= RTOL64 * s.r_d
    # per-row norms of b̂ (invariant to the orthogonal factor of Ψ_i)
    bh = prob.export(nrto.F_BHAT, 0)
    norms, o = [], 0
    for j in range(lin.n_state):
        n = (int(lin.row_t[j]) + 1) * inst.nx
        norms.append(np.linalg.norm(bh[o:o + n]))
        o += n
    assert_close(np.array(norms), np.linalg.norm(lin.bhat[:lin.n_state].reshape(lin.n_state, -1), axis=1), 1e-10,
                 "row norms of b-hat")
    prob.close()
