"""Pins of oracle/montecarlo.py (the Monte Carlo constraint-satisfaction check of Sec. V,
Methodology) against facts fixed outside it: the generator's published outputs, the moments of
the uniform distribution in a ball and of the standard normal, the boundary of the set, the
exactness of the robust reformulation for linear constraints, the undisturbed rollout, and the
first-order response of the linearized system."""
import math
import os

import numpy as np
import pytest

from oracle import models, montecarlo as MC, problem as P
from paper_2603_02642_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_matches_its_published_outputs():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.strip() and l[0] != "#"]
    got = [int(v) for v in MC.draws(0, np.arange(len(want)))]
    assert got == want
    # the scalar and the array forms of the output function agree
    assert [MC.mix64((MC.GAMMA * (n + 1)) & MC.MASK) for n in range(3)] == want


def test_box_muller_normals_have_standard_moments():
    g = MC.normals(MC.stream_key(7, 3, 11), 200000)
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.015
    # P(g ≤ 1) = Φ(1)
    assert abs(np.mean(g <= 1.0) - 0.5 * (1 + math.erf(1 / math.sqrt(2)))) < 0.004
    # odd and even members of a pair are uncorrelated
    assert abs(np.mean(g[0::2] * g[1::2])) < 0.01


def test_interior_samples_are_uniform_in_the_ball():
    """n = (T+1) n_x = 6: P(‖w‖ ≤ 1/2) = 2⁻⁶ and E[w wᵀ] = I/(n+2) for w uniform in the unit ball."""
    inst = W.unicycle(0, T=1, n_obs=1)
    N = 20000
    ws = np.stack([MC.whitened_sample(inst, None, None, 5, 0, s, N).reshape(-1) for s in range(N)])
    r = np.linalg.norm(ws, axis=1)
    assert np.all(r < 1.0)
    p = 2.0 ** -6
    assert abs(np.mean(r <= 0.5) - p) < 5 * math.sqrt(p * (1 - p) / N)
    C = ws.T @ ws / N
    assert np.allclose(C, np.eye(6) / 8.0, atol=0.006)
    assert np.all(np.abs(ws.mean(axis=0)) < 0.012)


def _inst_with_policy(kind, seed=3):
    rng = np.random.default_rng(seed)
    if kind == "uni":
        inst = W.unicycle(seed, T=6, n_obs=2)
    else:
        inst = W.quadcopter(seed, T=5, n_obs=2)
    for i in range(inst.T + 1):
        M = rng.normal(size=(inst.nx, inst.nx)) * 0.01
        inst.Sigma[i] = inst.Sigma[i] + M @ M.T
    inst.tau = 0.8
    u = inst.u_init + 0.05 * rng.normal(size=inst.u_init.shape)
    K = 0.3 * rng.normal(size=(inst.T, inst.nu, inst.nx))
    return inst, u, K


@pytest.mark.parametrize("kind", ["uni", "quad"])
def test_edge_samples_lie_on_the_boundary(kind):
    inst, u, K = _inst_with_policy(kind)
    lin = P.linearize(inst, u)
    Sinv = [np.linalg.inv(S) for S in inst.Sigma]
    for s in range(10, 22):
        w = MC.whitened_sample(inst, lin, K, 1, 2, s, 10)
        assert abs(np.linalg.norm(w) - 1.0) < 1e-12
        z = MC.disturbance(inst, w)
        q = sum(z[i] @ Sinv[i] @ z[i] for i in range(inst.T + 1))
        assert abs(q - inst.tau) < 1e-10 * inst.tau
    for s in range(10):   # interior samples stay inside
        z = MC.disturbance(inst, MC.whitened_sample(inst, lin, K, 1, 2, s, 10))
        assert sum(z[i] @ Sinv[i] @ z[i] for i in range(inst.T + 1)) < inst.tau


@pytest.mark.parametrize("kind", ["uni", "quad"])
def test_edge_sample_of_a_control_row_attains_its_robust_value(kind):
    """A control bound is linear in the disturbance, so the single-row edge sample of control
    row j drives that constraint to exactly g_j + ‖Â_j k + b̂_j‖ (the SOC row of Problem 2)."""
    inst, u, K = _inst_with_policy(kind)
    lin = P.linearize(inst, u)
    Y = MC.soc_rows(lin, K)
    ct = models.control_rows(inst)
    n_st, n_rows = lin.n_state, lin.g0.shape[0]
    hits = 0
    for e in range(0, 300, 3):   # n_c = 1
        key = MC.stream_key(4, 0, 10 + e)
        j = min(int(MC.uniforms(key, [0])[0] * n_rows), n_rows - 1)
        if j < n_st or np.linalg.norm(Y[j]) == 0.0:
            continue
        w = MC.whitened_sample(inst, lin, K, 4, 0, 10 + e, 10, Y)
        x, uu = MC.rollout(inst, u, K, MC.disturbance(inst, w))
        k, i, s = ct[j - n_st]
        val = uu[k, i] - inst.u_hi[i] if s > 0 else inst.u_lo[i] - uu[k, i]
        assert abs(val - (lin.g0[j] + np.linalg.norm(Y[j]))) < 1e-12 * max(1.0, abs(val))
        hits += 1
    assert hits >= 10


@pytest.mark.parametrize("kind", ["uni", "quad"])
def test_without_disturbance_every_sample_is_the_nominal(kind):
    inst, u, K = _inst_with_policy(kind)
    inst.tau = 0.0
    lin = P.linearize(inst, u)
    ok, worst = MC.check(inst, u, K, 9, 1, 4, 4)
    assert np.allclose(worst, lin.g0.max(), rtol=0, atol=1e-12)
    assert ok == (8 if lin.g0.max() <= 0 else 0)


@pytest.mark.parametrize("kind", ["uni", "quad"])
def test_small_disturbance_follows_the_linearized_system(kind):
    """x(ζ) - x̄ = F_ζ ζ + F_u vec(K_k ζ_k) + O(‖ζ‖²) (the linearized closed loop of problem.py)."""
    inst, u, K = _inst_with_policy(kind)
    lin = P.linearize(inst, u)
    w = MC.whitened_sample(inst, lin, K, 2, 0, 0, 1)
    errs = []
    for eps in (1e-3, 1e-4):
        z = eps * MC.disturbance(inst, w)
        x, _ = MC.rollout(inst, u, K, z)
        du = np.einsum("kuc,kc->ku", K, z[:inst.T])
        dx_lin = (lin.Fz @ z.reshape(-1) + lin.Fu @ du.reshape(-1)).reshape(x.shape)
        errs.append(np.linalg.norm(x - lin.x_hat - dx_lin) / np.linalg.norm(dx_lin))
    assert errs[1] < 2e-3
    assert errs[1] < 0.2 * errs[0]   # the remainder shrinks with ‖ζ‖


def test_check_counts_the_samples_within_tolerance():
    inst, u, K = _inst_with_policy("uni")
    ok, worst = MC.check(inst, u, K, 3, 0, 6, 6)
    assert worst.shape == (12,)
    assert ok == int(np.sum(worst <= 0.0))
    ok2, worst2 = MC.check(inst, u, K, 3, 0, 6, 6, tol=np.inf)
    assert ok2 == 12 and np.array_equal(worst, worst2)
