"""Pins for the oracle's linearized robust data (Problem 2, Supplementary Sec. I)."""
import numpy as np
import pytest

from oracle import models, problem as P
from paper_2603_02642_b300 import workloads as W

RNG = np.random.default_rng(11)


def _tiny(kind="quad"):
    if kind == "quad":
        inst = W.quadcopter(2, T=5, n_obs=2)
    elif kind == "arm":
        inst = W.arm(2, T=4)
    else:
        inst = W.unicycle(2, T=6, n_obs=2)
    # Non-trivial, non-diagonal covariance blocks so that Ψ is a full triangle.
    for i in range(inst.T + 1):
        M = RNG.normal(size=(inst.nx, inst.nx)) * 0.01
        inst.Sigma[i] = inst.Sigma[i] + M @ M.T
    inst.tau = 0.7
    u = inst.u_init + 0.1 * RNG.normal(size=inst.u_init.shape)
    return inst, u


@pytest.mark.parametrize("kind", ["uni", "quad", "arm"])
def test_Fu_Fz_match_ltv_rollout(kind):
    inst, u = _tiny(kind)
    lin = P.linearize(inst, u)
    T, nx, nu = inst.T, inst.nx, inst.nu
    du = RNG.normal(size=(T, nu))
    zeta = RNG.normal(size=(T + 1, nx))
    K = RNG.normal(size=(T, nu, nx))
    # δx_{k+1} = A_k δx_k + B_k(δu_k + K_k ζ_k) + ζ_{k+1}, δx_0 = ζ_0 (policy u_k = ū_k + K_k d_{k-1}).
    dx = np.zeros((T + 1, nx))
    dx[0] = zeta[0]
    for k in range(T):
        dx[k + 1] = lin.A[k] @ dx[k] + lin.B[k] @ (du[k] + K[k] @ zeta[k]) + zeta[k + 1]
    Kbar = np.zeros((T * nu, (T + 1) * nx))
    for k in range(T):
        Kbar[k * nu:(k + 1) * nu, k * nx:(k + 1) * nx] = K[k]
    pred = lin.Fu @ du.reshape(-1) + (lin.Fz + lin.Fu @ Kbar) @ zeta.reshape(-1)
    assert np.allclose(pred, dx.reshape(-1), atol=1e-12)


def test_linearization_is_first_order_accurate():
    inst, u = _tiny("quad")
    lin = P.linearize(inst, u)
    du = RNG.normal(size=u.shape)
    errs = []
    for eps in [1e-2, 1e-3]:
        xn = models.rollout(inst, u + eps * du)
        errs.append(np.abs(xn - lin.x_hat - P.delta_x(lin, eps * du)).max())
    assert errs[1] < errs[0] / 50   # second-order remainder


@pytest.mark.parametrize("kind", ["uni", "quad", "arm"])
def test_robust_reformulation_worst_case(kind):
    """max_{zᵀSz ≤ τ} ∇gᵀ(F_ζ + F_u K̄) z = ‖Â_j k_v + b̂_j‖ (the SOC row of Problem 2):
    equality at the analytic maximizer, never exceeded on sampled boundary points."""
    inst, u = _tiny(kind)
    lin = P.linearize(inst, u)
    T, nx, nu = inst.T, inst.nx, inst.nu
    K = 0.5 * RNG.normal(size=(T, nu, nx))
    Kbar = np.zeros((T * nu, (T + 1) * nx))
    for k in range(T):
        Kbar[k * nu:(k + 1) * nu, k * nx:(k + 1) * nx] = K[k]
    Sinv = np.zeros(((T + 1) * nx, (T + 1) * nx))
    for i in range(T + 1):
        Sinv[i * nx:(i + 1) * nx, i * nx:(i + 1) * nx] = inst.Sigma[i]
    S = np.linalg.inv(Sinv)
    Y = P.Ahat_apply(lin, K) + lin.bhat
    st = models.state_rows(inst)
    ct = models.control_rows(inst)
    Lc = np.linalg.cholesky(Sinv)
    for j in range(lin.g0.shape[0]):
        if j < len(st):
            t = st[j][0]
            a = np.zeros((T + 1) * nx)
            a[t * nx:(t + 1) * nx] = models.g_state_grad(inst, st[j], lin.x_hat[t])
            c = (lin.Fz + lin.Fu @ Kbar).T @ a
        else:
            k, i, s = ct[j - len(st)]
            e = np.zeros(T * nu)
            e[k * nu + i] = s
            c = Kbar.T @ e
        val = np.linalg.norm(Y[j])
        if np.linalg.norm(c) < 1e-14:
            assert val < 1e-12
            continue
        zstar = inst.tau * Sinv @ c / np.sqrt(inst.tau * c @ Sinv @ c)
        assert np.isclose(zstar @ S @ zstar, inst.tau)
        assert np.isclose(c @ zstar, val, rtol=1e-10)
        w = RNG.normal(size=(500, c.shape[0]))
        w /= np.linalg.norm(w, axis=1, keepdims=True)
        zs = np.sqrt(inst.tau) * w @ Lc.T            # zᵀ S z = τ
        assert np.all(zs @ c <= val * (1 + 1e-12))


def test_fast_Ahat_matches_dense_definition_and_adjoint():
    inst, u = _tiny("quad")
    lin = P.linearize(inst, u)
    T, nx, nu = inst.T, inst.nx, inst.nu
    K = RNG.normal(size=(T, nu, nx))
    kv = P.kv_from_K(K)
    assert np.allclose(P.K_from_kv(kv, T, nu, nx), K)
    Y = P.Ahat_apply(lin, K)
    Wm = RNG.normal(size=Y.shape)
    AT = P.Ahat_T_apply(lin, Wm)
    total = np.zeros_like(kv)
    for j in range(lin.g0.shape[0]):
        Ad = P.dense_Ahat(lin, j)
        assert np.allclose(Ad @ kv, Y[j].reshape(-1), atol=1e-12)
        total += Ad.T @ Wm[j].reshape(-1)
    assert np.allclose(P.kv_from_K(AT), total, atol=1e-12)


def test_gain_hessian_is_block_diagonal_kronecker():
    inst, u = _tiny("uni")
    lin = P.linearize(inst, u)
    T, nx, nu = inst.T, inst.nx, inst.nu
    n = T * nu * nx
    dense = np.zeros((n, n))
    for j in range(lin.g0.shape[0]):
        Ad = P.dense_Ahat(lin, j)
        dense += Ad.T @ Ad
    rho, shift = 3.0, 0.25
    Qv = 2 * np.kron(np.eye(T * nx), np.diag(inst.RK ** 2))
    full = Qv + shift * np.eye(n) + rho * dense
    H = P.gain_hessian_blocks(lin, inst, coef=rho, shift=shift)
    blk = np.zeros_like(full)
    b = nu * nx
    for m in range(T):
        blk[m * b:(m + 1) * b, m * b:(m + 1) * b] = H[m]
    assert np.allclose(full, blk, atol=1e-12)
    # gain_solve is the inverse of that block-diagonal operator.
    R = RNG.normal(size=(T, nu, nx))
    X = P.gain_solve(H, R)
    assert np.allclose(full @ P.kv_from_K(X), P.kv_from_K(R), atol=1e-10)


def test_tau_zero_removes_robust_terms():
    inst, u = _tiny("uni")
    inst.tau = 0.0
    lin = P.linearize(inst, u)
    assert np.all(lin.bhat == 0)
    assert np.all(P.Ahat_apply(lin, RNG.normal(size=(inst.T, inst.nu, inst.nx))) == 0)


def test_row_support_is_blocks_zero_to_t():
    inst, u = _tiny("quad")
    lin = P.linearize(inst, u)
    n_state = lin.n_state
    for j in range(n_state):
        t = lin.row_t[j]
        assert np.all(lin.bhat[j, t + 1:] == 0) and np.all(lin.bvec[j, t:] == 0)
    for j in range(n_state, lin.g0.shape[0]):
        assert np.all(lin.bhat[j] == 0) and np.count_nonzero(lin.bvec[j]) == 1


def test_general_gamma_robust_term_with_singular_sigma():
    """General block-diagonal Γ: the disturbance of each step enters through Γ_i (n_x × n_w, here the
    quadcopter's three velocity states only), z_i ∈ {zᵀS_i z ≤ τ}.  With Σ_i = Γ_i S_i^{-1} Γ_iᵀ of rank
    3, the SOC row ‖Â_j k_v + b̂_j‖ still equals max over the ellipsoid of ∇gᵀ(F_ζ + F_u K̄) Γ z:
    attained at the analytic maximizer and never exceeded on sampled boundary points of the z-ellipsoid."""
    inst = W.quadcopter(3, T=5, n_obs=2)
    T, nx, nu = inst.T, inst.nx, inst.nu
    G = np.zeros((nx, 3))
    G[3:6, :] = np.eye(3)
    Sw = np.diag([1.0 / 4e-4, 1.0 / 1e-4, 1.0 / 9e-4])
    inst.Sigma = np.stack([G @ np.linalg.inv(Sw) @ G.T for _ in range(T + 1)])
    u = inst.u_init + 0.05 * RNG.normal(size=inst.u_init.shape)
    lin = P.linearize(inst, u)
    Psi = lin.Psi
    assert np.allclose(np.einsum("ikr,ikc->irc", Psi, Psi), inst.Sigma, atol=1e-14)
    K = 0.3 * RNG.normal(size=(T, nu, nx))
    Kbar = np.zeros((T * nu, (T + 1) * nx))
    for k in range(T):
        Kbar[k * nu:(k + 1) * nu, k * nx:(k + 1) * nx] = K[k]
    Gbig = np.kron(np.eye(T + 1), G)                       # ζ = Γ z
    Swi = np.kron(np.eye(T + 1), np.linalg.inv(Sw))        # S^{-1} of z
    Y = P.Ahat_apply(lin, K) + lin.bhat
    st = models.state_rows(inst)
    for j in range(len(st)):
        t = st[j][0]
        a = np.zeros((T + 1) * nx)
        a[t * nx:(t + 1) * nx] = models.g_state_grad(inst, st[j], lin.x_hat[t])
        c = Gbig.T @ (lin.Fz + lin.Fu @ Kbar).T @ a        # ∇gᵀ(F_ζ + F_u K̄) Γ
        val = np.linalg.norm(Y[j])
        zstar = inst.tau * Swi @ c / np.sqrt(inst.tau * c @ Swi @ c)
        assert np.isclose(c @ zstar, val, rtol=1e-10)
        w = RNG.normal(size=(500, c.shape[0]))
        w /= np.linalg.norm(w, axis=1, keepdims=True)
        zs = np.sqrt(inst.tau) * w @ np.linalg.cholesky(Swi).T
        assert np.all(zs @ c <= val * (1 + 1e-12))
