"""Linearized robust problem data (oracle; test infrastructure only).

Follows Problem 2 ("Tractable Linearized Problem", Sec. II-B) and Supplementary Sec. I:
  b_j   = F_uᵀ ∇_x g_j(x̂)                             (Supplementary Sec. I, def. of b_j)
  Ā_j   = blkdiag(I_{nx} ⊗ b_{j,k}ᵀ)                     (same section)
  Â_j   = √τ Ψ Γᵀ [Ā_j; 0],  b̂_j = √τ Ψ Γᵀ F_ζᵀ ∇_x g_j(x̂),  ΨᵀΨ = S^{-1}
with Γ = I.  F_u and F_ζ are formed densely from their definition as the maps from
δû and ζ to the stacked state deviation of the linearized system
  δx_{k+1} = A_k δx_k + B_k (δu_k + K_k ζ_k) + ζ_{k+1},  δx_0 = ζ_0
(ζ-block 0 = d̄_0, ζ-block i+1 = d_i, and u_k = ū_k + K_k d_{k-1} with d_{-1} = d̄_0;
Problem 1 and the affine policy of Sec. II-A).

Row layout: every robust constraint j is one row; arrays are dense over the full
ζ dimension n_z = (T+1) nx (zero outside a row's support).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import models


@dataclass
class Linearization:
    x_hat: np.ndarray      # (T+1, nx) nominal rollout
    u_hat: np.ndarray      # (T, nu)
    A: np.ndarray          # (T, nx, nx)
    B: np.ndarray          # (T, nx, nu)
    Fu: np.ndarray         # ((T+1) nx, T nu)
    Fz: np.ndarray         # ((T+1) nx, (T+1) nx)
    Psi: np.ndarray        # (T+1, nx, nx), Ψ_i with Ψ_iᵀΨ_i = Σ_i
    g0: np.ndarray         # (n_g,) g_j at the nominal (control rows: ±û - bound)
    bvec: np.ndarray       # (n_g, T, nu)    b_{j,k}
    bhat: np.ndarray       # (n_g, T+1, nx)  b̂_j split in ζ-blocks
    n_state: int           # rows [0, n_state) are state rows, the rest control rows
    row_t: np.ndarray      # time index of a state row / step index of a control row
    sqrt_tau: float


def psi_blocks(Sigma):
    """Ψ_i with Ψ_iᵀΨ_i = Σ_i, so ΨᵀΨ = blkdiag(Σ_i) (Supplementary Sec. I: Ψ with ΨᵀΨ = S^{-1},
    for Γ = I).  Σ_i ≻ 0: Ψ_i = L_iᵀ with L_i L_iᵀ = Σ_i (Cholesky).  With a general block-diagonal
    Γ = blkdiag(Γ_i) (the disturbance of step i enters through Γ_i: ζ_i = Γ_i z_i, zᵀSz ≤ τ), the
    robust term is ‖Ψ Γᵀ c‖ with (ΨΓᵀ)ᵀ(ΨΓᵀ) = Γ S^{-1} Γᵀ = blkdiag(Γ_i S_i^{-1} Γ_iᵀ), so the same
    construction applies to Σ_i = Γ_i S_i^{-1} Γ_iᵀ, which is only positive semidefinite when Γ_i has
    fewer columns than rows; then Ψ_i = Λ_i^{1/2} V_iᵀ from Σ_i = V_i Λ_i V_iᵀ (negative rounding
    residue of zero eigenvalues taken as zero)."""
    out = []
    for S in Sigma:
        try:
            out.append(np.linalg.cholesky(S).T)
        except np.linalg.LinAlgError:
            lam, V = np.linalg.eigh(S)
            out.append(np.sqrt(np.maximum(lam, 0.0))[:, None] * V.T)
    return np.stack(out)


def transition(A, t, m):
    """Φ(t, m) = A_{t-1} ⋯ A_m (identity when t = m)."""
    nx = A.shape[1]
    P = np.eye(nx)
    for i in range(m, t):
        P = A[i] @ P
    return P


def dense_Fu_Fz(A, B):
    """F_u: block (t, i) = Φ(t, i+1) B_i for i < t; F_ζ: block (t, m) = Φ(t, m) for m ≤ t."""
    T, nx, nu = B.shape
    Fu = np.zeros(((T + 1) * nx, T * nu))
    Fz = np.zeros(((T + 1) * nx, (T + 1) * nx))
    for t in range(T + 1):
        for i in range(t):
            Fu[t * nx:(t + 1) * nx, i * nu:(i + 1) * nu] = transition(A, t, i + 1) @ B[i]
        for m in range(t + 1):
            Fz[t * nx:(t + 1) * nx, m * nx:(m + 1) * nx] = transition(A, t, m)
    return Fu, Fz


def linearize(inst, u_hat) -> Linearization:
    """Linearize Problem 1 at the nominal û (outer-loop step of Fig. 1 / Problem 2)."""
    T, nx, nu = inst.T, inst.nx, inst.nu
    x_hat = models.rollout(inst, u_hat)
    A = np.zeros((T, nx, nx))
    B = np.zeros((T, nx, nu))
    for k in range(T):
        A[k], B[k] = models.jacobians(inst, x_hat[k], u_hat[k])
    Fu, Fz = dense_Fu_Fz(A, B)
    Psi = psi_blocks(inst.Sigma)
    st = models.state_rows(inst)
    ct = models.control_rows(inst)
    n_g = len(st) + len(ct)
    g0 = np.zeros(n_g)
    bvec = np.zeros((n_g, T, nu))
    bhat = np.zeros((n_g, T + 1, nx))
    row_t = np.zeros(n_g, dtype=np.int64)
    sq = np.sqrt(inst.tau)
    Psi_big = np.zeros(((T + 1) * nx, (T + 1) * nx))
    for i in range(T + 1):
        Psi_big[i * nx:(i + 1) * nx, i * nx:(i + 1) * nx] = Psi[i]
    for j, row in enumerate(st):
        t = row[0]
        g0[j] = models.g_state(inst, row, x_hat[t])
        a_full = np.zeros((T + 1) * nx)
        a_full[t * nx:(t + 1) * nx] = models.g_state_grad(inst, row, x_hat[t])
        bvec[j] = (Fu.T @ a_full).reshape(T, nu)
        bhat[j] = (sq * Psi_big @ (Fz.T @ a_full)).reshape(T + 1, nx)
        row_t[j] = t
    for jj, (k, i, s) in enumerate(ct):
        j = len(st) + jj
        g0[j] = (u_hat[k, i] - inst.u_hi[i]) if s > 0 else (inst.u_lo[i] - u_hat[k, i])
        bvec[j, k, i] = s
        row_t[j] = k
    return Linearization(x_hat=x_hat, u_hat=np.array(u_hat, dtype=np.float64), A=A, B=B,
                         Fu=Fu, Fz=Fz, Psi=Psi, g0=g0, bvec=bvec, bhat=bhat,
                         n_state=len(st), row_t=row_t, sqrt_tau=sq)


# ---------------------------------------------------------------------------------------
# Operators on the gain variable k_v = [vec K_0; ...; vec K_{T-1}] (column-wise vec)
# ---------------------------------------------------------------------------------------

def kv_from_K(K):
    """k_v from K (T, nu, nx) with column-wise vec (Supplementary Sec. I)."""
    return np.concatenate([Kk.flatten(order="F") for Kk in K])


def K_from_kv(kv, T, nu, nx):
    return np.stack([kv[k * nu * nx:(k + 1) * nu * nx].reshape((nu, nx), order="F") for k in range(T)])


def Ahat_apply(lin, K):
    """Â_j k_v for every row j: block m (< T) is √τ Ψ_m K_mᵀ b_{j,m}
    (using K_kᵀ b_{j,k} = (I ⊗ b_{j,k}ᵀ) vec K_k), block T is 0. Returns (n_g, T+1, nx)."""
    n_g, T, nu = lin.bvec.shape
    nx = lin.Psi.shape[1]
    out = np.zeros((n_g, T + 1, nx))
    KtB = np.einsum("mux,jmu->jmx", K, lin.bvec)            # K_mᵀ b_{j,m}
    out[:, :T, :] = lin.sqrt_tau * np.einsum("mab,jmb->jma", lin.Psi[:T], KtB)
    return out


def Ahat_T_apply(lin, W):
    """Σ_j Â_jᵀ W_j as a gain-shaped array (T, nu, nx): block m of Â_jᵀ w is
    √τ (I ⊗ b_{j,m}) Ψ_mᵀ w_m = √τ vec(b_{j,m} (Ψ_mᵀ w_m)ᵀ)."""
    n_g, T, nu = lin.bvec.shape
    PtW = np.einsum("mba,jmb->jma", lin.Psi[:T], W[:, :T, :])  # Ψ_mᵀ w_{j,m}
    return lin.sqrt_tau * np.einsum("jmu,jmx->mux", lin.bvec, PtW)


def dense_Ahat(lin, j):
    """The paper's dense Â_j = √τ Ψ [Ā_j; 0] with Ā_j = blkdiag(I ⊗ b_{j,k}ᵀ), used only by
    tests on tiny horizons."""
    n_g, T, nu = lin.bvec.shape
    nx = lin.Psi.shape[1]
    Abar = np.zeros(((T + 1) * nx, T * nu * nx))
    for k in range(T):
        Abar[k * nx:(k + 1) * nx, k * nu * nx:(k + 1) * nu * nx] = np.kron(np.eye(nx), lin.bvec[j, k][None, :])
    Psi_big = np.zeros(((T + 1) * nx, (T + 1) * nx))
    for i in range(T + 1):
        Psi_big[i * nx:(i + 1) * nx, i * nx:(i + 1) * nx] = lin.Psi[i]
    return lin.sqrt_tau * Psi_big @ Abar


def gain_hessian_blocks(lin, inst, coef, shift=0.0):
    """Diagonal blocks of Q_v + shift·I + coef·Σ_j Â_jᵀ Â_j, one (nu nx)² block per step.

    Q_v = 2 blkdiag(I ⊗ R_KᵀR_K) (Supplementary Sec. I).  Because Â_j only couples ζ-block
    m with K_m, Σ_j Â_jᵀÂ_j is block diagonal, and its block m equals
    τ Σ_m ⊗ Σ_j b_{j,m} b_{j,m}ᵀ (from (I⊗b)Ψ_mᵀΨ_m(I⊗bᵀ) = Σ_m ⊗ b bᵀ); the tests check
    both facts against the dense Â_j of `dense_Ahat`."""
    T, nu = lin.bvec.shape[1], lin.bvec.shape[2]
    nx = lin.Psi.shape[1]
    W = np.diag(inst.RK ** 2)
    H = np.zeros((T, nu * nx, nu * nx))
    for m in range(T):
        G = lin.bvec[:, m, :].T @ lin.bvec[:, m, :]
        Sig = lin.Psi[m].T @ lin.Psi[m]
        H[m] = 2.0 * np.kron(np.eye(nx), W) + shift * np.eye(nu * nx) + coef * inst.tau * np.kron(Sig, G)
    return H


def gain_solve_pcg(lin, inst, coef, R, X0, tol, max_iter):
    """Matrix-free preconditioned conjugate gradients for (Q_v + coef·Σ_j Â_jᵀÂ_j) k = r, the k_v
    system of the FullADMM gain update solved iteratively as in Sec. IV ("GPU Implementation": the
    k_v update by PCG; Supplementary Tables VI-VIII: iteration cap and tolerance).  The operator is
    applied per step without forming it, (H X)_m = 2 R_KᵀR_K X_m + coef τ G_m X_m Σ_m with
    G_m = Σ_j b_{j,m} b_{j,m}ᵀ; the preconditioner is its diagonal (Jacobi),
    2 (R_K)_u² + coef τ (G_m)_uu (Σ_m)_cc.  Starts from X0 and stops before an iteration when
    ‖r - H x‖ ≤ tol ‖r‖, or after max_iter iterations.  Returns (X, iterations)."""
    T, nu = lin.bvec.shape[1], lin.bvec.shape[2]
    nx = lin.Psi.shape[1]
    W = inst.RK ** 2
    G = np.einsum("jmu,jmv->muv", lin.bvec, lin.bvec)
    Sig = np.einsum("mka,mkb->mab", lin.Psi[:T], lin.Psi[:T])
    ct = coef * inst.tau

    def apply(X):
        return 2.0 * W[None, :, None] * X + ct * np.einsum("muv,mvr,mrc->muc", G, X, Sig)

    dinv = 1.0 / (2.0 * W[None, :, None] + ct * np.einsum("muu->mu", G)[:, :, None]
                  * np.einsum("mcc->mc", Sig)[:, None, :])
    x = np.array(X0, dtype=np.float64)
    r = R - apply(x)
    z = dinv * r
    p = z.copy()
    rz = float(np.sum(r * z))
    rn0 = float(np.sqrt(np.sum(R * R)))
    it = 0
    while it < max_iter:
        if np.sqrt(np.sum(r * r)) <= tol * rn0:
            break
        Ap = apply(p)
        alpha = rz / float(np.sum(p * Ap))
        x = x + alpha * p
        r = r - alpha * Ap
        z = dinv * r
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it


def gain_solve(H, R):
    """Solve blkdiag(H_m) k = r for gain-shaped R (T, nu, nx); returns (T, nu, nx)."""
    T, nu, nx = R.shape
    out = np.zeros_like(R)
    for m in range(T):
        out[m] = np.linalg.solve(H[m], R[m].flatten(order="F")).reshape((nu, nx), order="F")
    return out


def ell(lin, du):
    """Linear part of g^{lin,1} in δû: b_jᵀ δû for every row (b_j = F_uᵀ∇g_j for state
    rows, ±e_i at step k for control rows)."""
    return np.einsum("jku,ku->j", lin.bvec, du)


def delta_x(lin, du):
    """δx = F_u δû, as (T+1, nx)."""
    T, nx = lin.x_hat.shape[0] - 1, lin.x_hat.shape[1]
    return (lin.Fu @ du.reshape(-1)).reshape(T + 1, nx)
