"""Pins for the oracle's NRTO-DR (Sec. II-B, Sec. III, Supplementary Sec. II)."""
import numpy as np

from oracle import dr as D, fulladmm as F, problem as P

from . import ipsolver
from .test_oracle_fulladmm import tiny_unicycle

RNG = np.random.default_rng(9)


def sub1_ip(inst, lin, p, lam, rho):
    """Subproblem (7) as a dense SOCP: min ½k_vᵀQ_vk_v + ρ/2‖p̃ - p - λ/ρ‖², ‖Â_jk+b̂_j‖ ≤ p̃_j."""
    T, nu, nx = inst.T, inst.nu, inst.nx
    n2, ng = T * nu * nx, lin.g0.shape[0]
    n = n2 + ng
    Pm = np.zeros((n, n))
    Pm[:n2, :n2] = 2 * np.kron(np.eye(T * nx), np.diag(inst.RK ** 2))
    Pm[n2:, n2:] = rho * np.eye(ng)
    q = np.zeros(n)
    q[n2:] = -rho * (p + lam / rho)
    socs = []
    for j in range(ng):
        A = np.zeros(((T + 1) * nx, n))
        A[:, :n2] = P.dense_Ahat(lin, j)
        c = np.zeros(n)
        c[n2 + j] = 1.0
        socs.append((A, lin.bhat[j].reshape(-1), c, 0.0))
    x0 = np.zeros(n)
    x0[n2:] = np.linalg.norm(lin.bhat.reshape(ng, -1), axis=1) + 1.0
    x = ipsolver.solve(Pm, q, socs, None, None, x0)
    return P.K_from_kv(x[:n2], T, nu, nx), x[n2:]


def test_dr_fixed_point_matches_interior_point():
    inst = tiny_unicycle(tau=4.0)
    lin = P.linearize(inst, inst.u_init)
    ng = lin.g0.shape[0]
    rho = 40.0
    p = 0.05 * RNG.normal(size=ng)
    lam = 0.5 * RNG.normal(size=ng)
    K_ip, pt_ip = sub1_ip(inst, lin, p, lam, rho)
    o = D.DROptions(rho=rho, eps_dr=1e-12, max_dr=40000)
    K, pt, st, it, r = D.dr_solve(inst, lin, p, lam, o)
    assert r <= 1e-12
    assert np.allclose(K, K_ip, atol=1e-7) and np.allclose(pt, pt_ip, atol=1e-7)
    # Some cones are active at this point, the others slack.
    Y = np.linalg.norm((P.Ahat_apply(lin, K) + lin.bhat).reshape(ng, -1), axis=1)
    assert np.any(np.abs(Y - pt) < 1e-6) and np.any(Y < pt - 1e-3)


def test_affine_step_solves_kkt_system():
    """χ from step 1 satisfies the KKT system of Supplementary Sec. II-B with y = R_s(s̃ - s)."""
    inst = tiny_unicycle(T=4)
    lin = P.linearize(inst, inst.u_init)
    T, nu, nx = inst.T, inst.nu, inst.nx
    ng = lin.g0.shape[0]
    rho, rc, sg = 40.0, 0.7, 1.3
    p, lam = RNG.normal(size=ng), RNG.normal(size=ng)
    st = D.DRState(Kt=RNG.normal(size=(T, nu, nx)), ptt=RNG.normal(size=ng), tt=RNG.normal(size=ng),
                   etat=RNG.normal(size=(ng, T + 1, nx)))
    o = D.DROptions(rho=rho, r_chi=rc, sigma=sg)
    K, pt, _, _, _ = D.dr_solve(inst, lin, p, lam, o, state=D.DRState(st.Kt.copy(), st.ptt.copy(), st.tt.copy(), st.etat.copy()), n_iter=1, check=False)
    # Build A, b, P, q densely (Supplementary Sec. II-A) and check both KKT rows.
    n2 = T * nu * nx
    nz = (T + 1) * nx
    m = ng * (1 + nz)
    A = np.zeros((m, n2 + ng))
    b = np.zeros(m)
    s_tilde = np.zeros(m)
    for j in range(ng):
        r0 = j * (1 + nz)
        A[r0, n2 + j] = -1.0
        A[r0 + 1:r0 + 1 + nz, :n2] = -P.dense_Ahat(lin, j)
        b[r0 + 1:r0 + 1 + nz] = lin.bhat[j].reshape(-1)
        s_tilde[r0] = st.tt[j]
        s_tilde[r0 + 1:r0 + 1 + nz] = st.etat[j].reshape(-1)
    Pm = np.zeros((n2 + ng, n2 + ng))
    Pm[:n2, :n2] = 2 * np.kron(np.eye(T * nx), np.diag(inst.RK ** 2))
    Pm[n2:, n2:] = rho * np.eye(ng)
    q = np.concatenate([np.zeros(n2), -rho * (p + lam / rho)])
    chi = np.concatenate([P.kv_from_K(K), pt])
    chi_t = np.concatenate([P.kv_from_K(st.Kt), st.ptt])
    s = b - A @ chi
    y = sg * (s_tilde - s)
    r1 = (Pm + rc * np.eye(n2 + ng)) @ chi + A.T @ y - (rc * chi_t - q)
    r2 = A @ chi - y / sg - (b - s_tilde)
    assert np.abs(r1).max() < 1e-10 and np.abs(r2).max() < 1e-10


def test_subproblem2_matches_interior_point():
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    T, nu = inst.T, inst.nu
    ng = lin.g0.shape[0]
    rho = 40.0
    for r_trust in [0.3, 100.0]:
        pt = 0.1 * RNG.normal(size=ng)
        lam = RNG.normal(size=ng)
        du, dx, p, mu = D.sub2_solve(inst, lin, rho, pt, lam, r_trust)
        H, Ft, Rbar, Qbar, Bm = F.block2_matrices(inst, lin, 0.0)
        n1 = T * nu
        n = n1 + ng
        Pm = np.zeros((n, n))
        Pm[:n1, :n1] = H
        Pm[n1:, n1:] = rho * np.eye(ng)
        qv = np.zeros(n)
        xdev = (lin.x_hat[1:] - inst.x_goal).reshape(-1)
        udev = (lin.u_hat - inst.u_ref).reshape(-1)
        qv[:n1] = 2 * Rbar @ udev + 2 * Ft.T @ Qbar @ xdev
        qv[n1:] = lam - rho * pt
        G = np.zeros((ng, n))
        G[:, :n1] = Bm
        G[:, n1:] = np.eye(ng)
        At = np.zeros((Ft.shape[0], n))
        At[:, :n1] = Ft
        x0 = np.zeros(n)
        x0[n1:] = -lin.g0 - 1.0
        x = ipsolver.solve(Pm, qv, [(At, np.zeros(Ft.shape[0]), np.zeros(n), r_trust)], G, -lin.g0, x0)
        assert np.allclose(du.reshape(-1), x[:n1], atol=1e-7)
        assert np.allclose(p, x[n1:], atol=1e-7)
        if r_trust < 1:
            assert mu > 0 and np.isclose(np.linalg.norm(Ft @ du.reshape(-1)), r_trust, rtol=1e-10)


def test_dr_and_fulladmm_reach_the_same_problem2_solution():
    inst = tiny_unicycle()
    lin = P.linearize(inst, inst.u_init)
    res = D.solve(inst, lin, D.DROptions(r_trust=0.5, eps_dr=1e-10, max_dr=5000, eps_p=1e-8, eps_d=1e-8, max_admm=400))
    s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=0.5, eps_p=1e-9, eps_d=1e-9, max_iter=30000))
    assert res.converged and s.converged
    assert np.allclose(res.du, s.du, atol=1e-5) and np.allclose(res.K, s.K, atol=1e-5)
