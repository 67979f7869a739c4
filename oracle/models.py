"""Dynamics and constraint functions (oracle; test infrastructure only).

All functions are written with operations that extend to complex arguments so that
Jacobians can be taken by complex-step differentiation (Im f(x + i h e_k) / h), which is
exact to rounding and needs nothing but f itself.
"""
from __future__ import annotations

import numpy as np

from paper_2603_02642_b300.workloads import KIND_ARM, KIND_QUADCOPTER, KIND_UNICYCLE

_H = 1e-30  # complex-step size


def f_unicycle(x, u, dt):
    """Forward-Euler unicycle, Supplementary Sec. IV-A ("Unicycle Model")."""
    return np.array([x[0] + u[0] * np.cos(x[2]) * dt,
                     x[1] + u[0] * np.sin(x[2]) * dt,
                     x[2] + u[1] * dt])


def quad_xdot(x, u, prm):
    """Continuous quadcopter dynamics, Supplementary Sec. IV-A ("Quadcopter Model"):
    ṗ = v, v̇ = -g e3 + (f/m) R(φ,θ,ψ) e3 with R = Rz(ψ)Ry(θ)Rx(φ),
    [φ̇,θ̇,ψ̇] = T(φ,θ) ω, ω̇ = J^{-1}(τ - ω × Jω)."""
    m, g, Jx, Jy, Jz = prm
    v = x[3:6]
    phi, th, psi = x[6], x[7], x[8]
    om = x[9:12]
    f, tau = u[0], u[1:4]
    cph, sph, cth, sth, cps, sps = np.cos(phi), np.sin(phi), np.cos(th), np.sin(th), np.cos(psi), np.sin(psi)
    Rz = np.array([[cps, -sps, 0 * cps], [sps, cps, 0 * cps], [0 * cps, 0 * cps, 1 + 0 * cps]])
    Ry = np.array([[cth, 0 * cth, sth], [0 * cth, 1 + 0 * cth, 0 * cth], [-sth, 0 * cth, cth]])
    Rx = np.array([[1 + 0 * cph, 0 * cph, 0 * cph], [0 * cph, cph, -sph], [0 * cph, sph, cph]])
    R = Rz @ Ry @ Rx
    vdot = np.array([0.0, 0.0, -g]) + (f / m) * R[:, 2]
    Tm = np.array([[1 + 0 * cph, sph * np.tan(th), cph * np.tan(th)],
                   [0 * cph, cph, -sph],
                   [0 * cph, sph / cth, cph / cth]])
    angdot = Tm @ om
    J = np.array([Jx, Jy, Jz])
    Jom = J * om
    cross = np.array([om[1] * Jom[2] - om[2] * Jom[1],
                      om[2] * Jom[0] - om[0] * Jom[2],
                      om[0] * Jom[1] - om[1] * Jom[0]])
    omdot = (tau - cross) / J
    return np.concatenate([v, vdot, angdot, omdot])


def _clip(z, lo, hi):
    """Element-wise clip that extends to complex arguments by comparing real parts: a clamped
    component takes the (real) bound, so its complex-step derivative is zero; inside the bounds
    (bounds included) the component passes through with derivative one."""
    out = np.array(z, copy=True)
    below = np.real(z) < lo
    above = np.real(z) > hi
    out[below] = lo[below]
    out[above] = hi[above]
    return out


def f_arm(x, u, dt, damping=None, inertia=None, clip=False, lo=None, hi=None):
    """Franka joint-space model (Supplementary Sec. IV-A, "Franka Manipulator Model"):
    q̈_i = (τ_i - d_i q̇_i) / I_i; forward Euler with post-update clamping,
    q̇_{k+1} = clip(q̇_k + q̈_k dt, -q̇_max, q̇_max), q_{k+1} = clip(q_k + q̇_{k+1} dt, q_min, q_max),
    the limits being the state bounds lo, hi.  Without damping, inertia or clipping (the defaults)
    this is the double integrator q̇_{k+1} = q̇_k + u dt, q_{k+1} = q_k + q̇_{k+1} dt."""
    q, dq = x[:7], x[7:]
    d = np.zeros(7) if damping is None else damping
    inr = np.ones(7) if inertia is None else inertia
    dq1 = dq + (u - d * dq) / inr * dt
    if clip:
        dq1 = _clip(dq1, lo[7:], hi[7:])
    q1 = q + dq1 * dt
    if clip:
        q1 = _clip(q1, lo[:7], hi[:7])
    return np.concatenate([q1, dq1])


# Parameter layout of the arm model (flat dyn_params): the DH table (a_i, d_i, α_i) × 7, then, when
# present, damping d (7), inertia I (7) and the clipping flag (1).
ARM_DH, ARM_DAMP, ARM_INERT, ARM_CLIP, ARM_NPRM = 0, 21, 28, 35, 36


def arm_params(inst):
    """(damping, inertia, clip) of an arm instance; the 21-value table is the double integrator."""
    prm = inst.dyn_params
    if prm.size >= ARM_NPRM:
        return prm[ARM_DAMP:ARM_DAMP + 7], prm[ARM_INERT:ARM_INERT + 7], bool(prm[ARM_CLIP] != 0.0)
    return np.zeros(7), np.ones(7), False


def step(inst, x, u):
    """x_{k+1} = f(x_k, u_k) for the instance's model (Problem 1 dynamics, d_k = 0)."""
    if inst.kind == KIND_UNICYCLE:
        return f_unicycle(x, u, inst.dt)
    if inst.kind == KIND_QUADCOPTER:
        return x + inst.dt * quad_xdot(x, u, inst.dyn_params)
    if inst.kind == KIND_ARM:
        d, inr, clip = arm_params(inst)
        return f_arm(x, u, inst.dt, d, inr, clip, inst.x_lo, inst.x_hi)
    raise ValueError(inst.kind)


def jacobians(inst, x, u):
    """A = ∂f/∂x, B = ∂f/∂u by complex step."""
    nx, nu = inst.nx, inst.nu
    A = np.zeros((nx, nx))
    B = np.zeros((nx, nu))
    for i in range(nx):
        xc = x.astype(complex)
        xc[i] += 1j * _H
        A[:, i] = np.imag(step(inst, xc, u.astype(complex))) / _H
    for i in range(nu):
        uc = u.astype(complex)
        uc[i] += 1j * _H
        B[:, i] = np.imag(step(inst, x.astype(complex), uc)) / _H
    return A, B


def rollout(inst, u):
    """Nominal trajectory x̂_0 = x̄_0, x̂_{k+1} = f(x̂_k, û_k)."""
    x = np.zeros((inst.T + 1, inst.nx))
    x[0] = inst.x0
    for k in range(inst.T):
        x[k + 1] = step(inst, x[k], u[k])
    return x


def dh_transform(theta, d, a, alpha):
    """Standard Denavit–Hartenberg link transform Rot_z(θ) Trans_z(d) Trans_x(a) Rot_x(α)."""
    ct, st = np.cos(theta), np.sin(theta)
    ca, sa = np.cos(alpha), np.sin(alpha)
    z = 0 * ct
    return np.array([[ct, -st * ca, st * sa, a * ct],
                     [st, ct * ca, -ct * sa, a * st],
                     [z, sa + z, ca + z, d + z],
                     [z, z, z, 1 + z]])


def arm_link_sphere_centres(inst, q):
    """World positions of the link spheres: frame_l = Π_{i≤l} DH_i(q_i), centre = frame_l·[offset;1]."""
    dh = inst.dyn_params[:21].reshape(7, 3)
    frames = []
    Tcur = np.eye(4) + 0 * q[0]
    for i in range(7):
        Tcur = Tcur @ dh_transform(q[i], dh[i, 1], dh[i, 0], dh[i, 2])
        frames.append(Tcur)
    out = []
    for s in inst.link_spheres:
        Tl = frames[int(s[0]) - 1]
        out.append(Tl[:3, :3] @ s[1:4] + Tl[:3, 3])
    return np.array(out)


def _norm(v):
    return np.sqrt(np.sum(v * v))


def state_rows(inst):
    """State-constraint rows in the shared row order: for t = 1..T: obstacle rows
    (unicycle/quadcopter: obstacle o; arm: link sphere l major, static sphere o minor),
    then state-box rows (state i ascending, upper bound before lower bound).
    Returns a list of (t, kind, a, b): kind 0 = sphere clearance (a = obstacle, b = link),
    kind 1 = upper box on state a, kind 2 = lower box on state a."""
    rows = []
    for t in range(1, inst.T + 1):
        if inst.kind == KIND_ARM:
            for l in range(inst.link_spheres.shape[0]):
                for o in range(inst.n_obs):
                    rows.append((t, 0, o, l))
        else:
            for o in range(inst.n_obs):
                rows.append((t, 0, o, -1))
        for i in range(inst.nx):
            if np.isfinite(inst.x_hi[i]):
                rows.append((t, 1, i, -1))
            if np.isfinite(inst.x_lo[i]):
                rows.append((t, 2, i, -1))
    return rows


def control_rows(inst):
    """Control-bound rows: for k = 0..T-1, input i ascending, upper before lower.
    Returns a list of (k, i, sign): sign +1 is u_{k,i} - u_hi ≤ 0, -1 is u_lo - u_{k,i} ≤ 0."""
    rows = []
    for k in range(inst.T):
        for i in range(inst.nu):
            if np.isfinite(inst.u_hi[i]):
                rows.append((k, i, +1))
            if np.isfinite(inst.u_lo[i]):
                rows.append((k, i, -1))
    return rows


def g_state(inst, row, x_t):
    """Robust state constraint g_j(x_t) ≤ 0 (Problem 1). Sphere clearance
    g = r - ‖P x - c‖ (concave); box rows are linear."""
    t, kind, a, b = row
    if kind == 0:
        if inst.kind == KIND_ARM:
            c = arm_link_sphere_centres(inst, x_t[:7])[b]
            r = inst.link_spheres[b, 4] + inst.obs_radius[a]
            return r - _norm(c - inst.obs_center[a])
        d = inst.obs_dim
        return inst.obs_radius[a] - _norm(x_t[:d] - inst.obs_center[a])
    if kind == 1:
        return x_t[a] - inst.x_hi[a]
    return inst.x_lo[a] - x_t[a]


def g_state_grad(inst, row, x_t):
    """∇_x g_j(x_t) by complex step."""
    grad = np.zeros(inst.nx)
    for i in range(inst.nx):
        xc = x_t.astype(complex)
        xc[i] += 1j * _H
        grad[i] = np.imag(g_state(inst, row, xc)) / _H
    return grad
