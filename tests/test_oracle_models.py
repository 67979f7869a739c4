"""Pins for the oracle's dynamics models and constraint gradients (Supplementary Sec. IV-A)."""
import math

import numpy as np

from oracle import models
from paper_2603_02642_b300 import workloads as W

RNG = np.random.default_rng(7)


def _central_jac(fun, x, h=1e-6):
    cols = []
    for i in range(x.shape[0]):
        e = np.zeros_like(x)
        e[i] = h
        cols.append((fun(x + e) - fun(x - e)) / (2 * h))
    return np.stack(cols, axis=-1)


def test_complex_step_jacobians_match_central_differences():
    for inst in [W.unicycle(0), W.quadcopter(0, T=5), W.arm(0, T=5)]:
        for _ in range(3):
            x = RNG.normal(size=inst.nx) * 0.5
            u = RNG.normal(size=inst.nu)
            A, B = models.jacobians(inst, x, u)
            An = _central_jac(lambda y: models.step(inst, y, u), x)
            Bn = _central_jac(lambda v: models.step(inst, x, v), u)
            assert np.allclose(A, An, atol=1e-7) and np.allclose(B, Bn, atol=1e-7)


def test_unicycle_straight_line_and_turn():
    inst = W.unicycle(0)
    x = np.array([1.0, 2.0, math.pi / 4])
    y = models.step(inst, x, np.array([2.0, 0.5]))
    assert np.allclose(y, [1 + 0.2 * math.cos(math.pi / 4), 2 + 0.2 * math.sin(math.pi / 4), math.pi / 4 + 0.05])


def test_quadcopter_hover_free_fall_and_attitude():
    inst = W.quadcopter(0, T=5)
    m, g = inst.dyn_params[0], inst.dyn_params[1]
    x = np.zeros(12)
    x[:3] = [1, 2, 3]
    # Hover: level attitude, thrust m g → equilibrium.
    assert np.allclose(models.step(inst, x, np.array([m * g, 0, 0, 0])), x)
    # Free fall: v_z decreases by g dt.
    y = models.step(inst, x, np.zeros(4))
    assert np.isclose(y[5], -g * inst.dt) and np.allclose(y[:5], x[:5])
    # Thrust along the body z axis: roll φ tilts it to -y (R = Rz Ry Rx, Rx(φ)e3 = [0,-sinφ,cosφ]).
    x2 = x.copy()
    x2[6] = 0.3
    xd = models.quad_xdot(x2, np.array([m * g, 0, 0, 0]), inst.dyn_params)
    assert np.allclose(xd[3:6], [0, -g * math.sin(0.3), g * math.cos(0.3) - g])
    # Yaw rate with level attitude maps one-to-one to ψ̇; torque τ_z spins up r by τ/J_z.
    x3 = x.copy()
    x3[11] = 0.7
    xd = models.quad_xdot(x3, np.array([m * g, 0, 0, 0.02]), inst.dyn_params)
    assert np.isclose(xd[8], 0.7) and np.isclose(xd[11], 0.02 / inst.dyn_params[4])


def test_arm_double_integrator_closed_form():
    inst = W.arm(0, T=5)
    x = np.concatenate([RNG.normal(size=7), RNG.normal(size=7)])
    u = RNG.normal(size=7)
    y = models.step(inst, x, u)
    dt = inst.dt
    assert np.allclose(y[7:], x[7:] + u * dt)
    assert np.allclose(y[:7], x[:7] + x[7:] * dt + u * dt * dt)


def test_dh_planar_chain_matches_textbook():
    # With α = 0 and d = 0 the DH chain is a planar arm: p = Σ a_i [cos Σθ, sin Σθ].
    inst = W.arm(0, T=5)
    inst.dyn_params = np.stack([np.full(7, 0.3), np.zeros(7), np.zeros(7)], axis=1).reshape(-1)
    inst.link_spheres = np.array([[7, 0, 0, 0, 0.1], [3, 0, 0, 0, 0.1]])
    q = RNG.normal(size=7)
    c = models.arm_link_sphere_centres(inst, q)
    cum = np.cumsum(q)
    assert np.allclose(c[0], [0.3 * np.sum(np.cos(cum)), 0.3 * np.sum(np.sin(cum)), 0])
    assert np.allclose(c[1], [0.3 * np.sum(np.cos(cum[:3])), 0.3 * np.sum(np.sin(cum[:3])), 0])


def test_constraint_values_and_gradients():
    inst = W.quadcopter(3, T=4, n_obs=2)
    x = RNG.normal(size=12) + 5
    row = (1, 0, 1, -1)
    gv = models.g_state(inst, row, x)
    assert np.isclose(gv, inst.obs_radius[1] - np.linalg.norm(x[:3] - inst.obs_center[1]))
    gr = models.g_state_grad(inst, row, x)
    expect = np.zeros(12)
    expect[:3] = -(x[:3] - inst.obs_center[1]) / np.linalg.norm(x[:3] - inst.obs_center[1])
    assert np.allclose(gr, expect)
    arm = W.arm(1, T=4)
    q = RNG.normal(size=14)
    for row in [(1, 0, 2, 5), (1, 1, 3, -1), (1, 2, 10, -1)]:
        gn = _central_jac(lambda y: np.array([models.g_state(arm, row, y)]), q)[0]
        assert np.allclose(models.g_state_grad(arm, row, q), gn, atol=1e-7)


def test_row_order_and_counts():
    inst = W.unicycle(0)
    st, ct = models.state_rows(inst), models.control_rows(inst)
    assert len(st) == 60 and len(ct) == 80          # 3 obstacles × 20 steps; 2 bounds × 2 inputs × 20
    assert [r[0] for r in st] == sorted(r[0] for r in st)
    arm = W.arm(0, T=100)
    assert len(models.state_rows(arm)) == 7600 and len(models.control_rows(arm)) == 0


def _modified_dh_flange(q):
    """Independent forward kinematics of the Panda from the manufacturer's modified (Craig) DH table:
    T = Π_i Rot_x(α_{i-1}) Trans_x(a_{i-1}) Rot_z(q_i) Trans_z(d_i), then the flange Trans_z(0.107)."""
    rows = [(0.0, 0.333, 0.0), (0.0, 0.0, -math.pi / 2), (0.0, 0.316, math.pi / 2), (0.0825, 0.0, math.pi / 2),
            (-0.0825, 0.384, -math.pi / 2), (0.0, 0.0, math.pi / 2), (0.088, 0.0, math.pi / 2)]

    def rx(a):
        c, s = math.cos(a), math.sin(a)
        return np.array([[1, 0, 0, 0], [0, c, -s, 0], [0, s, c, 0], [0, 0, 0, 1.0]])

    def rz(a):
        c, s = math.cos(a), math.sin(a)
        return np.array([[c, -s, 0, 0], [s, c, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1.0]])

    def tr(x, z):
        T = np.eye(4)
        T[0, 3], T[2, 3] = x, z
        return T

    T = np.eye(4)
    for (a, d, al), qi in zip(rows, q):
        T = T @ rx(al) @ tr(a, 0.0) @ rz(qi) @ tr(0.0, d)
    return (T @ tr(0.0, 0.107))[:3, 3]


def test_franka_kinematics_match_the_published_modified_dh_chain():
    """The standard-DH rows of the Franka model reproduce the manufacturer's modified-DH chain: the
    flange at q = 0 is the Panda's documented (0.088, 0, 0.926), and at random joint angles the
    flange position equals that of an independent modified-DH evaluation."""
    inst = W.franka(0, T=5)
    inst.link_spheres = np.array([[7, 0.0, 0.0, 0.0, 0.05]])
    assert np.allclose(models.arm_link_sphere_centres(inst, np.zeros(7))[0], [0.088, 0.0, 0.926], atol=1e-12)
    for _ in range(5):
        q = RNG.uniform(-2.5, 2.5, size=7)
        assert np.allclose(models.arm_link_sphere_centres(inst, q)[0], _modified_dh_flange(q), atol=1e-12)


def test_franka_dynamics_damping_and_clamping():
    """q̈ = (τ - d q̇)/I with forward Euler, velocity then position clamped to the limits; the
    Jacobian of a clamped component is zero, elsewhere it matches central differences."""
    inst = W.franka(1, T=5)
    dt, d = inst.dt, 0.5
    x = np.concatenate([inst.x0[:7], 0.3 * RNG.uniform(-1, 1, size=7)])
    u = RNG.uniform(-5, 5, size=7)
    y = models.step(inst, x, u)
    dq1 = x[7:] + (u - d * x[7:]) * dt
    assert np.allclose(y[7:], dq1, atol=1e-15) and np.allclose(y[:7], x[:7] + dq1 * dt, atol=1e-15)
    A, B = models.jacobians(inst, x, u)
    assert np.allclose(A, _central_jac(lambda z: models.step(inst, z, u), x), atol=1e-7)
    assert np.allclose(B, _central_jac(lambda v: models.step(inst, x, v), u), atol=1e-7)
    assert np.allclose(A[7:, 7:], (1 - d * dt) * np.eye(7)) and np.allclose(B[7:], dt * np.eye(7))
    # joint 0 pushed past its velocity limit, joint 1 past its position limit
    x2 = x.copy()
    x2[7] = inst.x_hi[7] - 1e-3
    u2 = u.copy()
    u2[0] = 80.0
    x2[1] = inst.x_hi[1] - 1e-4
    x2[8] = 1.0
    y2 = models.step(inst, x2, u2)
    assert y2[7] == inst.x_hi[7] and y2[1] == inst.x_hi[1]
    A2, B2 = models.jacobians(inst, x2, u2)
    assert not A2[7].any() and not B2[7].any() and not A2[1].any() and not B2[1].any()
    assert A2[0, 7] == 0.0 and B2[0, 0] == 0.0          # q_0 moves with the clamped velocity
    # the 21-value table (no damping, unit inertia, no clamping) is the double integrator
    dbl = W.arm(0, T=5)
    yd = models.step(dbl, x, u)
    assert np.allclose(yd[7:], x[7:] + u * dbl.dt) and np.allclose(yd[:7], x[:7] + yd[7:] * dbl.dt)
