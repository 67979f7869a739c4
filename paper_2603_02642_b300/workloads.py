"""Seeded synthetic workload generators for the robust trajectory problems.

This module only draws problem data (initial states, goals, obstacles, horizons,
disturbance covariances, DH tables); it performs none of the solver's arithmetic
(no rollouts, no linearization, no projections).  Both the CUDA library and the
CPU oracle consume the `Instance` objects it returns, so every parity comparison
starts from identical inputs.

Problem statement followed (Section II-A, Problem 1): dynamics x_{k+1} = f(x_k,u_k)+d_k,
x_0 = x̄_0 + d̄_0, disturbance ζ = [d̄_0; d_0; ...; d_{T-1}] in the ellipsoid
{ζ = Γz, zᵀSz ≤ τ} with Γ = I and S block diagonal (Supplementary Sec. V-D), affine
disturbance-feedback policy u_k = ū_k + K_k d_{k-1}, robust state constraints g ≤ 0 and
robust control constraints h ≤ 0.

Dynamics models (Supplementary Sec. IV-A): unicycle (3,2), quadcopter (12,4); the 7-DoF arm
as a double integrator with random-DH forward kinematics (`arm`), and the paper's Franka model
(`franka`: damping, unit inertia, clamped joint limits, torque bounds, the Panda's published
kinematics with this library's collision spheres).

Draw order is fixed per generator and documented inline; `numpy.random.default_rng(seed)`.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

KIND_UNICYCLE = 0
KIND_QUADCOPTER = 1
KIND_ARM = 2
KIND_NAMES = {KIND_UNICYCLE: "unicycle", KIND_QUADCOPTER: "quadcopter", KIND_ARM: "arm"}
DIMS = {KIND_UNICYCLE: (3, 2), KIND_QUADCOPTER: (12, 4), KIND_ARM: (14, 7)}

# Franka joint limits (Supplementary Table "Dynamics dimensions and model parameters").
ARM_Q_MIN = np.array([-2.9007, -1.8361, -2.9007, -3.0770, -2.8763, 0.4398, -3.0508])
ARM_Q_MAX = np.array([2.9007, 1.8361, 2.9007, -0.1169, 2.8763, 4.6216, 3.0508])
ARM_DQ_MAX = np.array([2.62, 2.62, 2.62, 2.62, 5.26, 4.18, 5.26])


@dataclass
class Instance:
    """One robust trajectory-optimization problem (Problem 1 data), all float64.

    kind        KIND_* code
    nx, nu, T   state dim, input dim, horizon
    dt          time step of the forward-Euler discretization
    dyn_params  flat model parameters: quadcopter [m, g, Jx, Jy, Jz]; arm DH table
                rows (a_i, d_i, alpha_i) for i = 1..7 (21 values); unicycle none
    x0          nominal initial state x̄_0                          (nx,)
    x_goal      goal state of the tracking cost                    (nx,)
    u_init      initial nominal controls û                         (T, nu)
    u_ref       reference control of the input cost                (nu,)
    Sigma       S^{-1} diagonal blocks, block i ↔ ζ-block i        (T+1, nx, nx)
    tau         ellipsoid radius τ
    Qx, Ru, RK  diagonals of the state-tracking, input and gain weights
    obs_dim     2 (planar) or 3; obstacles act on the first obs_dim states, or on the
                arm's link spheres
    obs_center  (n_obs, obs_dim), obs_radius (n_obs,)
    link_spheres (n_link, 5): [link index 1..7, offset x, y, z, radius] (arm only)
    u_lo, u_hi  control bounds, ±inf where absent                  (nu,)
    x_lo, x_hi  state bounds, ±inf where absent                    (nx,)
    """

    kind: int
    nx: int
    nu: int
    T: int
    dt: float
    dyn_params: np.ndarray
    x0: np.ndarray
    x_goal: np.ndarray
    u_init: np.ndarray
    u_ref: np.ndarray
    Sigma: np.ndarray
    tau: float
    Qx: np.ndarray
    Ru: np.ndarray
    RK: np.ndarray
    obs_dim: int
    obs_center: np.ndarray
    obs_radius: np.ndarray
    link_spheres: np.ndarray = field(default_factory=lambda: np.zeros((0, 5)))
    u_lo: np.ndarray = None
    u_hi: np.ndarray = None
    x_lo: np.ndarray = None
    x_hi: np.ndarray = None
    seed: int = -1

    @property
    def n_obs(self) -> int:
        return int(self.obs_radius.shape[0])

    @property
    def kind_name(self) -> str:
        return KIND_NAMES[self.kind]


def _diag_blocks(T: int, diag) -> np.ndarray:
    d = np.asarray(diag, dtype=np.float64)
    return np.repeat(np.diag(d)[None, :, :], T + 1, axis=0)


def _reject_obstacles(rng, n_obs, lo, hi, r_lo, r_hi, keep_clear, dim):
    """Draw n_obs spheres (centre U[lo,hi]^dim, radius U[r_lo,r_hi]); redraw any sphere
    whose surface comes within 0.3 of a point in keep_clear (start and goal)."""
    centers = np.zeros((n_obs, dim))
    radii = np.zeros(n_obs)
    for o in range(n_obs):
        for _ in range(1000):
            c = rng.uniform(lo, hi, size=dim)
            r = rng.uniform(r_lo, r_hi)
            if all(np.linalg.norm(c - p[:dim]) > r + 0.3 for p in keep_clear):
                break
        centers[o], radii[o] = c, r
    return centers, radii


def unicycle(seed: int, T: int = 20, n_obs: int = 3, dt: float = 0.1,
             x0_xy=(0.0, 0.0), goal_xy=(5.0, 5.0), box=(0.0, 5.0)) -> Instance:
    """Unicycle x=[px,py,θ], u=[v,ω]; |v|≤1.5, |ω|≤2; disturbance Q=diag(.02²,.02²,.01²), τ=1.
    Draws: obstacles (centre then radius, per obstacle, with rejection)."""
    rng = np.random.default_rng(seed)
    x0 = np.array([x0_xy[0], x0_xy[1], 0.0])
    xg = np.array([goal_xy[0], goal_xy[1], 0.0])
    centers, radii = _reject_obstacles(rng, n_obs, box[0], box[1], 0.3, 0.6, [x0, xg], 2)
    v0 = min(math.hypot(xg[0] - x0[0], xg[1] - x0[1]) / (T * dt), 1.5)
    u_init = np.tile(np.array([v0, 0.0]), (T, 1))
    return Instance(
        kind=KIND_UNICYCLE, nx=3, nu=2, T=T, dt=dt, dyn_params=np.zeros(0),
        x0=x0, x_goal=xg, u_init=u_init, u_ref=np.zeros(2),
        Sigma=_diag_blocks(T, [0.02 ** 2, 0.02 ** 2, 0.01 ** 2]), tau=1.0,
        Qx=np.ones(3), Ru=0.1 * np.ones(2), RK=math.sqrt(0.1) * np.ones(2),
        obs_dim=2, obs_center=centers, obs_radius=radii,
        u_lo=np.array([-1.5, -2.0]), u_hi=np.array([1.5, 2.0]),
        x_lo=np.full(3, -np.inf), x_hi=np.full(3, np.inf), seed=seed)


def quadcopter(seed: int, T: int = 100, n_obs: int = 10, dt: float = 0.05,
               x0_pos=(0.0, 0.0, 0.0), goal_pos=(10.0, 10.0, 10.0),
               box=(0.0, 10.0), inertia=(0.01, 0.01, 0.01)) -> Instance:
    """Quadcopter x=[p,v,φ,θ,ψ,ω] (12), u=[f,τ] (4); m=1, g=9.81; f∈[0,15], τ∈[-.5,.5]³;
    disturbance Q=1e-4·I, τ=1. Draws: obstacles (centre then radius, with rejection)."""
    rng = np.random.default_rng(seed)
    x0 = np.zeros(12)
    x0[:3] = x0_pos
    xg = np.zeros(12)
    xg[:3] = goal_pos
    centers, radii = _reject_obstacles(rng, n_obs, box[0], box[1], 0.4, 1.0, [x0, xg], 3)
    m, g = 1.0, 9.81
    hover = np.array([m * g, 0.0, 0.0, 0.0])
    return Instance(
        kind=KIND_QUADCOPTER, nx=12, nu=4, T=T, dt=dt,
        dyn_params=np.array([m, g, inertia[0], inertia[1], inertia[2]]),
        x0=x0, x_goal=xg, u_init=np.tile(hover, (T, 1)), u_ref=hover.copy(),
        Sigma=_diag_blocks(T, 1e-4 * np.ones(12)), tau=1.0,
        Qx=np.ones(12), Ru=0.1 * np.ones(4), RK=math.sqrt(0.1) * np.ones(4),
        obs_dim=3, obs_center=centers, obs_radius=radii,
        u_lo=np.array([0.0, -0.5, -0.5, -0.5]), u_hi=np.array([15.0, 0.5, 0.5, 0.5]),
        x_lo=np.full(12, -np.inf), x_hi=np.full(12, np.inf), seed=seed)


def arm(seed: int, T: int = 100, n_link: int = 8, n_static: int = 6, dt: float = 0.02) -> Instance:
    """7-DoF arm, double integrator on x=[q, q̇] (14), u=q̈ (7); joint position and velocity
    limits; link spheres vs static spheres through a seeded random DH chain.
    Draws, in order: DH a(7), d(7), α sign(7); link sphere (link, offset(3), radius) per sphere;
    static sphere (direction(3), radius-from-base, radius) per sphere; q0(7); q_goal(7)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 0.1, size=7)
    d = rng.uniform(0.1, 0.4, size=7)
    alpha = np.where(rng.uniform(size=7) < 0.5, -math.pi / 2, math.pi / 2)
    dh = np.stack([a, d, alpha], axis=1).reshape(-1)
    links = np.zeros((n_link, 5))
    for i in range(n_link):
        links[i, 0] = 1 + (i % 7)
        links[i, 1:4] = rng.uniform(-0.05, 0.05, size=3)
        links[i, 4] = rng.uniform(0.05, 0.1)
    centers = np.zeros((n_static, 3))
    radii = np.zeros(n_static)
    for o in range(n_static):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        centers[o] = u * rng.uniform(0.6, 1.2)
        radii[o] = rng.uniform(0.05, 0.15)
    mid = 0.5 * (ARM_Q_MIN + ARM_Q_MAX)
    half = 0.5 * (ARM_Q_MAX - ARM_Q_MIN) * 0.8
    q0 = mid + half * rng.uniform(-1, 1, size=7)
    qg = mid + half * rng.uniform(-1, 1, size=7)
    x0 = np.concatenate([q0, np.zeros(7)])
    xg = np.concatenate([qg, np.zeros(7)])
    return Instance(
        kind=KIND_ARM, nx=14, nu=7, T=T, dt=dt, dyn_params=dh,
        x0=x0, x_goal=xg, u_init=np.zeros((T, 7)), u_ref=np.zeros(7),
        Sigma=_diag_blocks(T, 1e-4 * np.ones(14)), tau=1.0,
        Qx=np.ones(14), Ru=0.1 * np.ones(7), RK=math.sqrt(0.1) * np.ones(7),
        obs_dim=3, obs_center=centers, obs_radius=radii, link_spheres=links,
        u_lo=np.full(7, -np.inf), u_hi=np.full(7, np.inf),
        x_lo=np.concatenate([ARM_Q_MIN, -ARM_DQ_MAX]),
        x_hi=np.concatenate([ARM_Q_MAX, ARM_DQ_MAX]), seed=seed)


# Franka Emika Panda kinematics: the manufacturer's published modified (Craig) DH table, rows
# (a_{i-1}, d_i, α_{i-1}) for joints 1..7 and the flange: (0, .333, 0), (0, 0, -π/2), (0, .316, π/2),
# (.0825, 0, π/2), (-.0825, .384, -π/2), (0, 0, π/2), (.088, 0, π/2), flange (0, .107, 0).  Since
# Rot_x and Trans_x commute, that chain equals a standard-DH chain whose joint i takes d_i and the
# (a, α) of the next row, with the flange offset as joint 7's d: the rows below, (a_i, d_i, α_i).
FRANKA_DH = np.array([
    [0.0, 0.333, -math.pi / 2],
    [0.0, 0.0, math.pi / 2],
    [0.0825, 0.316, math.pi / 2],
    [-0.0825, 0.0, -math.pi / 2],
    [0.0, 0.384, math.pi / 2],
    [0.088, 0.0, math.pi / 2],
    [0.0, 0.107, 0.0],
])
# Model parameters (Supplementary Table "Dynamics dimensions and model parameters").
FRANKA_TAU_MAX = np.array([87.0, 87.0, 87.0, 87.0, 12.0, 12.0, 12.0])
FRANKA_DAMPING = np.full(7, 0.5)
FRANKA_INERTIA = np.ones(7)
# Collision spheres of this library (the paper's come from a simulator and are not given): link
# index of the standard-DH frame, offset in that frame, radius; at q = 0 they sit on the shoulder
# (0, 0, .333), the upper-arm axis (0, 0, .491), the elbow (.0825, 0, .649) and (0, 0, .649), the
# forearm axis (0, 0, .841), the wrist (0, 0, 1.033), (.088, 0, 1.033) and the hand (.088, 0, .876).
FRANKA_SPHERES = np.array([
    [1, 0.0, 0.0, 0.0, 0.09],
    [2, 0.0, 0.0, 0.158, 0.08],
    [3, 0.0, 0.0, 0.0, 0.08],
    [4, 0.0, 0.0, 0.0, 0.07],
    [4, 0.0, 0.0, 0.192, 0.07],
    [5, 0.0, 0.0, 0.0, 0.07],
    [6, 0.0, 0.0, 0.0, 0.06],
    [7, 0.0, 0.0, 0.05, 0.07],
])
FRANKA_Q_READY = np.array([0.0, -math.pi / 4, 0.0, -3 * math.pi / 4, 0.0, math.pi / 2, math.pi / 4])


def franka(seed: int, T: int = 100, n_static: int = 6, dt: float = 0.02) -> Instance:
    """The paper's Franka model: x = [q, q̇] (14), u = τ (7); q̈ = (τ - d q̇)/I with d = 0.5, I = 1,
    forward Euler with the joint position and velocity limits clamped after each step, torque bounds
    |τ_i| ≤ τ_max,i as robust control constraints, the limits also as robust state constraints; the
    Panda's published kinematics with this library's link spheres against static spheres.
    Draws, in order: static sphere centre (3) and radius per sphere (centres at |y| in [.35, .7]
    beside the arm, x in [.1, .6], z in [.1, .8]); q0 (7) and q_goal (7) within ±0.4 rad of the
    ready pose, inside 80% of the joint range."""
    rng = np.random.default_rng(seed)
    centers = np.zeros((n_static, 3))
    radii = np.zeros(n_static)
    for o in range(n_static):
        side = 1.0 if rng.uniform() < 0.5 else -1.0
        centers[o] = [rng.uniform(0.1, 0.6), side * rng.uniform(0.35, 0.7), rng.uniform(0.1, 0.8)]
        radii[o] = rng.uniform(0.05, 0.12)
    mid = 0.5 * (ARM_Q_MIN + ARM_Q_MAX)
    half = 0.5 * (ARM_Q_MAX - ARM_Q_MIN) * 0.8
    q0 = np.clip(FRANKA_Q_READY + rng.uniform(-0.4, 0.4, size=7), mid - half, mid + half)
    qg = np.clip(FRANKA_Q_READY + rng.uniform(-0.4, 0.4, size=7), mid - half, mid + half)
    prm = np.concatenate([FRANKA_DH.reshape(-1), FRANKA_DAMPING, FRANKA_INERTIA, [1.0]])
    return Instance(
        kind=KIND_ARM, nx=14, nu=7, T=T, dt=dt, dyn_params=prm,
        x0=np.concatenate([q0, np.zeros(7)]), x_goal=np.concatenate([qg, np.zeros(7)]),
        u_init=np.zeros((T, 7)), u_ref=np.zeros(7),
        Sigma=_diag_blocks(T, 1e-4 * np.ones(14)), tau=1.0,
        Qx=np.ones(14), Ru=0.1 * np.ones(7), RK=math.sqrt(0.1) * np.ones(7),
        obs_dim=3, obs_center=centers, obs_radius=radii, link_spheres=FRANKA_SPHERES.copy(),
        u_lo=-FRANKA_TAU_MAX, u_hi=FRANKA_TAU_MAX.copy(),
        x_lo=np.concatenate([ARM_Q_MIN, -ARM_DQ_MAX]),
        x_hi=np.concatenate([ARM_Q_MAX, ARM_DQ_MAX]), seed=seed)


def batched_mix(n: int = 2048, base_seed: int = 10000) -> list[Instance]:
    """Mixed batch: kind ~ Bernoulli(0.5) per instance (seed base_seed+i).
    Unicycle: T~U{20..200}, n_obs~U{1..20}, x0~U[-.5,.5]²×{0}, goal~(5,5)+U[-.5,.5]²,
    obstacles in the [0,5]² start-goal box.  Quadcopter: T~U{50..150}, n_obs~U{1..15},
    x0 position ~U[0,1]³, goal position ~U[9,10]³."""
    out = []
    for i in range(n):
        seed = base_seed + i
        rng = np.random.default_rng(seed)
        if rng.uniform() < 0.5:
            T = int(rng.integers(20, 201))
            n_obs = int(rng.integers(1, 21))
            x0 = rng.uniform(-0.5, 0.5, size=2)
            goal = np.array([5.0, 5.0]) + rng.uniform(-0.5, 0.5, size=2)
            out.append(unicycle(seed=int(rng.integers(1 << 31)), T=T, n_obs=n_obs,
                                x0_xy=x0, goal_xy=goal))
        else:
            T = int(rng.integers(50, 151))
            n_obs = int(rng.integers(1, 16))
            x0 = rng.uniform(0.0, 1.0, size=3)
            goal = rng.uniform(9.0, 10.0, size=3)
            out.append(quadcopter(seed=int(rng.integers(1 << 31)), T=T, n_obs=n_obs,
                                  x0_pos=x0, goal_pos=goal))
        out[-1].seed = seed
    return out


def warmstart_quad(seed: int, T: int = 100, max_obs: int = 15) -> Instance:
    """Quadcopter T=100 with n_obs~U{1..max_obs}, x0 position ~U[0,1]³, goal ~U[9,10]³."""
    rng = np.random.default_rng(seed)
    n_obs = int(rng.integers(1, max_obs + 1))
    x0 = rng.uniform(0.0, 1.0, size=3)
    goal = rng.uniform(9.0, 10.0, size=3)
    inst = quadcopter(seed=int(rng.integers(1 << 31)), T=T, n_obs=n_obs, x0_pos=x0, goal_pos=goal)
    inst.seed = seed
    return inst


def config(name: str, seed: int = 0):
    """Named workloads: 'unicycle_T20' (single), 'quadcopter_T100', 'arm_T100',
    'batch2048' (list), and small parity cases."""
    if name == "unicycle_T20":
        return unicycle(seed)
    if name == "quadcopter_T100":
        return quadcopter(seed)
    if name == "arm_T100":
        return arm(seed)
    if name == "franka_T100":
        return franka(seed)
    if name == "batch2048":
        return batched_mix(2048)
    raise KeyError(name)
