"""Monte Carlo check of robust-constraint satisfaction (oracle; test infrastructure only).

Sec. V ("Methodology", constraint satisfaction): a solution is rolled out through the nonlinear
dynamics under sampled disturbances of the uncertainty set, 1,000 drawn uniformly from its
interior and 1,000 reproducible edge cases on its boundary built from convex combinations of
the worst-case directions of the constraints; the satisfaction probability is the fraction of
rollouts that violate no constraint.  The paper gives no formulas for the sampling, so this
module fixes one reading of it (each choice below is a reading, not the paper's text):

- Whitened coordinates.  The disturbance is ζ = (ζ_0, …, ζ_T), ζ_i = √τ Ψ_iᵀ w_i with
  Ψ_iᵀΨ_i = Σ_i (problem.psi_blocks) and w ∈ R^{(T+1) n_x}, ‖w‖ ≤ 1.  For Γ = I this is the
  ellipsoid {ζ : ζᵀSζ ≤ τ}, S = blkdiag(Σ_i⁻¹), and w uniform in the unit ball makes ζ uniform
  in it.
- Interior sample: w = ρ g/‖g‖ with g standard normal in R^{(T+1) n_x} and ρ = U^{1/n}
  (U uniform in [0, 1), n = (T+1) n_x): the standard construction of a uniform point in a ball.
- Edge sample e (counted from 0): n_c = 1 + (e mod 3) rows j_1..j_{n_c} drawn uniformly from all
  rows (state rows, then control rows, the order of models.state_rows / control_rows) with
  weights a_c = 1 - U in (0, 1]; w = v/‖v‖ with v = Σ_c a_c y_{j_c}/‖y_{j_c}‖ and
  y_j = Â_j k + b̂_j the SOC row of Problem 2, whose direction maximizes the linearized
  constraint j over the set (rows with y_j = 0 contribute nothing; v = 0 gives w = 0).
- Rollout (the affine disturbance-feedback policy of Sec. II-A, as in problem.py):
  x_0 = x̄_0 + ζ_0, u_k = ū_k + K_k ζ_k, x_{k+1} = f(x_k, u_k) + ζ_{k+1}.  A rollout satisfies the
  constraints when every row of Problem 1 holds: g_j(x_t) ≤ tol for the state rows of
  t = 1..T and the control bounds at k = 0..T-1; its worst value is the largest constraint value.
- Random numbers: one counter-based generator, SplitMix64 (Steele, Lea and Flood, "Fast
  splittable pseudorandom number generators", OOPSLA 2014; output function and increment of
  S. Vigna's public-domain splitmix64.c).  The stream of (instance index i, sample s) is
  seeded with key = mix(seed XOR mix(i·2³² + s)); its n-th draw (n = 0, 1, …) is
  mix(key + (n+1)·γ), the n-th output of SplitMix64 started at key; U = (draw >> 11)·2⁻⁵³.
  Standard normal k of a sample is the Box–Muller pair of draws 2⌊k/2⌋, 2⌊k/2⌋+1:
  r = √(-2 ln(1 - U_0)), g_k = r cos(2π U_1) for even k, r sin(2π U_1) for odd k; the interior
  radius uses draw 2⌈n/2⌉.  Edge samples use draws 0..n_c-1 for the rows and n_c..2n_c-1 for
  the weights.
"""
from __future__ import annotations

import numpy as np

from . import models, problem

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def mix64(z):
    """SplitMix64 output function (works on Python ints and numpy uint64 arrays)."""
    if isinstance(z, np.ndarray):
        z = z.astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def stream_key(seed, inst_index, sample):
    return mix64((seed ^ mix64(((inst_index << 32) + sample) & MASK)) & MASK)


def draws(key, idx):
    """Draws idx (an integer array) of the stream seeded with key, as uint64."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(key) + (idx + np.uint64(1)) * np.uint64(GAMMA))


def uniforms(key, idx):
    return (draws(key, idx) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normals(key, n):
    """Standard normals 0..n-1 of the stream (Box–Muller over consecutive draw pairs)."""
    npair = (n + 1) // 2
    u = uniforms(key, np.arange(2 * npair))
    r = np.sqrt(-2.0 * np.log(1.0 - u[0::2]))
    a = 2.0 * np.pi * u[1::2]
    g = np.empty(2 * npair)
    g[0::2] = r * np.cos(a)
    g[1::2] = r * np.sin(a)
    return g[:n]


def soc_rows(lin, K):
    """y_j = Â_j k + b̂_j for every row, shape (n_g, T+1, n_x) (Problem 2)."""
    return problem.Ahat_apply(lin, K) + lin.bhat


def whitened_sample(inst, lin, K, seed, inst_index, sample, n_interior, Y=None):
    """The whitened disturbance w (shape (T+1, n_x)) of one sample (module docstring)."""
    T, nx = inst.T, inst.nx
    n = (T + 1) * nx
    key = stream_key(seed, inst_index, sample)
    if sample < n_interior:
        g = normals(key, n)
        rad = uniforms(key, [2 * ((n + 1) // 2)])[0] ** (1.0 / n)
        return (rad * g / np.linalg.norm(g)).reshape(T + 1, nx)
    if Y is None:
        Y = soc_rows(lin, K)
    e = sample - n_interior
    n_rows = Y.shape[0]
    nc = 1 + e % 3 if n_rows > 0 else 0
    u = uniforms(key, np.arange(2 * nc))
    rows = np.minimum((u[:nc] * n_rows).astype(np.int64), n_rows - 1)
    wts = 1.0 - u[nc:]
    v = np.zeros((T + 1, nx))
    for j, a in zip(rows, wts):
        nj = np.linalg.norm(Y[j])
        if nj > 0.0:
            v += a * Y[j] / nj
    nv = np.linalg.norm(v)
    return v / nv if nv > 0.0 else v


def disturbance(inst, w):
    """ζ_i = √τ Ψ_iᵀ w_i, shape (T+1, n_x)."""
    Psi = problem.psi_blocks(inst.Sigma)
    return np.sqrt(inst.tau) * np.einsum("iab,ia->ib", Psi, w)


def rollout(inst, u_bar, K, zeta):
    """Closed-loop nonlinear rollout (x of shape (T+1, n_x), u of shape (T, n_u))."""
    T = inst.T
    x = np.zeros((T + 1, inst.nx))
    u = np.zeros((T, inst.nu))
    x[0] = inst.x0 + zeta[0]
    for k in range(T):
        u[k] = u_bar[k] + K[k] @ zeta[k]
        x[k + 1] = models.step(inst, x[k], u[k]) + zeta[k + 1]
    return x, u


def worst_constraint(inst, x, u):
    """Largest constraint value of a trajectory over the rows of Problem 1."""
    vals = [models.g_state(inst, row, x[row[0]]) for row in models.state_rows(inst)]
    for (k, i, s) in models.control_rows(inst):
        vals.append(u[k, i] - inst.u_hi[i] if s > 0 else inst.u_lo[i] - u[k, i])
    return max(vals) if vals else -np.inf


def check(inst, u_bar, K, seed, inst_index, n_interior, n_edge, tol=0.0):
    """Monte Carlo satisfaction of one instance: (number of rollouts with every constraint ≤ tol,
    per-sample worst constraint values)."""
    lin = problem.linearize(inst, u_bar)
    Y = soc_rows(lin, K)
    worst = np.zeros(n_interior + n_edge)
    for s in range(n_interior + n_edge):
        w = whitened_sample(inst, lin, K, seed, inst_index, s, n_interior, Y)
        x, u = rollout(inst, u_bar, K, disturbance(inst, w))
        worst[s] = worst_constraint(inst, x, u)
    return int(np.sum(worst <= tol)), worst
