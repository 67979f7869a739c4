"""Learned warm start for the FullADMM inner solve of the quadcopter workload (T = 100, up to 15
spherical obstacles).

The paper names learning a warm start as future work; this module is the library's version.
A GELU MLP (nrto.MLP: tcgen05 kernels) maps an instance's parameters to the inner solver's initial
(k_v, p̃, λ_p), with λ_ν starting at zero (so ν = Π(Â k + b̂)), or, in the lifted layout, to the
whole state of the lifted iteration.  Training targets are the converged iterates of the
cold-started solver at the first outer step.

Layouts (fixed; obstacles padded to 15 and masked):
  features (99) = x̄_0 (12) | goal (12) | 15 × (centre (3), radius) | obstacle mask (15)
  outputs (9400) = K (T·n_u·n_x = 4800, the library's [m][u][c] layout)
                 | p̃ (2300) | λ_p (2300), each over rows: state rows (t-1)·15 + o, then the 800
                   control-bound rows in the library's order (step k, input i, upper before lower).
  lifted outputs (15608) = the 9400 above | θ (2300) | λ_w (2300) over the same rows | δû (T·n_u)
                 | λ_e (T·n_x, steps 1..T) | log ρ | 7 unused: the rest of the lifted iteration's state
                   (nrto_set_warm_start_lifted), with λ_ν = θ (Â k + b̂) and θ = 1/s - 1 from the
                   rows' projection scales.
The feature standardization and the target scaling learned on the training set are folded into the
first and last layers, so the deployed network maps raw features to raw solver values.  This module
only arranges data; every arithmetic step of training and inference runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import nrto

T, NX, NU, N_OBS_MAX = 100, 12, 4, 15
N_K = T * NU * NX
N_STATE = T * N_OBS_MAX
N_CTRL = T * NU * 2
N_ROWS = N_STATE + N_CTRL
N_OUT = N_K + 2 * N_ROWS
N_IN = 12 + 12 + 4 * N_OBS_MAX + N_OBS_MAX
DIMS = [N_IN, 256, 256, 256, N_OUT]
# lifted layout: offsets of θ, λ_w, δû, λ_e, log ρ after the plain outputs
O_TH, O_LW = N_OUT, N_OUT + N_ROWS
O_DU = N_OUT + 2 * N_ROWS
O_LE = O_DU + T * NU
O_RHO = O_LE + T * NX
N_OUT_LIFTED = (O_RHO + 1 + 7) // 8 * 8   # the network's widths are multiples of 8 (7 unused outputs)
DIMS_LIFTED = [N_IN, 256, 256, 256, N_OUT_LIFTED]
THETA_MAX = 100.0   # targets θ = 1/s - 1 clipped (a row projected almost to zero)


def _check_inst(inst):
    if inst.kind != 1 or inst.T != T or inst.n_obs > N_OBS_MAX or np.isfinite(inst.x_lo).any() \
            or np.isfinite(inst.x_hi).any() or not (np.isfinite(inst.u_lo).all() and np.isfinite(inst.u_hi).all()):
        raise ValueError("warm start covers quadcopter instances with T = 100, <= 15 obstacles and full control bounds")


def features(insts):
    out = np.zeros((len(insts), N_IN), dtype=np.float32)
    for i, inst in enumerate(insts):
        _check_inst(inst)
        f = out[i]
        f[0:12] = inst.x0
        f[12:24] = inst.x_goal
        for o in range(inst.n_obs):
            f[24 + 4 * o:24 + 4 * o + 3] = inst.obs_center[o]
            f[24 + 4 * o + 3] = inst.obs_radius[o]
            f[24 + 4 * N_OBS_MAX + o] = 1.0
    return out


def row_index(inst):
    """Network row index of each of the instance's constraint rows (library order)."""
    _check_inst(inst)
    t = np.repeat(np.arange(1, T + 1), inst.n_obs)
    o = np.tile(np.arange(inst.n_obs), T)
    state = (t - 1) * N_OBS_MAX + o
    ctrl = N_STATE + np.arange(N_CTRL)
    return np.concatenate([state, ctrl])


def collect_targets(prob, insts, statuses, lifted=False):
    """(features, targets, masks) of the instances whose inner solve converged (status 1); with
    `lifted`, the lifted layout's targets as well (θ from the projection scales, the final ρ)."""
    keep = [i for i in range(len(insts)) if statuses[i] == 1]
    X = features([insts[i] for i in keep])
    n_out = N_OUT_LIFTED if lifted else N_OUT
    Y = np.zeros((len(keep), n_out), dtype=np.float32)
    Mk = np.zeros((len(keep), n_out), dtype=np.float32)
    rho = prob.stats()["rho"] if lifted else None
    for r, i in enumerate(keep):
        idx = row_index(insts[i])
        Y[r, :N_K] = prob.export(nrto.F_K, i)
        Mk[r, :N_K] = 1.0
        Y[r, N_K + idx] = prob.export(nrto.F_PT, i)
        Y[r, N_K + N_ROWS + idx] = prob.export(nrto.F_LAMP, i)
        Mk[r, N_K + idx] = 1.0
        Mk[r, N_K + N_ROWS + idx] = 1.0
        if lifted:
            sc = prob.export(nrto.F_S, i)
            th = np.where(sc > 0.0, 1.0 / np.where(sc > 0.0, sc, 1.0) - 1.0, 0.0)
            Y[r, O_TH + idx] = np.clip(th, 0.0, THETA_MAX)
            Y[r, O_LW + idx] = prob.export(nrto.F_LAMW, i)
            Y[r, O_DU:O_DU + T * NU] = prob.export(nrto.F_DU, i)
            Y[r, O_LE:O_LE + T * NX] = prob.export(nrto.F_LAME, i)[NX:]
            Y[r, O_RHO] = np.log(rho[i])
            Mk[r, O_TH + idx] = 1.0
            Mk[r, O_LW + idx] = 1.0
            Mk[r, O_DU:O_RHO + 1] = 1.0
    return X, Y, Mk


class WarmStart:
    """Train and apply the warm-start network."""

    def __init__(self, max_batch=4096, seed=0, stream=None, lifted=False):
        self.lifted = lifted
        dims = DIMS_LIFTED if lifted else DIMS
        self.n_out = dims[-1]
        self.net = nrto.MLP(dims, max_batch=max_batch, stream=stream)
        rng = np.random.default_rng(seed)
        flat = []
        for din, dout in zip(dims[:-1], dims[1:]):
            s = 1.0 / np.sqrt(din)
            flat.append(rng.uniform(-s, s, size=dout * din))
            flat.append(rng.uniform(-s, s, size=dout))
        self.net.set_params(np.concatenate(flat).astype(np.float32))
        self.x_mu = np.zeros(N_IN)
        self.x_sd = np.ones(N_IN)
        self.y_mu = np.zeros(self.n_out)
        self.y_sd = np.ones(self.n_out)
        self.deployed = False

    def fit(self, X, Y, Mk, steps=2000, batch=256, lr=1e-3, seed=0):
        """Adam on the standardized data; returns the loss history."""
        X = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float32)
        Mk32 = np.asarray(Mk, dtype=np.float32)
        self.x_mu = X.mean(axis=0)
        self.x_sd = X.std(axis=0)
        self.x_sd[self.x_sd < 1e-6] = 1.0
        # target statistics in FP64, over row blocks (the target matrix can be several GB)
        blocks = range(0, Y.shape[0], 4096)
        cnt = np.maximum(sum(Mk32[b:b + 4096].astype(np.float64).sum(axis=0) for b in blocks), 1.0)
        self.y_mu = sum((Mk32[b:b + 4096] * Y[b:b + 4096]).astype(np.float64).sum(axis=0) for b in blocks) / cnt
        self.y_sd = np.sqrt(sum((Mk32[b:b + 4096] * (Y[b:b + 4096] - self.y_mu) ** 2).sum(axis=0) for b in blocks) / cnt)
        self.y_sd[self.y_sd < 1e-6] = 1.0
        Xn = ((X - self.x_mu) / self.x_sd).astype(np.float32)
        Yn = np.empty_like(Y)
        for b in blocks:
            Yn[b:b + 4096] = (Mk32[b:b + 4096] * (Y[b:b + 4096] - self.y_mu) / self.y_sd).astype(np.float32)
        rng = np.random.default_rng(seed)
        n = X.shape[0]
        batch = min(batch, (n // 8) * 8)
        hist = []
        for s in range(steps):
            idx = rng.choice(n, size=batch, replace=False)
            hist.append(self.net.train_step(Xn[idx], Yn[idx], Mk32[idx], lr))
        self._deploy()
        return hist

    def _deploy(self):
        """Fold the feature standardization into layer 1 and the target scaling into the last layer."""
        W, b = self.net.unpack(self.net.get_params().astype(np.float64))
        W[0] = W[0] / self.x_sd[None, :]
        b[0] = b[0] - W[0] @ self.x_mu
        W[-1] = W[-1] * self.y_sd[:, None]
        b[-1] = b[-1] * self.y_sd + self.y_mu
        self.net.set_params(self.net.pack(W, b))
        self.deployed = True

    def predict(self, insts):
        """Per-instance (K (T, n_u, n_x), p̃ (n_rows), λ_p (n_rows)) for the instances' own rows."""
        if not self.deployed:
            raise RuntimeError("fit() the network first")
        Ys = []
        for s in range(0, len(insts), self.net.max_batch):
            Ys.append(self.net.forward(features(insts[s:s + self.net.max_batch])))
        Y = np.concatenate(Ys).astype(np.float64)
        out = []
        for i, inst in enumerate(insts):
            idx = row_index(inst)
            o = (Y[i, :N_K].reshape(T, NU, NX), Y[i, N_K + idx], Y[i, N_K + N_ROWS + idx])
            if self.lifted:
                o = o + (np.maximum(Y[i, O_TH + idx], 0.0), Y[i, O_LW + idx], Y[i, O_DU:O_DU + T * NU].reshape(T, NU),
                         Y[i, O_LE:O_LE + T * NX].reshape(T, NX), float(np.exp(Y[i, O_RHO])))
            out.append(o)
        return out

    # Lifted parts applied by default: δû only.  Measured on 512 held-out instances after 2048
    # training solves (mean iterations relative to cold on the instances every variant solved):
    # (k_v, p̃, λ_p) 0.78, + δû 0.68, + δû and θ or λ_w 0.69, + δû and λ_e 0.88, all parts 0.88 with
    # the duals rescaled to the start penalty and 1.11 at the predicted penalty; the predicted λ_e
    # and penalty cost more than they save.
    LIFTED_PARTS = ("du",)

    def apply(self, prob, insts, lifted=None, parts=None):
        """Install the network's warm start for the problem's next inner solve: the forward pass and
        the scatter into each instance's (K, p̃, λ_p), and with the lifted layout (unless lifted is
        False) the lifted parts named in `parts` (of "th", "lw", "du", "le", "rho"; default
        LIFTED_PARTS), run on the device."""
        if not self.deployed:
            raise RuntimeError("fit() the network first")
        row_map = np.concatenate([row_index(inst) for inst in insts]).astype(np.int32)
        if self.lifted and lifted is not False:
            use = self.LIFTED_PARTS if parts is None else parts
            off = {"th": O_TH, "lw": O_LW, "du": O_DU, "le": O_LE, "rho": O_RHO}
            prob.set_warm_start_from_network_lifted(self.net, features(insts), row_map,
                                                    [0, N_K, N_K + N_ROWS] + [off[k] if k in use else -1
                                                                              for k in ("th", "lw", "du", "le", "rho")])
        else:
            prob.set_warm_start_from_network(self.net, features(insts), row_map, 0, N_K, N_K + N_ROWS)

    def apply_host(self, prob, insts, parts=None):
        """Same warm start through host arrays (predict, then nrto_set_warm_start and, with the lifted
        layout, nrto_set_warm_start_lifted with the parts not applied set to zero)."""
        pred = self.predict(insts)
        K = np.concatenate([p[0].reshape(-1) for p in pred])
        pt = np.concatenate([p[1] for p in pred])
        lp = np.concatenate([p[2] for p in pred])
        prob.set_warm_start(K, pt, lp)
        if self.lifted:
            use = self.LIFTED_PARTS if parts is None else parts
            pick = lambda k, j: [p[j] if k in use else 0.0 * p[j] for p in pred]
            prob.set_warm_start_lifted(pick("th", 3), pick("lw", 4), pick("du", 5), pick("le", 6),
                                       [p[7] for p in pred] if "rho" in use else None)
        return pred
