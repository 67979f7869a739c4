"""FP64 reference of the learned warm-start network (oracle; test infrastructure only).

The paper names learning a warm start for the inner solver as future work and fixes no network.
The network here is a plain multilayer perceptron with GELU hidden layers:

    h_0 = x,   z_l = h_{l-1} W_lᵀ + b_l,   h_l = gelu(z_l)  (l < L),   y = z_L,
    gelu(z) = z Φ(z) = ½ z (1 + erf(z / √2)),

trained on the masked mean-squared error

    loss = Σ_{m,n} mask_{m,n} (y_{m,n} - t_{m,n})² / Σ_{m,n} mask_{m,n}

with Adam (bias-corrected first and second moments) on the parameters.  Weights W_l are stored
(out, in), as z = h Wᵀ.  Everything here is float64 NumPy, written from these definitions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_SQRT2 = math.sqrt(2.0)
_INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)
_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(z):
    """z Φ(z) with the exact error function."""
    return 0.5 * z * (1.0 + _erf(z / _SQRT2))


def gelu_grad(z):
    """d/dz [z Φ(z)] = Φ(z) + z φ(z)."""
    return 0.5 * (1.0 + _erf(z / _SQRT2)) + z * _INV_SQRT_2PI * np.exp(-0.5 * z * z)


@dataclass
class Params:
    W: list          # W[l]: (d_{l+1}, d_l)
    b: list          # b[l]: (d_{l+1},)

    @property
    def dims(self):
        return [self.W[0].shape[1]] + [w.shape[0] for w in self.W]


def init_params(dims, seed=0):
    """Uniform(-1/√fan_in, 1/√fan_in) weights and biases (the common default for linear layers)."""
    rng = np.random.default_rng(seed)
    W, b = [], []
    for din, dout in zip(dims[:-1], dims[1:]):
        s = 1.0 / math.sqrt(din)
        W.append(rng.uniform(-s, s, size=(dout, din)))
        b.append(rng.uniform(-s, s, size=dout))
    return Params(W, b)


def forward(p: Params, x):
    """Returns (y, cache) with cache = (h_0..h_{L-1}, z_1..z_L)."""
    hs, zs = [x], []
    h = x
    L = len(p.W)
    for l in range(L):
        z = h @ p.W[l].T + p.b[l]
        zs.append(z)
        h = gelu(z) if l < L - 1 else z
        if l < L - 1:
            hs.append(h)
    return h, (hs, zs)


def loss(y, t, mask):
    n = float(np.sum(mask))
    return float(np.sum(mask * (y - t) ** 2) / n)


def backward(p: Params, cache, y, t, mask):
    """Gradients of the masked MSE w.r.t. W_l and b_l by the chain rule, layer by layer."""
    hs, zs = cache
    n = float(np.sum(mask))
    dz = 2.0 * mask * (y - t) / n
    L = len(p.W)
    gW, gb = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        gW[l] = dz.T @ hs[l]
        gb[l] = dz.sum(axis=0)
        if l > 0:
            dh = dz @ p.W[l]
            dz = dh * gelu_grad(zs[l - 1])
    return gW, gb


@dataclass
class Adam:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    t: int = 0
    m: list = field(default_factory=list)
    v: list = field(default_factory=list)

    def step(self, params: list, grads: list):
        """In place: m ← β₁m + (1-β₁)g, v ← β₂v + (1-β₂)g², θ ← θ - lr m̂/(√v̂ + ε),
        m̂ = m/(1-β₁ᵗ), v̂ = v/(1-β₂ᵗ)."""
        if not self.m:
            self.m = [np.zeros_like(q) for q in params]
            self.v = [np.zeros_like(q) for q in params]
        self.t += 1
        c1 = 1.0 - self.beta1 ** self.t
        c2 = 1.0 - self.beta2 ** self.t
        for q, g, m, v in zip(params, grads, self.m, self.v):
            m *= self.beta1
            m += (1.0 - self.beta1) * g
            v *= self.beta2
            v += (1.0 - self.beta2) * g * g
            q -= self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps)


def flat(p: Params):
    return [*p.W, *p.b]
