"""GPU parity of the warm-start network (nrto_mlp_*: tcgen05 bf16 GEMMs with FP32 accumulation)
against the FP64 oracle (oracle/mlp.py).

Two comparisons per result:
- tight: against the oracle's forward/backward evaluated with the kernel's bf16 roundings applied
  at the same points (inputs, weights, hidden activations, back-propagated gradients), which leaves
  only FP32 accumulation order and the float erf/exp (bound 2e-3 norm-wise relative);
- loose: against the plain FP64 oracle with bf16-rounded parameters and inputs.  Each of the L
  layers rounds one activation (forward) and one gradient (backward) to bf16, unit roundoff
  u = 2⁻⁸, so to first order the norm-wise relative error is ≤ 2·L·u·κ with κ the amplification
  of the layer maps; at the default initialization κ ≤ 2, giving 4·L·u.
"""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2603_02642_b300 import nrto

from .gpu_common import relerr

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8
RNG = np.random.default_rng(21)


def bf16(a):
    """Round to bfloat16 (nearest, ties to even) and return float64."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def params_of(net, flat):
    W, b = net.unpack(flat.astype(np.float64))
    return M.Params([w.copy() for w in W], [bb.copy() for bb in b])


def emulated_forward(p, x):
    """Oracle forward with bf16 rounding of the input, the weights and each hidden activation."""
    h = bf16(x)
    hs, zs = [h], []
    L = len(p.W)
    for l in range(L):
        z = h @ bf16(p.W[l]).T + p.b[l]
        zs.append(z)
        if l < L - 1:
            h = bf16(M.gelu(z))
            hs.append(h)
    return z, (hs, zs)


def emulated_backward(p, cache, y, t, mask):
    """Oracle backward with the kernel's rounding points: dY and every dZ are bf16, weights bf16."""
    hs, zs = cache
    n = float(np.sum(mask))
    dz = bf16(2.0 * mask * (y - t) / n)
    L = len(p.W)
    gW, gb = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        gW[l] = dz.T @ hs[l]
        gb[l] = dz.sum(axis=0)
        if l > 0:
            dz = bf16((dz @ bf16(p.W[l])) * M.gelu_grad(zs[l - 1]))
    return gW, gb


def flat_grads(gW, gb):
    return np.concatenate([np.concatenate([w.reshape(-1), b.reshape(-1)]) for w, b in zip(gW, gb)])


def make(dims, batch, seed):
    net = nrto.MLP(dims, max_batch=max(batch, 8))
    p = M.init_params(dims, seed=seed)
    flat = np.concatenate([np.concatenate([w.reshape(-1), b]) for w, b in zip(p.W, p.b)]).astype(np.float32)
    net.set_params(flat)
    return net, params_of(net, flat)


# (dims, batch): one linear layer (raw GEMM + bias), ragged M and N tiles, the warm-start shape
SHAPES = [([64, 128], 256), ([99, 256, 136], 200), ([99, 256, 256, 256, 9400], 256)]


@pytest.mark.parametrize("dims,batch", SHAPES)
def test_forward_parity(dims, batch):
    net, p = make(dims, batch, seed=len(dims))
    x = RNG.normal(size=(batch, dims[0]))
    y = net.forward(x)
    ye, _ = emulated_forward(p, x)
    assert relerr(y, ye) < 2e-3
    pq = M.Params([bf16(w) for w in p.W], p.b)
    y64, _ = M.forward(pq, bf16(x))
    assert relerr(y, y64) < 4 * (len(dims) - 1) * U_BF16
    net.close()


@pytest.mark.parametrize("dims,batch", SHAPES)
def test_gradient_parity(dims, batch):
    net, p = make(dims, batch, seed=10 + len(dims))
    x = RNG.normal(size=(batch, dims[0]))
    t = RNG.normal(size=(batch, dims[-1]))
    mask = (RNG.uniform(size=(batch, dims[-1])) < 0.8).astype(np.float64)
    loss, g = net.train_step(x, t, mask, lr=0.0, want_grads=True)
    ye, cache = emulated_forward(p, x)
    gWe, gbe = emulated_backward(p, cache, ye, t, mask)
    assert abs(loss - M.loss(ye, t, mask)) <= 1e-3 * M.loss(ye, t, mask)
    Wg, bg = net.unpack(g.astype(np.float64))
    for l in range(len(dims) - 1):
        assert relerr(Wg[l], gWe[l]) < 2e-3, f"dW[{l}]"
        assert relerr(bg[l], gbe[l]) < 2e-3, f"db[{l}]"
    pq = M.Params([bf16(w) for w in p.W], p.b)
    y64, c64 = M.forward(pq, bf16(x))
    gW64, gb64 = M.backward(pq, c64, y64, t, mask)
    assert relerr(g, flat_grads(gW64, gb64)) < 4 * (len(dims) - 1) * U_BF16
    net.close()


def test_adam_step_matches_oracle_update():
    """One Adam step on the GPU equals the oracle's Adam applied to the GPU's own gradient."""
    dims, batch = [99, 256, 136], 64
    net, p = make(dims, batch, seed=5)
    theta0 = net.get_params().astype(np.float64)
    x = RNG.normal(size=(batch, dims[0]))
    t = RNG.normal(size=(batch, dims[-1]))
    mask = np.ones((batch, dims[-1]))
    _, g = net.train_step(x, t, mask, lr=0.0, want_grads=True)
    net.set_params(theta0.astype(np.float32))
    net.train_step(x, t, mask, lr=1e-3)
    theta1 = net.get_params().astype(np.float64)
    q = [theta0.copy()]
    M.Adam(lr=1e-3).step(q, [g.astype(np.float64)])
    assert np.abs(theta1 - q[0]).max() < 1e-6
    net.close()


def test_training_reduces_loss_on_a_teacher_network():
    """A few hundred Adam steps fit a random teacher of the same shape: the loss falls by > 10x."""
    dims, batch = [32, 256, 256, 64], 512
    teacher = M.init_params(dims, seed=99)
    x = RNG.normal(size=(batch, dims[0]))
    t, _ = M.forward(teacher, x)
    net, _ = make(dims, batch, seed=7)
    mask = np.ones_like(t)
    l0 = net.train_step(x, t, mask, lr=2e-3)
    for _ in range(300):
        l1 = net.train_step(x, t, mask, lr=2e-3)
    assert l1 < 0.1 * l0
    assert net.kernel_launches() > 0
    net.close()


def test_gemm_profile_counts_the_forward_gemms():
    dims, batch = [99, 256, 256, 256, 9400], 1024
    net, _ = make(dims, batch, seed=3)
    x = RNG.normal(size=(batch, dims[0]))
    net.profile(True)
    net.forward(x)
    ms, flops, n = net.profile(False)
    assert n == len(dims) - 1 and ms > 0
    assert flops == 2.0 * batch * sum(a * b for a, b in zip([104] + dims[1:-1], dims[1:]))
    net.close()
