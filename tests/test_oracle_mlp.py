"""Pins for the FP64 reference of the warm-start network (oracle/mlp.py)."""
import numpy as np
import scipy.special

from oracle import mlp as M

RNG = np.random.default_rng(3)


def test_gelu_against_independent_normal_cdf_and_symmetry():
    z = np.linspace(-6, 6, 241)
    assert np.allclose(M.gelu(z), z * scipy.special.ndtr(z), rtol=1e-14, atol=1e-15)
    # Φ(-z) = 1 - Φ(z)  ⇒  gelu(-z) = gelu(z) - z
    assert np.allclose(M.gelu(-z), M.gelu(z) - z, atol=1e-14)
    assert M.gelu(np.array([0.0]))[0] == 0.0 and M.gelu_grad(np.array([0.0]))[0] == 0.5


def test_gelu_grad_by_central_differences():
    z = np.linspace(-5, 5, 101)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.allclose(M.gelu_grad(z), fd, atol=1e-9)


def test_backward_by_central_differences():
    dims = [5, 7, 6, 4]
    p = M.init_params(dims, seed=1)
    x = RNG.normal(size=(9, 5))
    t = RNG.normal(size=(9, 4))
    mask = (RNG.uniform(size=(9, 4)) < 0.7).astype(float)
    y, cache = M.forward(p, x)
    gW, gb = M.backward(p, cache, y, t, mask)
    h = 1e-6

    def f():
        return M.loss(M.forward(p, x)[0], t, mask)

    for l in range(len(dims) - 1):
        for arr, g in ((p.W[l], gW[l]), (p.b[l], gb[l])):
            fd = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + h
                fp = f()
                arr[idx] = old - h
                fm = f()
                arr[idx] = old
                fd[idx] = (fp - fm) / (2 * h)
            assert np.linalg.norm(g - fd) <= 1e-6 * max(np.linalg.norm(fd), 1e-12)


def test_single_linear_layer_gradient_vanishes_at_least_squares():
    """One linear layer, full mask: the gradient is zero exactly at the least-squares fit (a
    library least-squares solve, independent of the network code) and not elsewhere."""
    x = RNG.normal(size=(40, 6))
    t = RNG.normal(size=(40, 3))
    xa = np.hstack([x, np.ones((40, 1))])
    sol, *_ = np.linalg.lstsq(xa, t, rcond=None)
    p = M.Params([sol[:6].T.copy()], [sol[6].copy()])
    mask = np.ones_like(t)
    y, cache = M.forward(p, x)
    gW, gb = M.backward(p, cache, y, t, mask)
    assert np.abs(gW[0]).max() < 1e-12 and np.abs(gb[0]).max() < 1e-12
    p.W[0][0, 0] += 0.1
    y, cache = M.forward(p, x)
    gW, _ = M.backward(p, cache, y, t, mask)
    assert gW[0][0, 0] > 1e-3


def test_adam_first_step_moves_by_lr_times_sign():
    """At t = 1 the bias-corrected moments are m̂ = g and v̂ = g², so θ moves by -lr g/(|g| + ε)."""
    q = [RNG.normal(size=(4, 3))]
    g = [RNG.normal(size=(4, 3))]
    q0 = q[0].copy()
    opt = M.Adam(lr=1e-2, eps=1e-8)
    opt.step(q, g)
    assert np.allclose(q[0], q0 - 1e-2 * g[0] / (np.abs(g[0]) + 1e-8), atol=1e-15)
