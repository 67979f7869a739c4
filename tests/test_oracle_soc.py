"""Pins for the oracle's SOC projection (Supplementary Sec. II-C, Fig. 3)."""
import numpy as np
import pytest

from oracle import soc

RNG = np.random.default_rng(1234)


def test_three_cases_of_fig3():
    # Left panel: inside the cone → unchanged.
    t, e = soc.project(2.0, np.array([0.6, 0.8]))
    assert t == 2.0 and np.allclose(e, [0.6, 0.8])
    # Right panel: inside the polar cone (‖η‖ ≤ -t) → origin.
    t, e = soc.project(-2.0, np.array([0.6, 0.8]))
    assert t == 0.0 and np.all(e == 0)
    # Middle panel: outside both → onto the boundary, direction of η kept.
    t, e = soc.project(1.0, np.array([3.0, 4.0]))
    assert np.isclose(t, np.linalg.norm(e)) and np.allclose(e / np.linalg.norm(e), [0.6, 0.8])


@pytest.mark.parametrize("n", [1, 3, 12, 37])
def test_projection_invariants(n):
    for _ in range(200):
        rt = RNG.normal() * 3
        re = RNG.normal(size=n) * RNG.uniform(0.1, 3)
        t, e = soc.project(rt, re)
        # In the cone.
        assert np.linalg.norm(e) <= t + 1e-12
        # Idempotent.
        t2, e2 = soc.project(t, e)
        assert np.isclose(t2, t, atol=1e-13) and np.allclose(e2, e, atol=1e-13)
        # Moreau decomposition for the self-dual SOC: x = Π_K(x) - Π_K(-x), and the two
        # parts are orthogonal.
        tn, en = soc.project(-rt, -re)
        assert np.isclose(t - tn, rt, atol=1e-12) and np.allclose(e - en, re, atol=1e-12)
        assert abs(t * tn + e @ en) <= 1e-10 * (1 + abs(rt) + np.linalg.norm(re)) ** 2


def test_projection_is_nearest_point_brute_force():
    # No sampled cone point may be closer to x than Π_K(x).
    for _ in range(50):
        n = int(RNG.integers(1, 6))
        rt = RNG.normal() * 2
        re = RNG.normal(size=n) * 2
        t, e = soc.project(rt, re)
        d0 = (t - rt) ** 2 + np.sum((e - re) ** 2)
        dirs = RNG.normal(size=(4000, n))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        rad = RNG.uniform(0, 1, size=(4000, 1)) ** 0.5
        tt = RNG.uniform(0, 6, size=4000)
        pts = dirs * rad * tt[:, None]
        d = (tt - rt) ** 2 + np.sum((pts - re) ** 2, axis=1)
        assert d0 <= d.min() + 1e-12


def test_ball_projection():
    v = RNG.normal(size=20)
    r = 0.5 * np.linalg.norm(v)
    e = soc.project_ball(v, r)
    assert np.isclose(np.linalg.norm(e), r) and np.allclose(e / r, v / np.linalg.norm(v))
    assert np.all(soc.project_ball(v, 10 * r) == v)
