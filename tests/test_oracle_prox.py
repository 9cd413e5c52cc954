"""Pins for the oracle's proximal operators (closed forms, Moreau identity, optimality)."""

import numpy as np
import pytest

import synth
from oracle import prox


def test_soft_threshold_closed_form_real():
    x = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 1.5, 4.0])
    out = prox.soft_threshold(x, 1.0)
    assert np.array_equal(out, np.array([-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.5, 3.0]))  # |x| = lambda -> 0


def test_soft_threshold_complex_radial():
    x = np.array([3 + 4j, 0.3 - 0.4j, 0j])
    out = prox.soft_threshold(x, 1.0)
    assert out[0] == pytest.approx((3 + 4j) * 4 / 5)
    assert out[1] == 0 and out[2] == 0


def test_soft_threshold_minimises_objective_bruteforce():
    rng = np.random.default_rng(0)
    x = rng.normal(0, 2, 50)
    lam = 0.7
    grid = np.linspace(-10, 10, 200001)
    for xi, si in zip(x, prox.soft_threshold(x, lam)):
        obj = lam * np.abs(grid) + 0.5 * (grid - xi) ** 2
        assert si == pytest.approx(grid[np.argmin(obj)], abs=2e-4)


@pytest.mark.parametrize("sigma", [0.3, 1.0, 7.0])
def test_moreau_decomposition(sigma):
    # prox_{sigma f*}(z) + sigma prox_{f/sigma}(z/sigma) = z for f = lambda ||.||_1:
    # f* is the indicator of the l-inf ball of radius lambda, whose prox is the clip.
    lam = 0.8
    z = synth.normal(1000, seed=1) * 3
    lhs = prox.clip_linf(z, lam) + sigma * prox.soft_threshold(z / sigma, lam / sigma)
    assert np.allclose(lhs, z, rtol=0, atol=1e-14)
    assert np.allclose(prox.clip_linf(z, lam), np.clip(z, -lam, lam), rtol=0, atol=1e-15)


def test_proj_positive():
    x = np.array([-1.0, 0.0, 2.5])
    assert np.array_equal(prox.proj_positive(x), np.array([0.0, 0.0, 2.5]))


def test_proj_l2ball_inside_boundary_outside():
    c = synth.normal(64, seed=2) + 1j * synth.normal(64, seed=3)
    d = synth.normal(64, seed=4) + 1j * synth.normal(64, seed=5)
    nd = np.linalg.norm(d)
    out, nrm = prox.proj_l2ball(c + d, c, 2 * nd)            # inside: unchanged
    assert np.array_equal(out, c + d) and nrm == pytest.approx(nd)
    out, _ = prox.proj_l2ball(c + d, c, nd)                  # on the sphere: unchanged ("<=" branch)
    assert np.allclose(out, c + d)
    out, _ = prox.proj_l2ball(c + d, c, 0.25 * nd)           # outside: radial scaling onto the sphere
    assert np.linalg.norm(out - c) == pytest.approx(0.25 * nd, rel=1e-14)
    assert np.allclose(out - c, 0.25 * d)


def test_proj_l2ball_is_the_nearest_point():
    # variational inequality Re <x - P(x), v - P(x)> <= 0 for every v in the ball
    rng = np.random.default_rng(7)
    c = rng.normal(size=20)
    x = c + rng.normal(size=20) * 5
    eps = 1.5
    p, _ = prox.proj_l2ball(x, c, eps)
    for _ in range(500):
        v = rng.normal(size=20)
        v = c + v / np.linalg.norm(v) * eps * rng.uniform() ** (1 / 20)
        assert np.dot(x - p, v - p) <= 1e-12
