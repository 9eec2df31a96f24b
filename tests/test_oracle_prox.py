"""Pins of the oracle's proximity operators (Eqs. 21-24, l1-ball projection).

Each projection P onto a closed convex set C is checked by its defining
variational inequality, <x - P(x), z - P(x)> <= 0 for every z in C: for the
l1 ball it is enough to test the 2n vertices +-r e_k (the ball is their convex
hull), which makes the check exact at any size.  The l1 projection is also
checked against brute-force enumeration of active sets on small vectors, and
the group prox (Eq. 24) against Moreau's identity (Eq. 3) with an independent
projection onto the unit disc.
"""
import itertools

import numpy as np
import pytest

from oracle import ppds as o


def _vertex_check(x, p, r, tol=1e-10):
    assert np.abs(p).sum() <= r * (1 + 1e-12) + 1e-14
    g = x - p
    # <g, z - p> for z = +-r e_k
    lhs = np.concatenate([r * g - np.vdot(g, p), -r * g - np.vdot(g, p)])
    assert lhs.max() <= tol * max(1.0, np.abs(x).max() * r)


def _brute_l1(x, r):
    a = np.abs(x)
    if a.sum() <= r:
        return x.copy()
    if r == 0:
        return np.zeros_like(x)
    n = x.size
    for k in range(1, n + 1):
        for S in itertools.combinations(range(n), k):
            S = list(S)
            tau = (a[S].sum() - r) / k
            rest = np.setdiff1d(np.arange(n), S)
            if tau < 0:
                continue
            if a[S].min() > tau and (rest.size == 0 or a[rest].max() <= tau + 1e-15):
                return np.sign(x) * np.maximum(a - tau, 0.0)
    raise AssertionError("no active set found")


@pytest.mark.parametrize("seed", range(12))
def test_l1_projection_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 10))
    x = rng.standard_normal(n) * rng.uniform(0.1, 3)
    r = float(rng.uniform(0.0, 1.2) * np.abs(x).sum())
    p, tau = o.proj_l1ball(x, r)
    np.testing.assert_allclose(p, _brute_l1(x, r), rtol=1e-12, atol=1e-14)
    _vertex_check(x, p, r)


@pytest.mark.parametrize("n", [1, 7, 1000, 100_000])
def test_l1_projection_variational(n):
    rng = np.random.default_rng(n)
    x = rng.laplace(size=n)
    r = 0.3 * np.abs(x).sum()
    p, tau = o.proj_l1ball(x, r)
    assert np.abs(p).sum() == pytest.approx(r, rel=1e-12)
    assert tau > 0
    # same sign pattern, soft-threshold form
    np.testing.assert_array_equal(np.sign(p)[p != 0], np.sign(x)[p != 0])
    _vertex_check(x, p, r, tol=1e-9)


def test_l1_projection_edge_cases():
    x = np.array([0.5, -0.25, 0.0, 0.125])
    # inside the ball: identity, tau = 0
    p, tau = o.proj_l1ball(x, 1.0)
    np.testing.assert_array_equal(p, x)
    assert tau == 0.0
    # on the sphere exactly: identity
    p, tau = o.proj_l1ball(x, 0.875)
    np.testing.assert_array_equal(p, x)
    # radius 0: the ball is {0}
    p, tau = o.proj_l1ball(x, 0.0)
    np.testing.assert_array_equal(p, np.zeros(4))
    # all zeros
    p, tau = o.proj_l1ball(np.zeros(5), 0.0)
    np.testing.assert_array_equal(p, np.zeros(5))
    # ties: equal magnitudes are shrunk equally
    x = np.array([1.0, -1.0, 1.0, 0.5, -0.5])
    p, tau = o.proj_l1ball(x, 1.5)
    np.testing.assert_allclose(p, [0.5, -0.5, 0.5, 0.0, 0.0], atol=1e-15)
    assert tau == pytest.approx(0.5)
    _vertex_check(x, p, 1.5)


@pytest.mark.parametrize("seed", range(5))
def test_l2_ball_projection(seed):
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(50)
    x = c + rng.standard_normal(50) * 3
    eps = 2.0
    p = o.proj_l2ball(x, c, eps)
    assert np.linalg.norm(p - c) == pytest.approx(eps, rel=1e-13)
    # P - c is a positive multiple of x - c
    cos = np.vdot(p - c, x - c) / (np.linalg.norm(p - c) * np.linalg.norm(x - c))
    assert cos == pytest.approx(1.0, abs=1e-13)
    # variational inequality against random points of the ball
    for _ in range(200):
        z = rng.standard_normal(50)
        z = c + z / np.linalg.norm(z) * eps * rng.uniform() ** (1 / 50)
        assert np.vdot(x - p, z - p) <= 1e-10
    # inside: identity; eps = 0: the centre
    np.testing.assert_array_equal(o.proj_l2ball(c + 0.1, c, 10.0), c + 0.1)
    np.testing.assert_allclose(o.proj_l2ball(x, c, 0.0), c)


def test_box_projection():
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 2, size=1000)
    p = o.proj_box(x, 0.0, 1.0)
    for _ in range(50):
        z = rng.uniform(0, 1, size=1000)
        assert np.vdot(x - p, z - p) <= 1e-12


def _proj_unit_discs(z):
    """Projection of each 2-vector group onto the unit disc (independent code)."""
    out = z.copy()
    for idx in np.ndindex(z.shape[0], *z.shape[2:]):
        g, rest = idx[0], idx[1:]
        a, b = z[(g, 0) + rest], z[(g, 1) + rest]
        n = (a * a + b * b) ** 0.5
        if n > 1:
            out[(g, 0) + rest] = a / n
            out[(g, 1) + rest] = b / n
    return out


@pytest.mark.parametrize("gamma", [0.05, 0.25, 1.0])
def test_group_prox_moreau(gamma):
    """Eq. 3 with f = ||.||_{1,2}: f* is the indicator of the unit discs, so
    x = prox_{gamma f}(x) + gamma P_discs(x / gamma)."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 2, 2, 3, 4)) * 0.5
    p = o.prox_l12(x, gamma)
    np.testing.assert_allclose(p + gamma * _proj_unit_discs(x / gamma), x, atol=1e-14)


def test_group_prox_minimises():
    """Eq. 1: prox minimises f(z) + ||x - z||^2 / (2 gamma)."""
    rng = np.random.default_rng(2)
    gamma = 0.3
    x = rng.standard_normal((1, 2, 40))
    x[:, :, :5] *= 0.05          # some groups below the threshold
    p = o.prox_l12(x, gamma)

    def obj(z):
        return np.sqrt(z[:, 0] ** 2 + z[:, 1] ** 2).sum() + ((x - z) ** 2).sum() / (2 * gamma)

    base = obj(p)
    for _ in range(300):
        assert obj(p + rng.standard_normal(p.shape) * 1e-3) >= base - 1e-15
    assert np.all(p[:, :, :5] == 0)
    # zero group maps to zero
    assert np.all(o.prox_l12(np.zeros((3, 2, 4)), 0.1) == 0)
