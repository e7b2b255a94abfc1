"""Pins of the exploration oracle (oracle/explore.py) against what the definitions fix: the identity map, the
map's Jacobian from its own intervals, the mixture of densities by a linear scan, and unbiasedness of the
balance-heuristic weights for a closed-form integral."""
import math

import numpy as np
import pytest

import oracle as orc
from oracle import explore as X
from paper_2408_09229_gb300 import workloads as W


def random_map(rng, d, G):
    e = np.empty((d, G + 1))
    for a in range(d):
        w = rng.exponential(1.0, G) + 0.05
        e[a] = np.concatenate([[0.0], np.cumsum(w) / w.sum()])
        e[a, -1] = 1.0
    return e


def test_uniforms_layout_and_range():
    y8 = X.uniforms(12345, 77, 8)
    assert np.array_equal(X.uniforms(12345, 77, 4), y8[:4])  # axes 0-3 from the first call
    assert np.all((y8 > 0) & (y8 < 1))
    u = orc.philox4x32_10([77, 0, 4, X.TAG], [12345, 0])
    assert y8[4] == (float(u[0]) + 0.5) * 2.0 ** -32  # axes 4-7 from the counter's third word = 4
    ys = np.array([X.uniforms(9, r, 4) for r in range(4000)])
    assert abs(ys.mean() - 0.5) < 5 * math.sqrt(1 / 12 / ys.size)


def test_uniform_map_is_the_identity():
    G, d = 16, 3
    e = np.tile(np.linspace(0.0, 1.0, G + 1), (d, 1))
    rng = np.random.default_rng(1)
    for _ in range(100):
        y = rng.random(d)
        assert np.allclose(X.map_point(e, y), y, rtol=0, atol=1e-15)
        assert X.map_density(e, X.map_point(e, y)) == pytest.approx(1.0, rel=1e-12)


def test_density_is_the_inverse_jacobian_of_the_sample():
    rng = np.random.default_rng(2)
    d, G = 4, 12
    e = random_map(rng, d, G)
    for _ in range(200):
        y = rng.random(d)
        i = np.minimum((y * G).astype(int), G - 1)
        J = np.prod([G * (e[a, i[a] + 1] - e[a, i[a]]) for a in range(d)])
        assert X.map_density(e, X.map_point(e, y)) * J == pytest.approx(1.0, rel=1e-12)


def test_mixture_by_linear_scan():
    rng = np.random.default_rng(3)
    d, G = 3, 10
    maps = [random_map(rng, d, G) for _ in range(3)]

    def dens_scan(E, x):
        q = 1.0
        for a in range(d):
            j = max(k for k in range(G) if E[a, k] <= x[a])
            q /= G * (E[a, j + 1] - E[a, j])
        return q

    for _ in range(100):
        x = rng.random(d)
        assert X.mixture_density(maps, x) == pytest.approx(sum(dens_scan(E, x) for E in maps) / 3, rel=1e-12)


def test_balance_weights_are_unbiased():
    """samples of three different maps, r mod 3, weighted |f| / q_mix: their mean is the integral (a Gaussian in
    d = 3 with its closed form), within 5 standard errors"""
    rng = np.random.default_rng(4)
    d, G = 3, 20
    maps = [random_map(rng, d, G) for _ in range(3)]
    params = W.gaussian(d, 0.4, 0.1)
    xs, q = X.explore_points(maps, 3000, 2024)
    w = X.weights(orc.GAUSS_SUM, params, xs, q)
    exact = W.exact(W.GAUSS_SUM, d, params)
    assert abs(w.mean() - exact) < 5 * w.std() / math.sqrt(w.size), (w.mean(), exact)
