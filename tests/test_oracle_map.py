"""Pins of the oracle's map refinement (Sec. 2.1.1: "refined through the
iterations varying the interval sizes, controlled by a damping parameter
alpha"; Algorithm 1 adjustWeights / updateMap; readings R6-R8).

* a worked example at N_g = 4 whose smoothed weights are derived by hand
  (below) and whose new edges come from an independent inverse-CDF
  interpolation (numpy.interp), not from the oracle's interval walk;
* special cases: alpha = 0, uniform weights, zero or non-finite weights
  leave the map unchanged;
* invariants: end points fixed, edges strictly increasing;
* the inverse-CDF property on random weights: the piecewise-linear cumulative
  damped weight takes the values j * total / N_g at the new edges.
"""
import math

import numpy as np
import pytest


def _damp(r, alpha):
    # the damping of reading R7: ((1 - r) / ln(1/r))^alpha, 0 at r = 0
    return 0.0 if r == 0 else ((1 - r) / math.log(1 / r)) ** alpha


def test_worked_example_ng4(orc):
    # w = (0, 0, 8, 0).  Smoothing (7,1)/8 - (1,6,1)/8 - (1,7)/8 by hand:
    #   ws0 = (7*0 + 0)/8 = 0, ws1 = (0 + 0 + 8)/8 = 1, ws2 = (0 + 48 + 0)/8 = 6,
    #   ws3 = (8 + 7*0)/8 = 1;  sum = 8  ->  r = (0, 1/8, 3/4, 1/8)
    r = [0.0, 1 / 8, 3 / 4, 1 / 8]
    edges = np.array([0.0, 0.1, 0.5, 0.6, 1.0])
    for alpha in (0.5, 1.0, 1.5):
        m = np.array([_damp(x, alpha) for x in r])
        cum = np.concatenate([[0.0], np.cumsum(m)])
        targets = np.arange(1, 4) * cum[-1] / 4
        want = np.interp(targets, cum, edges)
        got, unchanged = orc.refine_axis([0.0, 0.0, 8.0, 0.0], edges, alpha)
        assert not unchanged
        assert got[0] == 0.0 and got[4] == 1.0
        assert np.allclose(got[1:4], want, rtol=0, atol=1e-15)
    # alpha = 1 numbers: m = (0, 0.875/ln 8, 0.25/ln(4/3), 0.875/ln 8) = (0, .420784, .869016, .420784),
    # total 1.710584.  m is symmetric about interval 2, so the middle edge is its midpoint 0.55;
    # the first target total/4 = .427646 lies .006862 into interval 2: 0.5 + .1 * .006862/.869016
    got, _ = orc.refine_axis([0.0, 0.0, 8.0, 0.0], edges, 1.0)
    assert got[2] == pytest.approx(0.55, abs=1e-15)
    assert got[1] == pytest.approx(0.500790, abs=2e-6)
    assert got[3] == pytest.approx(0.599210, abs=2e-6)


def test_alpha_zero_and_uniform_unchanged(orc):
    edges = np.array([0.0, 0.05, 0.3, 0.31, 0.7, 1.0])
    got, unchanged = orc.refine_axis([1.0, 2.0, 3.0, 4.0, 5.0], edges, 0.0)
    assert unchanged and np.array_equal(got, edges)
    for alpha in (0.5, 1.5):
        got, unchanged = orc.refine_axis([3.0] * 5, edges, alpha)
        assert not unchanged
        assert np.allclose(got, edges, rtol=0, atol=4e-16)


@pytest.mark.parametrize("w", [[0.0, 0.0, 0.0], [1.0, math.nan, 1.0], [1.0, math.inf, 2.0], [1.0, -1.0, 3.0]])
def test_degenerate_weights_unchanged(orc, w):
    edges = np.array([0.0, 0.2, 0.9, 1.0])
    got, unchanged = orc.refine_axis(w, edges, 0.5)
    assert unchanged and np.array_equal(got, edges)


def test_inverse_cdf_property_and_monotone(orc):
    rng = np.random.default_rng(7)
    for trial in range(30):
        N = int(rng.integers(2, 200))
        alpha = float(rng.uniform(0.1, 2.0))
        w = rng.exponential(1.0, N) * (rng.random(N) < 0.7)
        if w.sum() == 0:
            w[0] = 1.0
        edges = np.concatenate([[0.0], np.sort(rng.random(N - 1)), [1.0]])
        got, unchanged = orc.refine_axis(w, edges, alpha)
        assert not unchanged
        assert got[0] == 0.0 and got[-1] == 1.0 and np.all(np.diff(got) > 0)
        ws = np.empty(N)
        ws[0] = (7 * w[0] + w[1]) / 8
        ws[-1] = (w[-2] + 7 * w[-1]) / 8
        ws[1:-1] = (w[:-2] + 6 * w[1:-1] + w[2:]) / 8
        r = ws / ws.sum()
        m = np.array([_damp(x, alpha) for x in r])
        cum = np.concatenate([[0.0], np.cumsum(m)])
        at_new = np.interp(got[1:-1], edges, cum)
        assert np.allclose(at_new, np.arange(1, N) * cum[-1] / N, rtol=1e-11, atol=1e-12 * cum[-1])


def test_concentrated_weight_narrows_interval(orc):
    edges = np.linspace(0, 1, 11)
    w = np.full(10, 0.01)
    w[6] = 10.0
    got, _ = orc.refine_axis(w, edges, 1.0)
    assert got[7] - got[6] < 0.1
    assert (np.diff(got)[6] == np.diff(got).min())
