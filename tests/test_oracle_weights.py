"""Pins of the oracle's accumulation of map weights and of its one-cube
statistics (Algorithm 2, "GetMapWeights" and the cube weights; Sec. 2.1.1 for
what the map is trained on; reading R11: w_{k,i} = sum over the evaluations in
interval i of axis k of (J f)^2 / n_h).

The geometry makes every value known in closed form, with no Philox draw in the
expected values:
* the number of intervals equals the number of strata on every axis (N_g = s),
  so the evaluations of cube h lie in interval c_k(h) of axis k (the point's
  z = c + u with 0 <= u < 1);
* the sampling map has dyadic edges, so every interval width dx and every
  factor N_g dx is exact, and the Jacobian of cube h is the exact product
  J_h = prod_k N_g dx_{k, c_k(h)};
* the integrand is the density of the uniform two-interval map (f = 1 exactly),
  so every evaluation of cube h has J f = J_h.
The expected weights are then sums of exact rationals over the cubes:
w_{k,i} = sum_{h : c_k(h) = i} J_h^2 m_h / n_h, with m_h the number of cube
h's evaluations inside the filled range and n_h its count.  The counts are
uneven and the range cuts cubes in two, so m_h / n_h varies from cube to cube:
writing v for v^2, dropping the 1/n_h, mixing up axis and interval, or
decoding cube coordinates in the wrong axis order each fails.

orc_cube_stats, the second copy of the sample loop that checks the full-size
runs one cube at a time, must equal orc_fill_range's per-cube mean and centred
second moment bit for bit on every cube (the same samples in the same order).
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2408_09229_gb300 import workloads as W

# per-axis dyadic interval widths, each row summing to 1; N_g = 4 intervals
WIDTHS = [
    [Fraction(1, 8), Fraction(3, 8), Fraction(1, 4), Fraction(1, 4)],
    [Fraction(1, 2), Fraction(1, 16), Fraction(3, 16), Fraction(1, 4)],
    [Fraction(1, 4), Fraction(1, 4), Fraction(1, 4), Fraction(1, 4)],
]
G = 4


def dyadic_edges(widths):
    e = [np.concatenate([[0.0], np.cumsum([float(w) for w in row])]) for row in widths]
    edges = np.stack(e)
    assert np.all(edges[:, -1] == 1.0)
    return edges


def uneven_offsets(ncubes, seed):
    """a count of at least 2 per cube, uneven, summing to neval"""
    rng = np.random.default_rng(seed)
    n = 2 + rng.integers(0, 9, ncubes)
    n[rng.integers(0, ncubes)] += 40  # one long cube
    return np.concatenate([[0], np.cumsum(n)]).astype(np.int64)


def cube_coords(h, nstrat):
    c = []
    for s in nstrat:
        c.append(h % s)
        h //= s
    return c


def expected(widths, nstrat, offsets, j_begin, j_end):
    d = len(nstrat)
    nh = len(offsets) - 1
    w = [[Fraction(0)] * G for _ in range(d)]
    cnt, jac = [], []
    for h in range(nh):
        lo, hi = int(offsets[h]), int(offsets[h + 1])
        m = max(0, min(hi, j_end) - max(lo, j_begin))
        c = cube_coords(h, nstrat)
        J = Fraction(1)
        for k in range(d):
            J *= G * widths[k][c[k]]
        cnt.append(m)
        jac.append(J)
        for k in range(d):
            w[k][c[k]] += J * J * m / (hi - lo)
    return w, cnt, jac


@pytest.mark.parametrize("points_f32", [False, True])
@pytest.mark.parametrize("j_begin,j_end", [(0, None), (37, 301), (5, 6)])
def test_map_weights_closed_form(orc, points_f32, j_begin, j_end):
    nstrat = [G] * 3
    cfg = orc.Config(3, G, nstrat, 0.5, 0.75, points_f32=points_f32)
    edges = dyadic_edges(WIDTHS)
    off = uneven_offsets(cfg.ncubes, seed=3)
    neval = int(off[-1])
    j_end = neval if j_end is None else j_end
    f_one = np.tile([0.0, 0.5, 1.0], 3)  # density of the uniform two-interval map: f = 1
    cnt, mean, m2, bins = orc.fill_range(cfg, W.MAP_DENSITY, f_one, neval, 2, 17, edges, off, j_begin, j_end)
    w, m, jac = expected(WIDTHS, nstrat, off, j_begin, j_end)
    assert list(cnt) == m
    for h in range(cfg.ncubes):
        if m[h]:
            assert mean[h] == float(jac[h])  # every value of the cube is J_h exactly
            assert m2[h] == 0.0
    want = np.array([[float(x) for x in row] for row in w])
    # the oracle adds J^2/n_h per evaluation in sequence: a few ulps of each weight
    assert np.allclose(bins, want, rtol=1e-14, atol=0.0)
    if j_begin == 0 and j_end == neval:
        # every cube whole: each axis's weights sum to sum_h J_h^2
        total = float(sum(J * J for J in jac))
        assert np.allclose(bins.sum(axis=1), total, rtol=1e-14)


def test_map_weights_catch_dropped_factors(orc):
    """the closed form separates the reading from its plausible slips"""
    nstrat = [G] * 3
    off = uneven_offsets(G ** 3, seed=3)
    w, m, jac = expected(WIDTHS, nstrat, off, 0, int(off[-1]))
    right = np.array([[float(x) for x in row] for row in w])
    # v instead of v^2
    lin = np.zeros_like(right)
    # no 1/n_h
    no_n = np.zeros_like(right)
    for h in range(G ** 3):
        c = cube_coords(h, nstrat)
        n = int(off[h + 1] - off[h])
        for k in range(3):
            lin[k, c[k]] += float(jac[h]) * n / n
            no_n[k, c[k]] += float(jac[h] ** 2) * n
    assert not np.allclose(lin, right, rtol=1e-3)
    assert not np.allclose(no_n, right, rtol=1e-3)
    assert not np.allclose(right.T[:3, :3], right[:3, :3], rtol=1e-3)  # axis and interval not interchangeable


@pytest.mark.parametrize("points_f32", [False, True])
def test_cube_stats_equals_fill_range(orc, points_f32):
    d, Gq = 3, 11
    nstrat = [3, 4, 2]
    cfg = orc.Config(d, Gq, nstrat, 0.5, 0.75, points_f32=points_f32)
    rng = np.random.default_rng(5)
    edges = np.stack([np.concatenate([[0.0], np.sort(rng.random(Gq - 1)), [1.0]]) for _ in range(d)])
    off = uneven_offsets(cfg.ncubes, seed=9)
    neval = int(off[-1])
    p = W.ridge(d, 3, 0.2)
    t, seed = 4, 1234
    cnt, mean, m2, _ = orc.fill_range(cfg, W.GAUSS_SUM, p, neval, t, seed, edges, off, 0, neval)
    for h in range(cfg.ncubes):
        mh, qh = orc.cube_stats(cfg, W.GAUSS_SUM, p, t, seed, edges, h, int(off[h]), int(off[h + 1] - off[h]))
        assert mh == mean[h] and qh == m2[h], h
