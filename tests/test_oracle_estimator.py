"""Pins of the oracle's estimator and iteration loop (Secs. 2.1.1-2.1.3,
Eqs. (2)-(9), Algorithms 1 and 2 of the paper).

* the map's own density as integrand makes J f = 1 for every sample, so the
  iteration estimate is 1 and its variance 0 (a wrong bin, a dropped Jacobian
  factor or a wrong interval width fails);
* Eqs. (8)-(9) on inputs worked out by hand;
* every integrand family within 4 sigma of its closed form, and a d = 2 case
  against brute-force quadrature;
* the scale of sigma: z-scores over seeds have unit spread (a missing 1/n_h
  or 1/N_h^2 in Eq. (6) fails);
* splitting the samples into two ranges and merging the cube statistics
  reproduces the single-range fill (the sharding of Sec. 3.4);
* the paper's own ablation (Sec. 4.6): adaptive stratification (beta > 0)
  lowers the error of a peaked integrand against beta = 0;
* lagged weights (R20) on inputs worked out by hand, and their point: on
  iterations whose sigma_t is correlated with I_t (lognormal draws, mean known
  in closed form) Eq. (8) is biased low and the lagged mean is not.
"""
import math

import numpy as np
import pytest

from paper_2408_09229_gb300 import workloads as W


def test_map_density_gives_unit_weights(orc):
    rng = np.random.default_rng(8)
    d, G = 3, 7
    cfg = orc.Config(d, G, [3, 2, 4], 0.5, 0.75)
    edges = np.stack([np.concatenate([[0.0], np.sort(rng.random(G - 1)), [1.0]]) for _ in range(d)])
    params = edges.ravel()
    off = orc.allocate(None, cfg.ncubes, 5000, 0.75)
    r = orc.iteration(cfg, W.MAP_DENSITY, params, 5000, 0, 11, edges, off)
    assert r["est"] == pytest.approx(1.0, rel=1e-13)
    assert r["var"] < 1e-28
    # every cube mean is exactly J f = 1 up to rounding
    assert np.allclose(r["mean"], 1.0, rtol=1e-13)


def test_combination_by_hand(orc):
    c = orc.combine([1.0, 2.0], [1.0, 1.0])
    assert c["estimate"] == 1.5 and c["sigma"] == pytest.approx(math.sqrt(0.5))
    assert c["chi2_dof"] == pytest.approx(0.5)
    # weights 1 and 1/4: (1 + 3/4)/1.25 = 1.4; sigma^2 = 1/1.25; chi2 = 0.4^2 + 1.6^2/4 = 0.8
    c = orc.combine([1.0, 3.0], [1.0, 2.0])
    assert c["estimate"] == pytest.approx(1.4) and c["sigma"] == pytest.approx(math.sqrt(0.8))
    assert c["chi2_dof"] == pytest.approx(0.8) and c["n_used"] == 2
    c = orc.combine([9.0, 1.0, 3.0], [0.1, 1.0, 2.0], skip=1)
    assert c["estimate"] == pytest.approx(1.4) and c["n_used"] == 2
    c = orc.combine([5.0], [0.5])
    assert c["estimate"] == 5.0 and c["sigma"] == 0.5 and c["chi2_dof"] == 0.0
    c = orc.combine([2.0, 2.0, 7.0], [0.0, 0.0, 1.0])
    assert c["estimate"] == 2.0 and c["sigma"] == 0.0


def test_lagged_combination_by_hand(orc):
    # weights 1 (own sigma at t = 0), 1/sigma_0^2 = 1, 1/sigma_1^2 = 1/4: estimate 4 / 2.25 = 16/9;
    # sigma = sqrt(1 + 4 + 1/16) / 2.25 = 1; chi2 = (49/81 + (4/81)/4 + 400/81) / 2 = 25/9
    c = orc.combine([1.0, 2.0, 4.0], [1.0, 2.0, 1.0], lagged=True)
    assert c["estimate"] == pytest.approx(16 / 9, rel=1e-15) and c["sigma"] == pytest.approx(1.0, rel=1e-15)
    assert c["chi2_dof"] == pytest.approx(25 / 9, rel=1e-15) and c["n_used"] == 3
    # a skipped iteration still lends its sigma: weights 1 and 1/4, estimate 3 / 1.25, sigma sqrt(4 + 1/16) / 1.25
    c = orc.combine([1.0, 2.0, 4.0], [1.0, 2.0, 1.0], skip=1, lagged=True)
    assert c["estimate"] == pytest.approx(2.4, rel=1e-15)
    assert c["sigma"] == pytest.approx(math.sqrt(4.0625) / 1.25, rel=1e-15) and c["n_used"] == 2
    # equal sigma: the plain mean and sigma / sqrt(n), as Eq. (8)
    c = orc.combine([1.0, 2.0, 3.0, 6.0], [0.5] * 4, lagged=True)
    assert c["estimate"] == 3.0 and c["sigma"] == 0.25
    # a zero sigma before the used range: that iteration weighs with its own sigma
    c = orc.combine([2.0, 3.0, 5.0], [0.0, 1.0, 2.0], skip=1, lagged=True)
    assert c["estimate"] == 4.0 and c["sigma"] == pytest.approx(math.sqrt(5.0) / 2.0, rel=1e-15)
    # exact iterations in the used range: the same rule as Eq. (8)
    c = orc.combine([2.0, 2.0, 7.0], [0.0, 0.0, 1.0], lagged=True)
    assert c["estimate"] == 2.0 and c["sigma"] == 0.0


def test_lagged_weights_unbiased_where_eq8_is_not(orc):
    # each iteration averages m lognormal draws: I_t and its sigma_t are strongly correlated (a run that misses
    # the tail is low in both), the integral E[x] = exp(mu + s^2 / 2) is known
    rng = np.random.default_rng(20)
    mu, s, m, n, R = 0.0, 1.5, 20, 50, 400
    true = math.exp(mu + s * s / 2)
    inv, lag = [], []
    for _ in range(R):
        x = rng.lognormal(mu, s, size=(n, m))
        I, S = x.mean(1), x.std(1, ddof=1) / math.sqrt(m)
        inv.append(orc.combine(I, S)["estimate"])
        lag.append(orc.combine(I, S, lagged=True)["estimate"])
    inv, lag = np.array(inv), np.array(lag)
    se = lambda a: a.std(ddof=1) / math.sqrt(R)
    assert abs(lag.mean() - true) < 4 * se(lag)
    assert (true - inv.mean()) > 20 * se(inv)


CASES = [
    ("ridge d=4 K=3", W.GAUSS_SUM, 4, W.ridge4_params(), 100_000, 10),
    ("product peak d=4", W.PRODUCT_PEAK, 4, W.product_peak(4, seed=1), 40_000, 8),
    ("oscillatory d=3", W.OSCILLATORY, 3, W.oscillatory(3, seed=2), 20_000, 6),
    ("sin-exp d=2", W.SIN_EXP, 2, [], 20_000, 6),
    ("linear d=10", W.LINEAR, 10, [], 20_000, 6),
    ("cosine d=10", W.COSINE, 10, [], 20_000, 6),
    ("exponential d=10", W.EXPONENTIAL, 10, [], 20_000, 6),
    ("roos-arnold d=10", W.ROOS_ARNOLD, 10, [], 40_000, 8),
    ("morokoff-caflisch d=8", W.MOROKOFF_CAFLISCH, 8, [], 40_000, 8),
    ("gaussian d=4", W.GAUSS_SUM, 4, W.gaussian(4), 40_000, 10),
    ("paper ridge d=4 N=1000", W.GAUSS_SUM, 4, W.paper_ridge(4, 1000), 10_000, 6),
]


@pytest.mark.parametrize("name,iid,d,params,neval,nitn", CASES, ids=[c[0] for c in CASES])
def test_closed_form_within_4_sigma(orc, name, iid, d, params, neval, nitn):
    cfg = orc.Config(d, 50, orc.default_nstrat(neval, d), 0.5, 0.75)
    r = orc.integrate(cfg, iid, params, neval, nitn, seed=3)
    exact = W.exact(iid, d, params)
    assert r["sigma"] > 0
    assert abs(r["estimate"] - exact) < 4 * r["sigma"], (r["estimate"], r["sigma"], exact)
    assert r["n_used"] == nitn


def test_brute_force_quadrature_d2(orc):
    params = W.ridge(2, 2, 0.07)
    nodes, weights = np.polynomial.legendre.leggauss(200)
    x = 0.5 * (nodes + 1)
    w = 0.5 * weights
    total = sum(wi * wj * orc.integrand(W.GAUSS_SUM, [xi, xj], params) for xi, wi in zip(x, w)
                for xj, wj in zip(x, w))
    cfg = orc.Config(2, 50, orc.default_nstrat(20000, 2), 0.5, 0.75)
    r = orc.integrate(cfg, W.GAUSS_SUM, params, 20000, 8, seed=5)
    assert abs(r["estimate"] - total) < 4 * r["sigma"]
    assert r["sigma"] < 2e-3


def test_sigma_scale_over_seeds(orc):
    params = W.ridge(3, 2, 0.1)
    cfg = orc.Config(3, 30, 6, 0.5, 0.75)
    z = []
    for seed in range(40):
        r = orc.integrate(cfg, W.GAUSS_SUM, params, 4000, 4, seed=seed)
        z.append((r["estimate"] - 1.0) / r["sigma"])
    z = np.array(z)
    assert abs(z.mean()) < 0.6
    assert 0.65 < z.std() < 1.45


def _merge(n1, m1, q1, n2, m2, q2):
    # Chan et al. pairwise update of (count, mean, centred second moment)
    n = n1 + n2
    with np.errstate(invalid="ignore", divide="ignore"):
        delta = m2 - m1
        mean = np.where(n > 0, m1 + delta * n2 / np.maximum(n, 1), 0.0)
        q = q1 + q2 + np.where(n > 0, delta * delta * n1 * n2 / np.maximum(n, 1), 0.0)
    return n, mean, q


def test_range_split_reproduces_fill(orc):
    d = 4
    cfg = orc.Config(d, 20, 5, 0.5, 0.75)
    params = W.ridge(d, 3, 0.1)
    neval = 9001
    rng = np.random.default_rng(9)
    ell = rng.normal(0, 3, cfg.ncubes).astype(np.float32)
    off = orc.allocate(ell, cfg.ncubes, neval, 0.75)
    edges = cfg.uniform_edges()
    full = orc.fill_range(cfg, W.GAUSS_SUM, params, neval, 2, 1, edges, off, 0, neval)
    for cut in (1, 4000, 4501, 9000):
        a = orc.fill_range(cfg, W.GAUSS_SUM, params, neval, 2, 1, edges, off, 0, cut)
        b = orc.fill_range(cfg, W.GAUSS_SUM, params, neval, 2, 1, edges, off, cut, neval)
        n, mean, q = _merge(a[0], a[1], a[2], b[0], b[1], b[2])
        assert np.array_equal(n, full[0])
        assert np.allclose(mean, full[1], rtol=1e-13, atol=0)
        assert np.allclose(q, full[2], rtol=1e-9, atol=1e-12 * np.abs(full[2]).max())
        assert np.allclose(a[3] + b[3], full[3], rtol=1e-13)


def test_adaptive_stratification_helps_peaked_integrand(orc):
    # Sec. 4.6: beta > 0 against beta = 0 on a peaked integrand, equal evaluations
    params = W.ridge(4, 3, 0.05)
    sig = {}
    for beta in (0.0, 0.75):
        cfg = orc.Config(4, 50, 6, 0.5, beta)
        s = [orc.integrate(cfg, W.GAUSS_SUM, params, 50_000, 8, seed=seed)["sigma"] for seed in range(3)]
        sig[beta] = np.mean(s)
    assert sig[0.75] < 0.8 * sig[0.0], sig


def test_first_iteration_uniform_map_is_plain_stratified_mc(orc):
    # with the uniform map J = 1 and x = y: cube means are plain MC means of f;
    # the iteration estimate must equal the fill's cube means averaged (Eq. (5))
    cfg = orc.Config(2, 10, 3, 0.5, 0.75)
    off = orc.allocate(None, 9, 200, 0.75)
    r = orc.iteration(cfg, W.LINEAR, [], 200, 0, 4, cfg.uniform_edges(), off)
    assert r["est"] == pytest.approx(r["mean"].mean(), rel=1e-15)
    # linear integrand: cube (a, b) has mean ~ centre sum; 9 cubes over [0,1]^2 -> ~1
    assert abs(r["est"] - 1.0) < 5 * math.sqrt(r["var"])


@pytest.mark.parametrize("name,iid,d,params", [
    ("ridge d=4", W.GAUSS_SUM, 4, W.ridge4_params()),
    ("product peak d=5", W.PRODUCT_PEAK, 5, W.product_peak(5, seed=1)),
    ("roos-arnold d=10", W.ROOS_ARNOLD, 10, []),
    ("sin-exp d=2 many strata", W.SIN_EXP, 2, []),
])
def test_fp32_points_closed_form(orc, name, iid, d, params):
    """FP32-mode points (23-bit exact c + u, FP32 z) still sample every cube uniformly:
    the estimate stays within 4 sigma of the closed form, including with 2^9 strata per axis"""
    neval = 200_000
    cfg = orc.Config(d, 50, orc.default_nstrat(neval, d), 0.5, 0.75, points_f32=True)
    r = orc.integrate(cfg, iid, params, neval, 6, seed=4)
    assert abs(r["estimate"] - W.exact(iid, d, params)) < 4 * r["sigma"]


def test_fp32_points_uniform_in_a_cube(orc):
    # one cube of a 1-d map with 7 strata: the linear integrand's cube mean is the stratum centre
    cfg = orc.Config(1, 10, 7, 0.5, 0.75, points_f32=True)
    edges = cfg.uniform_edges()
    for h in range(7):
        m, q = orc.cube_stats(cfg, W.LINEAR, [], 0, 5, edges, h, h * 20_000, 20_000)
        assert m == pytest.approx((h + 0.5) / 7, abs=4 * math.sqrt((1 / 7) ** 2 / 12 / 20_000))
        assert q / 19_999 == pytest.approx((1 / 7) ** 2 / 12, rel=0.05)
