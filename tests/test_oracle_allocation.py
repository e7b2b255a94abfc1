"""Pins of the oracle's allocation of evaluations to hypercubes (Sec. 2.1.2,
Eq. (7) of the paper; readings R4/R5).

* the reproducible log2 / exp2 against math.log2 / 2**y within their stated
  error (a wrong series coefficient or a lost exponent fails);
* ell_h = (beta/2) log2(M2/(n-1)) against the definition sigma_h^beta with the
  unbiased variance (a dropped n-1 or beta instead of beta/2 fails);
* invariants fixed by the method: sum n_h = N_eval exactly, n_h >= 2, every
  n_h within one of its proportional share 2 + R q_h / Q, uniform counts for
  beta = 0 and for the first iteration;
* sigma^beta proportionality checked on cubes of known variance for beta = 1
  and beta = 1/2 (n_h - 2 proportional to sigma and to sqrt(sigma));
* brute force: on tiny cube counts the offsets equal the exact rational
  cumulative shares computed with Python integers.
"""
import math

import numpy as np
import pytest


def test_log2r_accuracy(orc):
    rng = np.random.default_rng(3)
    for x in np.concatenate([rng.uniform(1e-300, 1e-290, 50), 10.0 ** rng.uniform(-30, 30, 400),
                             [1.0, 2.0, 0.5, 1.4142135, 1.4142136, 3.0, 1e300]]):
        got = orc.log2r(x)
        want = math.log2(x)
        assert abs(got - want) <= 4e-7 * max(1.0, abs(want)), (x, got, want)
    assert orc.log2r(0.0) == -math.inf
    assert math.isnan(orc.log2r(-1.0))
    assert orc.log2r(1.0) == 0.0
    assert orc.log2r(0.25) == -2.0


def test_exp2r_accuracy(orc):
    for y in np.linspace(-29.9, 0.0, 997):
        got = orc.exp2r(float(np.float32(y)))
        want = 2.0 ** float(np.float32(y))
        assert abs(got - want) <= 3e-7 * want
    assert orc.exp2r(0.0) == 1.0
    assert orc.exp2r(-31.0) == 0.0
    assert orc.exp2r(-3.0) == 0.125


def test_cube_ell_definition(orc):
    # sigma_h^beta with sigma_h^2 = M2/(n-1): two samples 1 and 3 -> M2 = 2, var = 2
    assert orc.cube_ell(2.0, 2, 1.0) == pytest.approx(0.5 * math.log2(2.0), abs=1e-7)
    # n = 5, M2 = 64 -> var = 16 -> sigma = 4 -> log2 sigma^0.75 = 1.5
    assert orc.cube_ell(64.0, 5, 0.75) == pytest.approx(1.5, abs=1e-6)
    assert orc.cube_ell(0.0, 3, 0.75) == -math.inf


def test_quant_weight(orc):
    assert orc.quant_weight(3.0, 3.0) == 2 ** 24
    assert orc.quant_weight(2.0, 3.0) == 2 ** 23
    assert orc.quant_weight(-math.inf, 1.0) == 0
    assert orc.quant_weight(-40.0, 0.0) == 0


def test_uniform_first_iteration(orc):
    for nh, neval in [(1, 2), (7, 100), (38416, 100000), (1000, 2000), (13, 13 * 2 + 12)]:
        off = orc.allocate(None, nh, neval, 0.75)
        n = np.diff(off)
        assert off[0] == 0 and off[-1] == neval
        R = neval - 2 * nh
        assert n.min() >= 2 + R // nh and n.max() <= 2 + -(-R // nh)


def test_beta_zero_is_uniform(orc):
    rng = np.random.default_rng(4)
    ell = rng.normal(0, 5, 500).astype(np.float32)
    a = orc.allocate(ell, 500, 12345, 0.0)
    b = orc.allocate(None, 500, 12345, 0.0)
    assert np.array_equal(a, b)


def test_exact_sum_minimum_and_share(orc):
    rng = np.random.default_rng(5)
    for trial in range(20):
        nh = int(rng.integers(1, 3000))
        neval = 2 * nh + int(rng.integers(0, 100000))
        ell = rng.normal(0, 4, nh).astype(np.float32)
        ell[rng.random(nh) < 0.1] = -np.inf
        off = orc.allocate(ell, nh, neval, 0.75)
        n = np.diff(off)
        assert off[0] == 0 and off[-1] == neval and n.min() >= 2
        emax = float(ell.max())
        q = np.array([orc.quant_weight(float(e), emax) for e in ell], dtype=np.float64)
        share = 2 + (neval - 2 * nh) * q / q.sum()
        assert np.all(np.abs(n - share) < 1.0 + 1e-9)


def test_all_zero_variance_is_uniform(orc):
    ell = np.full(10, -np.inf, dtype=np.float32)
    assert np.array_equal(orc.allocate(ell, 10, 1000, 0.75), orc.allocate(None, 10, 1000, 0.75))


def test_too_few_evaluations_rejected(orc):
    with pytest.raises(ValueError):
        orc.allocate(None, 10, 19, 0.75)


@pytest.mark.parametrize("beta,power", [(1.0, 1.0), (0.5, 0.5)])
def test_sigma_power_proportionality(orc, beta, power):
    # four cubes with sample variances 1, 4, 16, 64 (sigma 1, 2, 4, 8) from
    # counts 2, 3, 5, 9: extra samples follow sigma^beta
    sig = np.array([1.0, 2.0, 4.0, 8.0])
    n = np.array([2, 3, 5, 9])
    m2 = sig ** 2 * (n - 1)
    ell = np.array([orc.cube_ell(a, b, beta) for a, b in zip(m2, n)], dtype=np.float32)
    R = 10 ** 7
    off = orc.allocate(ell, 4, R + 8, beta)
    extra = np.diff(off) - 2
    want = R * sig ** power / (sig ** power).sum()
    assert np.all(np.abs(extra - want) <= 1.0 + 2e-6 * want)


def test_brute_force_rational_shares(orc):
    # cumulative rounding written with exact integers: off_h = 2h + floor(R Q_h / Q)
    rng = np.random.default_rng(6)
    for trial in range(50):
        nh = int(rng.integers(1, 6))
        neval = 2 * nh + int(rng.integers(0, 50))
        ell = rng.normal(0, 2, nh).astype(np.float32)
        off = orc.allocate(ell, nh, neval, 0.75)
        q = [orc.quant_weight(float(e), float(ell.max())) for e in ell]
        Q, R = sum(q), neval - 2 * nh
        acc, want = 0, []
        for h in range(nh + 1):
            want.append(2 * h + (R * acc) // Q)
            if h < nh:
                acc += q[h]
        assert list(off) == want


def test_default_strata_rule(orc):
    """R10: the automatic strata per axis are the largest s with s^d <= N_eval / 2 (about two evaluations per
    cube); checked by exact integer powers, and at the workloads' own sizes"""
    for neval in (2, 3, 7, 100, 1000, 99_999, 100_000, 1_000_000, 10_000_000, 100_000_000, 400_000_000):
        for d in (1, 2, 3, 4, 8, 12, 30):
            s = orc.default_nstrat(neval, d)
            assert s >= 1
            assert s ** d <= max(neval // 2, 1) or s == 1
            assert (s + 1) ** d > neval // 2
    assert orc.default_nstrat(100_000, 4) == 14      # 14^4 = 38,416 cubes, 2.6 evaluations each
    assert orc.default_nstrat(100_000_000, 8) == 9   # 9^8 = 43,046,721 cubes
    cfg = orc.Config(3, 10, [2, 3, 5], 0.5, 0.75)
    assert cfg.ncubes == 30
