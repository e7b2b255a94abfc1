"""Pins of the oracle's integrands (Table 3 of the paper and the synthetic families).

* values at points worked out by hand;
* the closed-form integrals in workloads.py against independent numerical
  quadrature (scipy quad on the one-dimensional factors);
* the oracle's integrand itself against brute-force Gauss-Legendre quadrature
  in d <= 2, which fails on a dropped term, a wrong sign or a swapped operand.
"""
import math

import numpy as np
import pytest
from scipy import integrate as si

from paper_2408_09229_gb300 import workloads as W


def test_point_values(orc):
    # Table 3 (1): sin(0) + exp(0) = 1 ; sin(pi/2) + exp(1) = 1 + e
    assert orc.integrand(W.SIN_EXP, [0.0, 0.0]) == 1.0
    assert orc.integrand(W.SIN_EXP, [math.pi / 2, 1.0]) == pytest.approx(1.0 + math.e, rel=1e-15)
    # (2) linear: sum
    assert orc.integrand(W.LINEAR, [0.1, 0.2, 0.7]) == pytest.approx(1.0, rel=1e-15)
    # (3) cosine: prod cos
    assert orc.integrand(W.COSINE, [0.0, math.pi / 3]) == pytest.approx(0.5, rel=1e-15)
    # (4) exponential: exp(sum x^2) ; at (1, 1) -> e^2
    assert orc.integrand(W.EXPONENTIAL, [1.0, 1.0]) == pytest.approx(math.e ** 2, rel=1e-15)
    # (5) Roos & Arnold: |4x-2| product: zero at 1/2, 2^d at the corner
    assert orc.integrand(W.ROOS_ARNOLD, [0.5, 0.9, 0.1]) == 0.0
    assert orc.integrand(W.ROOS_ARNOLD, [0.0, 1.0, 0.0]) == 8.0
    # (6) Morokoff & Caflisch: (1+1/d)^d prod x^(1/d); all ones -> (1+1/d)^d
    assert orc.integrand(W.MOROKOFF_CAFLISCH, [1.0] * 4) == pytest.approx(1.25 ** 4, rel=1e-15)
    assert orc.integrand(W.MOROKOFF_CAFLISCH, [0.0, 1.0]) == 0.0
    # gauss sum at a peak centre: A * (1 + far tails)
    p = W.gauss_sum(2, [[0.3, 0.6]], 0.1, 2.0)
    assert orc.integrand(W.GAUSS_SUM, [0.3, 0.6], p) == 2.0
    # one sigma away along an axis: A exp(-1/2)
    assert orc.integrand(W.GAUSS_SUM, [0.4, 0.6], p) == pytest.approx(2.0 * math.exp(-0.5), rel=1e-14)
    # product peak at the centre: prod c_i^2
    pp = np.array([5.0, 10.0, 0.3, 0.7])
    assert orc.integrand(W.PRODUCT_PEAK, [0.3, 0.7], pp) == pytest.approx(2500.0, rel=1e-14)
    # oscillatory at the origin: cos(2 pi u)
    po = np.array([0.125, 1.0, 2.0])
    assert orc.integrand(W.OSCILLATORY, [0.0, 0.0], po) == pytest.approx(math.cos(math.pi / 4), rel=1e-14)


def test_bad_parameters_rejected(orc):
    with pytest.raises(ValueError):
        orc.integrand(W.PRODUCT_PEAK, [0.1, 0.2], [1.0, 2.0, 3.0])
    with pytest.raises(ValueError):
        orc.integrand(W.SIN_EXP, [0.1, 0.2, 0.3])
    with pytest.raises(ValueError):
        orc.integrand(99, [0.1])


def _quad1(f):
    return si.quad(f, 0.0, 1.0, epsabs=1e-14, epsrel=1e-13, limit=200)[0]


def test_closed_forms_against_quadrature():
    # Table 3 closed forms
    assert W.table3_exact(W.SIN_EXP, 2) == pytest.approx(_quad1(math.sin) + _quad1(math.exp), rel=1e-12)
    assert W.table3_exact(W.COSINE, 10) == pytest.approx(_quad1(math.cos) ** 10, rel=1e-12)
    assert W.table3_exact(W.EXPONENTIAL, 10) == pytest.approx(_quad1(lambda x: math.exp(x * x)) ** 10,
                                                              rel=1e-12)
    assert _quad1(lambda x: abs(4 * x - 2)) == pytest.approx(1.0, rel=1e-12)
    d = 8
    assert (1 + 1 / d) * _quad1(lambda x: x ** (1 / d)) == pytest.approx(1.0, rel=1e-10)
    # gauss sum: separable per peak
    p = W.ridge(4, 3, 0.05)
    s = p[1]
    mass = sum(math.prod(_quad1(lambda x, m=m: math.exp(-(x - m) ** 2 / (2 * s * s))) for m in row)
               for row in p[3:].reshape(3, 4))
    assert p[0] * mass == pytest.approx(1.0, rel=1e-12)
    assert W.exact(W.GAUSS_SUM, 4, p) == pytest.approx(1.0, rel=1e-14)
    # the paper's ridge (Table 3 (8)) at N = 1000, d = 4
    pr = W.paper_ridge(4, 1000)
    assert W.exact(W.GAUSS_SUM, 4, pr) == pytest.approx(0.8513177582, rel=1e-9)
    # product peak and oscillatory
    pp = W.product_peak(6, seed=3)
    c, w = pp[:6], pp[6:]
    q = math.prod(_quad1(lambda x, ci=ci, wi=wi: 1.0 / (ci ** -2 + (x - wi) ** 2)) for ci, wi in zip(c, w))
    assert W.exact(W.PRODUCT_PEAK, 6, pp) == pytest.approx(q, rel=1e-11)
    po = W.oscillatory(3, seed=4)
    u, a = po[0], po[1:]
    re = si.tplquad(lambda z, y, x: math.cos(2 * math.pi * u + a[0] * x + a[1] * y + a[2] * z),
                    0, 1, 0, 1, 0, 1, epsabs=1e-11, epsrel=1e-10)[0]
    assert W.exact(W.OSCILLATORY, 3, po) == pytest.approx(re, abs=1e-9)


@pytest.mark.parametrize("iid,params", [
    (W.SIN_EXP, []),
    (W.GAUSS_SUM, list(W.ridge(2, 3, 0.08))),
    (W.PRODUCT_PEAK, list(W.product_peak(2, seed=5))),
    (W.OSCILLATORY, list(W.oscillatory(2, seed=6))),
    (W.ROOS_ARNOLD, []),
])
def test_oracle_integrand_brute_force_2d(orc, iid, params):
    # Gauss-Legendre on a 20x20 grid of panels, 10 nodes each: brute force in d = 2;
    # kinks of |4x-2| fall on panel edges
    nodes, weights = np.polynomial.legendre.leggauss(10)
    panels = 20
    xs, ws = [], []
    for p in range(panels):
        a, b = p / panels, (p + 1) / panels
        xs.extend(0.5 * (b - a) * nodes + 0.5 * (a + b))
        ws.extend(0.5 * (b - a) * weights)
    total = 0.0
    for xi, wi in zip(xs, ws):
        for yj, wj in zip(xs, ws):
            total += wi * wj * orc.integrand(iid, [xi, yj], params)
    assert total == pytest.approx(W.exact(iid, 2, params), rel=1e-9)
