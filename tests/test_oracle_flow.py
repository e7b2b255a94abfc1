"""Pins of the oracle of the learned proposal (oracle/flow.py): the affine
coupling flow composed after the VEGAS map, and its training.

Each pin is fixed by mathematics independent of the oracle's formulas:
  * the sampling map inverts the normalising map (a dropped or misplaced
    layer, mask or sign fails);
  * the log-determinant equals log|det| of the Jacobian taken by central
    differences of the map itself;
  * the sampling map is a bijection of the unit cube, so its Jacobian
    determinant integrates to 1 and a Gaussian integrated through it keeps
    its closed-form value (Monte Carlo within 5 standard errors): the change
    of variables that keeps the learned proposal's estimator unbiased;
  * the analytic gradient of the loss equals central differences of the
    loss;
  * the zero-output flow is the identity with log-determinant 0;
  * the first Adam step moves every coordinate by the learning rate against
    the sign of its gradient (bias correction makes m / sqrt(v) = sign(g));
  * training on samples of a peaked density lowers the loss and the variance
    of the importance weights |f| / q.
"""
import math

import numpy as np
import pytest

from oracle import flow as F
from paper_2408_09229_gb300 import workloads as W


def points(n, d, seed):
    return np.random.default_rng(seed).uniform(0.02, 0.98, (n, d))


@pytest.mark.parametrize("d", [2, 3, 7, 12])
def test_sampling_inverts_normalising(d):
    th = W.flow_params(d, seed=d, out_scale=0.05)
    x = points(200, d, 1)
    xp, ld_n = F.normalise(th, x, d)
    xb, ld_s = F.sample(th, xp, d)
    # the round trip loses what the contraction exp(ld) amplifies of an ulp of logit(x')
    assert np.allclose(xb, x, rtol=0, atol=1e-9)
    assert np.allclose(ld_s, -ld_n, rtol=0, atol=1e-8)
    # the flow is not the identity
    assert np.abs(xp - x).max() > 0.05


def test_identity_flow():
    d = 5
    th = W.flow_params(d, seed=3, out_scale=0.0)
    x = points(100, d, 2)
    xp, ld = F.normalise(th, x, d)
    assert np.allclose(xp, x, rtol=0, atol=1e-14)
    assert np.abs(ld).max() < 1e-12


@pytest.mark.parametrize("direction", ["normalise", "sample"])
def test_logdet_is_log_abs_det_of_jacobian(direction):
    d = 4
    th = W.flow_params(d, seed=11, out_scale=0.08)
    fn = F.normalise if direction == "normalise" else F.sample
    x = points(6, d, 5)
    _, ld = fn(th, x, d)
    h = 1e-6
    for i in range(x.shape[0]):
        J = np.empty((d, d))
        for k in range(d):
            xp, xm = x[i:i + 1].copy(), x[i:i + 1].copy()
            xp[0, k] += h
            xm[0, k] -= h
            J[:, k] = (fn(th, xp, d)[0][0] - fn(th, xm, d)[0][0]) / (2 * h)
        assert ld[i] == pytest.approx(math.log(abs(np.linalg.det(J))), abs=2e-6)


@pytest.mark.parametrize("d", [2, 5])
def test_change_of_variables(d):
    """integral over [0,1]^d of |det dF/dx'| is 1 (F is a bijection of the cube), and of
    f(F(x')) |det dF/dx'| is the integral of f (a Gaussian bump, closed form by erf).  The ReLU
    conditioners make the integrand only piecewise smooth, so the check is Monte Carlo over 2^20
    uniform points, within 5 standard errors of the sample itself"""
    th = W.flow_params(d, seed=4, out_scale=0.1)
    n = 1 << 20
    xp = np.random.default_rng(17).uniform(0, 1, (n, d))
    x, ld = F.sample(th, xp, d)
    jac = np.exp(ld)
    assert abs(jac.mean() - 1.0) < 5 * jac.std() / math.sqrt(n)
    assert jac.std() > 0.05  # the flow is far from the identity
    mu, s = 0.4, 0.15
    g = np.exp(-((x - mu) ** 2).sum(axis=1) / (2 * s * s)) * jac
    one = math.sqrt(math.pi / 2) * s * (math.erf((1 - mu) / (s * math.sqrt(2))) + math.erf(mu / (s * math.sqrt(2))))
    assert abs(g.mean() - one ** d) < 5 * g.std() / math.sqrt(n)


@pytest.mark.parametrize("d", [3, 6])
def test_gradient_matches_finite_differences(d):
    th = W.flow_params(d, seed=20 + d, out_scale=0.05)
    rng = np.random.default_rng(d)
    x = points(64, d, 9)
    w = rng.exponential(1.0, 64)
    L, g = F.grad(th, x, w, d)
    assert L == pytest.approx(F.loss(th, x, w, d), rel=1e-14)
    # every block of every layer: a few coordinates each
    idx, off = [], 0
    for l in range(F.LAYERS):
        for name, shape in F.layer_sizes(d, l):
            n = int(np.prod(shape))
            idx += list(off + rng.choice(n, min(n, 3), replace=False))
            off += n
    h = 1e-6
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (F.loss(tp, x, w, d) - F.loss(tm, x, w, d)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), i


def test_first_adam_step_has_the_learning_rate():
    rng = np.random.default_rng(1)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    lr = 3e-3
    new, m, v = F.adam(th, g, np.zeros(50), np.zeros(50), 1, lr=lr, eps=0.0)
    assert np.allclose(new - th, -lr * np.sign(g), rtol=1e-12, atol=0)
    # on a quadratic the iterates approach the minimiser
    c = rng.normal(size=50)
    th, m, v = np.zeros(50), np.zeros(50), np.zeros(50)
    for step in range(1, 3001):
        th, m, v = F.adam(th, th - c, m, v, step, lr=1e-2)
    assert np.abs(th - c).max() < 1e-3


def test_training_fits_a_peaked_density():
    """weighted maximum likelihood on samples of a diagonal ridge in d = 2: loss down, weight variance down"""
    d = 2
    rng = np.random.default_rng(7)
    n = 4096

    def f(x):
        return np.exp(-((x[:, 0] - x[:, 1]) ** 2) / (2 * 0.05 ** 2))

    xs = rng.uniform(0, 1, (n, d))  # samples of the uniform proposal; weights |f| / 1
    w = f(xs)
    th = W.flow_params(d, seed=1)
    m, v = np.zeros_like(th), np.zeros_like(th)
    L0 = F.loss(th, xs, w, d)
    for step in range(1, 201):
        L, g = F.grad(th, xs, w, d)
        th, m, v = F.adam(th, g, m, v, step, lr=3e-3)
    L1 = F.loss(th, xs, w, d)
    assert L1 < L0 - 0.3
    # fresh samples through the trained sampling map: relative variance of f(F(x')) |dF/dx'|
    xp = rng.uniform(0, 1, (n, d))
    x, ld = F.sample(th, xp, d)
    gw = f(x) * np.exp(ld)
    assert np.var(gw) / np.mean(gw) ** 2 < 0.7 * np.var(w) / np.mean(w) ** 2


def test_bf16_path_stays_close():
    d = 12
    th = W.flow_params(d, seed=2, out_scale=0.05)
    x = points(256, d, 3)
    a, la = F.normalise(th, x, d)
    b, lb = F.normalise(th, x, d, bf16_path=True)
    assert np.abs(a - b).max() < 0.05 and np.abs(la - lb).max() < 0.5
    assert F.bf16(np.array([1.0 + 2 ** -9]))[0] == 1.0  # tie to even
    assert F.bf16(np.array([1.0 + 3 * 2 ** -9]))[0] == 1.0 + 2 ** -7
