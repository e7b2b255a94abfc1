"""Seeded synthetic workloads: integrand parameters and their exact integrals.

This module holds no arithmetic of the VEGAS+ method.  It builds the parameter
arrays of the integrand families and the closed-form value of each integral
over the unit cube.  Both the CUDA path and the CPU oracle receive the same
arrays.  The families are:

* GAUSS_SUM: f = A * sum_k exp(-|x - mu_k|^2 / (2 s^2)), params [A, s, K, mu(K*d)].
  - ``ridge(d, K, s)`` puts K peaks on the main diagonal at t_k = k/(K+1), so
    K = 3 gives 0.25, 0.5 and 0.75.  A normalises the integral over [0,1]^d to
    exactly 1.
  - ``paper_ridge(d, N)`` is integrand (8) of Table 3 in the cuVegas paper:
    N peaks at (i-1)/(N-1) on the diagonal, exponent -100 |x - mu|^2, and
    prefactor 1e4 / (pi^2 N).
  - ``gaussian(d)`` is integrand (7) of Table 3.
* PRODUCT_PEAK: f = prod_i 1/(c_i^-2 + (x_i - w_i)^2), with c_i ~ U[5,15] and
  w_i ~ U[0.2,0.8] drawn from a seeded numpy generator.
* OSCILLATORY: f = cos(2 pi u + sum_i a_i x_i), with a_i ~ U[0,5] and
  u ~ U[0,1).
* Table 3 integrands (1)-(6) of the paper, which take no parameters.
"""
import math

import numpy as np

GAUSS_SUM, PRODUCT_PEAK, OSCILLATORY, SIN_EXP, LINEAR, COSINE, EXPONENTIAL, \
    ROOS_ARNOLD, MOROKOFF_CAFLISCH, MAP_DENSITY = range(10)

NAMES = {GAUSS_SUM: "gauss_sum", PRODUCT_PEAK: "product_peak", OSCILLATORY: "oscillatory",
         SIN_EXP: "sin_exp", LINEAR: "linear", COSINE: "cosine", EXPONENTIAL: "exponential",
         ROOS_ARNOLD: "roos_arnold", MOROKOFF_CAFLISCH: "morokoff_caflisch", MAP_DENSITY: "map_density"}


def _gauss_mass_1d(mu, s):
    """integral over [0,1] of exp(-(x-mu)^2/(2 s^2))"""
    r = s * math.sqrt(2.0)
    return s * math.sqrt(math.pi / 2.0) * (math.erf((1.0 - mu) / r) + math.erf(mu / r))


def gauss_sum(d, centres, s, A):
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, d)
    return np.concatenate([[A, s, float(centres.shape[0])], centres.ravel()])


def gauss_sum_exact(d, params):
    A, s, K = params[0], params[1], int(params[2])
    mu = np.asarray(params[3:]).reshape(K, d)
    return A * sum(math.prod(_gauss_mass_1d(m, s) for m in row) for row in mu)


def ridge(d, K, s):
    """K isotropic Gaussians of width s on the main diagonal at t_k = k/(K+1),
    normalised so that the integral over the unit cube is exactly 1."""
    t = [(k + 1) / (K + 1) for k in range(K)]
    centres = np.array([[tk] * d for tk in t])
    mass = sum(math.prod(_gauss_mass_1d(m, s) for m in row) for row in centres)
    return gauss_sum(d, centres, s, 1.0 / mass)


def two_diagonal_ridge(d, s, t_main=(0.2, 0.4, 0.8), t_anti=(0.2, 0.6, 0.8)):
    """6 peaks on two diagonals: (t,...,t) and (t on the first half, 1-t on the
    second half of the axes); normalised to integral 1."""
    rows = [[t] * d for t in t_main]
    half = d // 2
    rows += [[t] * half + [1.0 - t] * (d - half) for t in t_anti]
    centres = np.array(rows)
    mass = sum(math.prod(_gauss_mass_1d(m, s) for m in row) for row in centres)
    return gauss_sum(d, centres, s, 1.0 / mass)


def paper_ridge(d=4, N=1000):
    """Table 3 integrand (8): 1e4/(pi^2 N) sum_i exp(-100 sum_j (x_j - (i-1)/(N-1))^2)"""
    centres = np.array([[i / (N - 1)] * d for i in range(N)])
    s = math.sqrt(1.0 / 200.0)
    return gauss_sum(d, centres, s, 1.0e4 / (math.pi ** 2 * N))


def gaussian(d=4, mu=0.5, s=0.01):
    """Table 3 integrand (7): normalised Gaussian density at (mu,...,mu)"""
    return gauss_sum(d, [[mu] * d], s, (2.0 * math.pi * s * s) ** (-d / 2.0))


def product_peak(d, seed=0):
    rng = np.random.default_rng([seed, 0x5EED])
    c = rng.uniform(5.0, 15.0, d)
    w = rng.uniform(0.2, 0.8, d)
    return np.concatenate([c, w])


def product_peak_exact(d, params):
    c, w = np.asarray(params[:d]), np.asarray(params[d:])
    return float(np.prod(c * (np.arctan(c * (1.0 - w)) + np.arctan(c * w))))


def oscillatory(d, seed=0):
    rng = np.random.default_rng([seed, 0x05C1])
    u = rng.uniform(0.0, 1.0)
    a = rng.uniform(0.0, 5.0, d)
    return np.concatenate([[u], a])


def oscillatory_exact(d, params):
    u, a = params[0], np.asarray(params[1:])
    z = complex(math.cos(2 * math.pi * u), math.sin(2 * math.pi * u))
    for aj in a:
        z *= (complex(math.cos(aj), math.sin(aj)) - 1.0) / complex(0.0, aj) if aj != 0.0 else 1.0
    return z.real


def table3_exact(iid, d):
    """closed forms of Table 3 integrands (1)-(6) over the unit cube"""
    if iid == SIN_EXP:
        return (1.0 - math.cos(1.0)) + (math.e - 1.0)
    if iid == LINEAR:
        return d / 2.0
    if iid == COSINE:
        return math.sin(1.0) ** d
    if iid == EXPONENTIAL:
        # integral_0^1 exp(x^2) dx = sqrt(pi)/2 * erfi(1); erfi(1) by its power series
        erfi1 = 2.0 / math.sqrt(math.pi) * sum(1.0 / (math.factorial(n) * (2 * n + 1)) for n in range(30))
        return (math.sqrt(math.pi) / 2.0 * erfi1) ** d
    if iid in (ROOS_ARNOLD, MOROKOFF_CAFLISCH):
        return 1.0
    raise ValueError(iid)


def exact(iid, d, params=()):
    if iid == GAUSS_SUM:
        return gauss_sum_exact(d, params)
    if iid == PRODUCT_PEAK:
        return product_peak_exact(d, params)
    if iid == OSCILLATORY:
        return oscillatory_exact(d, params)
    if iid == MAP_DENSITY:
        return 1.0
    return table3_exact(iid, d)


# The workloads the benchmark and the tests run, named by what they are.
RIDGE4_CFG = dict(name="ridge d=4 K=3 s=0.05, 1e5 evals x 10 it, Ng=50, beta=0.75, alpha=0.5",
                  dim=4, nbins=50, alpha=0.5, beta=0.75, neval=100_000, nitn=10, seed=0)
RIDGE8_CFG = dict(name="ridge d=8 K=5 s=0.05, 1e8 evals x 15 it, Ng=50, beta=0.75, alpha=0.5",
                  dim=8, nbins=50, alpha=0.5, beta=0.75, neval=100_000_000, nitn=15, seed=0)


def ridge4_params():
    return ridge(4, 3, 0.05)


def ridge8_params():
    return ridge(8, 5, 0.05)


def product_peak8_params():
    return product_peak(8, seed=0)


def batch_problems(n=256, seed=0, neval_range=(1e5, 1e8), dims=(2, 12), ridge_s=0.1):
    """n independent integrals for the batched form: d uniform over
    dims[0]..dims[1], evaluations per iteration log-uniform over neval_range,
    and the family drawn uniformly from the diagonal ridge (3 peaks of width
    ridge_s, integral 1), the product peak and the oscillatory integrand, each
    with parameters from its own seeded generator.  Returns dicts with keys
    dim, integrand, params, neval, exact."""
    rng = np.random.default_rng([seed, 0xBA7C])
    out = []
    for i in range(n):
        d = int(rng.integers(dims[0], dims[1] + 1))
        neval = int(round(10 ** rng.uniform(math.log10(neval_range[0]), math.log10(neval_range[1]))))
        fam = int(rng.integers(0, 3))
        if fam == 0:
            iid, params = GAUSS_SUM, ridge(d, 3, ridge_s)
        elif fam == 1:
            iid, params = PRODUCT_PEAK, product_peak(d, seed=seed * 100_003 + i)
        else:
            iid, params = OSCILLATORY, oscillatory(d, seed=seed * 100_003 + i)
        out.append({"dim": d, "integrand": iid, "params": [float(v) for v in params], "neval": neval,
                    "exact": exact(iid, d, params)})
    return out


def flow_params(d, seed=0, out_scale=0.0, hidden=64, layers=6):
    """Seeded parameter vector of the coupling flow of the learned proposal
    (layout in include/vegas.h, vegas_flow_param_count): He-normal W1, W2,
    zero b1, b2, and W3, b3 drawn with standard deviation out_scale (0: the
    identity flow, the usual starting point of training)."""
    rng = np.random.default_rng([seed, 0xF10E])
    parts = []
    for l in range(layers):
        a = (d + 1) // 2 if l % 2 == 0 else d // 2
        b = d - a
        parts += [rng.normal(0.0, math.sqrt(2.0 / a), hidden * a), np.zeros(hidden),
                  rng.normal(0.0, math.sqrt(2.0 / hidden), hidden * hidden), np.zeros(hidden),
                  rng.normal(0.0, out_scale / math.sqrt(hidden), 2 * b * hidden) if out_scale else np.zeros(2 * b * hidden),
                  rng.normal(0.0, out_scale, 2 * b) if out_scale else np.zeros(2 * b)]
    return np.concatenate(parts).astype(np.float32).astype(np.float64)
