"""Plain FP64 numpy oracle of the learned proposal's exploration step.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import this module; the product path
(paper_2408_09229_gb300) never does.  It shares no code with the CUDA library.

Not part of cuVegas (arXiv 2408.09229).  S VEGAS+ maps (Sec. 2.1.1: on each
axis N_g intervals [e_i, e_{i+1}); y in [0, 1) maps to
x = e_i + (y N_g - i)(e_{i+1} - e_i), i = floor(y N_g), with Jacobian
prod_a N_g (e_{i+1} - e_i)) each give samples; sample r comes from map
r mod S and carries the balance-heuristic weight of multiple importance
sampling (Veach and Guibas, SIGGRAPH 1995), |f(x)| / q(x) with
q = (1/S) sum_k q_k and q_k(x) = 1 / J_k(x) the density of map k at x.
The uniform numbers follow the library's stated layout: one Philox4x32-10
call per four axes, counter (r low, r high, 4 g, 0x45585052), key (seed low,
seed high), y = (u + 1/2) 2^-32.
"""
import numpy as np

import oracle as _orc

TAG = 0x45585052


def uniforms(seed, r, d):
    """the d uniform numbers of sample r"""
    y = np.empty(d)
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    for g in range(0, d, 4):
        u = _orc.philox4x32_10([r & 0xFFFFFFFF, (r >> 32) & 0xFFFFFFFF, g, TAG], key)
        for t in range(min(4, d - g)):
            y[g + t] = (float(u[t]) + 0.5) * 2.0 ** -32
    return y


def map_point(edges, y):
    """x = M(y) for one map edges [d][G+1] (Sec. 2.1.1)"""
    edges = np.asarray(edges, dtype=np.float64)
    G = edges.shape[1] - 1
    z = np.asarray(y, dtype=np.float64) * G
    i = np.minimum(np.floor(z).astype(np.int64), G - 1)
    ax = np.arange(edges.shape[0])
    e0 = edges[ax, i]
    return e0 + (z - i) * (edges[ax, i + 1] - e0)


def map_density(edges, x):
    """q(x) = prod_a 1 / (N_g dx_a) on the interval of each coordinate (e_j <= x_a < e_{j+1}, j in [0, G-1])"""
    edges = np.asarray(edges, dtype=np.float64)
    G = edges.shape[1] - 1
    q = 1.0
    for a in range(edges.shape[0]):
        j = int(np.clip(np.searchsorted(edges[a], x[a], side="right") - 1, 0, G - 1))
        q /= G * (edges[a, j + 1] - edges[a, j])
    return q


def mixture_density(maps, x):
    """(1/S) sum_k q_k(x)"""
    return float(np.mean([map_density(E, x) for E in maps]))


def explore_points(maps, samples_per_map, seed):
    """(x [m][d], q [m]) for m = S samples_per_map, sample r from map r mod S"""
    S = len(maps)
    d = np.asarray(maps[0]).shape[0]
    m = S * samples_per_map
    X = np.empty((m, d))
    q = np.empty(m)
    for r in range(m):
        X[r] = map_point(maps[r % S], uniforms(seed, r, d))
        q[r] = mixture_density(maps, X[r])
    return X, q


def weights(iid, params, X, q):
    """|f(x)| / q(x), 0 where not finite"""
    w = np.array([abs(_orc.integrand(iid, x, params)) for x in X]) / q
    return np.where(np.isfinite(w), w, 0.0)
