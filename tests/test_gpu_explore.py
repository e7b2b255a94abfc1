"""Exploration for the learned proposal on the GPU: vegas_explore_points against the oracle (oracle/explore.py)
on the same Philox numbers and maps, and vegas_flow_explore on the narrow 4-peak ridge in d = 12, where a single
adapted map (plain VEGAS+, or a flow trained on its samples) finds one peak.

Tolerances.  Both sides form x = e_i + (z - i) dx in FP64 (the GPU with one fused multiply-add), so the FP32 points
agree to one FP32 rounding; the mixture density is a product and sum of the same FP64 intervals: 1e-12."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import explore as X  # noqa: E402
from paper_2408_09229_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def V():
    import __graft_entry__ as g
    g.build()
    from paper_2408_09229_gb300 import vegas
    assert torch.cuda.is_available()
    return vegas


def random_map(rng, d, G):
    e = np.empty((d, G + 1))
    for a in range(d):
        w = rng.exponential(1.0, G) + 0.02
        e[a] = np.concatenate([[0.0], np.cumsum(w) / w.sum()])
        e[a, -1] = 1.0
    return e


@pytest.mark.parametrize("d,G,S,M", [(2, 8, 1, 500), (5, 16, 3, 700), (12, 50, 4, 300)])
def test_explore_points_match_oracle(V, d, G, S, M):
    rng = np.random.default_rng(d * 100 + S)
    maps = [random_map(rng, d, G) for _ in range(S)]
    seed = 0x1234_5678_9ABC + d
    md = torch.tensor(np.stack(maps), dtype=torch.float64, device="cuda")
    x = torch.empty((S * M, d), dtype=torch.float32, device="cuda")
    q = torch.empty(S * M, dtype=torch.float64, device="cuda")
    V.explore_points(d, G, md, M, seed, x, q)
    torch.cuda.synchronize()
    xo, qo = X.explore_points(maps, M, seed)
    assert np.allclose(x.cpu().numpy(), xo.astype(np.float32), rtol=2 ** -23, atol=0)
    assert np.allclose(q.cpu().numpy(), qo, rtol=1e-12, atol=0)


def test_explore_points_rejects_bad_arguments(V):
    md = torch.zeros((1, 2, 9), dtype=torch.float64, device="cuda")
    x = torch.empty((4, 2), dtype=torch.float32, device="cuda")
    q = torch.empty(4, dtype=torch.float64, device="cuda")
    for args in [(0, 8, md, 4), (2, 1, md, 4), (2, 8, md, -1)]:
        with pytest.raises(V.VegasError) as e:
            V.explore_points(*args, 0, x, q)
        assert e.value.status == V.EINVAL
    V.explore_points(2, 8, md, 0, 0, x, q)  # no samples: nothing to do


def test_flow_explore_needs_a_flow_and_the_fp32_form(V):
    prm = W.ridge(4, 3, 0.05)
    v = V.Vegas(4, 50, 0, 0.5, 0.75, precision=V.FP32)
    with pytest.raises(V.VegasError) as e:
        v.flow_explore(W.GAUSS_SUM, prm, 100_000, iterations=2, maps=2, samples_per_map=1000, steps=10)
    assert e.value.status == V.EINVAL
    v.set_flow(W.flow_params(4, seed=0))
    for bad in (dict(rounds=0), dict(maps=0), dict(maps=65), dict(steps=-1)):
        with pytest.raises(V.VegasError) as e:
            v.flow_explore(W.GAUSS_SUM, prm, 100_000, **dict(dict(iterations=2, maps=2, samples_per_map=1000,
                                                                  steps=10), **bad))
        assert e.value.status == V.EINVAL
    v.close()


@pytest.mark.parametrize("seed", [100, 200])
def test_flow_explore_finds_all_four_peaks(V, seed):
    """d = 12, 4 Gaussians of width 0.03 on the diagonal, 1e7 evaluations an iteration: one adapted map finds one
    peak (plain VEGAS+ ends near 1/4); sixteen maps pooled by the balance heuristic train a flow under which
    VEGAS+ finds all four: the estimate within 3 sigma + 2 % of 1 (two more rounds on the flow's own samples)"""
    d, neval = 12, 10_000_000
    prm = W.ridge(d, 4, 0.03)
    v = V.Vegas(d, 50, 0, 0.5, 0.75, precision=V.FP32)
    r = v.integrate(W.GAUSS_SUM, prm, neval, 20, seed=3)
    assert r["estimate"] < 0.5  # a single map: at most two of the four peaks
    v.set_flow(W.flow_params(d, seed=0))
    v.flow_explore(W.GAUSS_SUM, prm, neval, iterations=10, maps=16, samples_per_map=32768, steps=2000, rounds=3,
                   seed=seed)
    r = v.integrate(W.GAUSS_SUM, prm, neval, 40, seed=7)
    assert abs(r["estimate"] - 1.0) <= 3 * r["sigma"] + 0.02, (r["estimate"], r["sigma"])
    v.close()
