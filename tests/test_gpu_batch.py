"""The batched form: many independent integrals per launch (vegas_batch_*).

Each integral p of a batch draws its points with problem_id = p in the
Philox counter, so on the same map and counts its evaluations are those of
the oracle's iteration with problem_id = p and of vegas_fill with
problem_id = p.  Checked here, through the C ABI:
  * iteration 0 of every integral (uniform map, uniform counts) against the
    single-integral FP32 fill on the same inputs: I_t and sigma_t^2 to 1e-12
    relative, plus 1e-13 absolute for the oscillatory family whose cube means
    cancel (the same per-cube arithmetic; only the grouping of the
    float-float sums into threads and the order of the FP64 sums over CTAs
    differ), map weights to 1e-12 of the largest;
  * the same iteration against the oracle on the same FP32 points: I_t 2e-5
    relative, sigma_t^2 2e-3 relative, map weights 1e-3 of the largest (the
    FP32 evaluation tolerances of the single-integral parity tests);
  * every later iteration from the batch's own state (map edges and
    allocation weights read back through vegas_batch_get): counts bit-exact
    with the oracle's allocation, I_t against the oracle's iteration on those
    edges and counts, refined edges against the oracle's refinement of the
    batch's map weights to 1e-13;
  * the combination over iterations, the rtol stop, a non-finite integral
    that stops alone, launch shapes that agree, and argument errors.
Sizes span several 2048-evaluation tiles with ragged last tiles, and the
batch mixes dimensions (widths 4, 8 and 16 of the fill) and the three
families.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2408_09229_gb300 import workloads as W  # noqa: E402

SEED = 2024
BETA, ALPHA, G = 0.75, 0.5, 50

# (dim, family, params, evaluations per iteration): dims across the three
# fill widths, budgets with ragged last tiles
PROBLEMS = [
    (2, W.OSCILLATORY, W.oscillatory(2, seed=1), 5_000),
    (3, W.GAUSS_SUM, W.ridge(3, 2, 0.1), 20_000),
    (4, W.PRODUCT_PEAK, W.product_peak(4, seed=2), 12_345),
    (5, W.GAUSS_SUM, W.ridge(5, 3, 0.08), 30_001),
    (8, W.PRODUCT_PEAK, W.product_peak(8, seed=3), 9_000),
    (9, W.OSCILLATORY, W.oscillatory(9, seed=4), 4_097),
    (12, W.PRODUCT_PEAK, W.product_peak(12, seed=5), 40_000),
    (16, W.GAUSS_SUM, W.ridge(16, 2, 0.2), 70_000),
]


@pytest.fixture(scope="module")
def V():
    import __graft_entry__ as g
    g.build()
    from paper_2408_09229_gb300 import vegas
    assert torch.cuda.is_available()
    return vegas


def as_dicts(problems):
    return [{"dim": d, "integrand": iid, "params": list(p), "neval": n} for d, iid, p, n in problems]


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def single_fill(V, d, nstrat, iid, params, neval, t, edges, offsets, pid, tile_log2=0):
    """the single-integral FP32 fill on the same inputs and tiles, problem_id = pid"""
    sb = V.fill_scratch_bytes(d, G, [nstrat] * d, neval)
    nh = nstrat ** d
    scratch = torch.empty(sb, dtype=torch.uint8, device="cuda")
    ell = torch.zeros(nh, dtype=torch.float32, device="cuda")
    bins = torch.zeros(d * G, dtype=torch.float64, device="cuda")
    res = torch.zeros(2, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    V.fill(d, G, [nstrat] * d, V.FP32, iid, dev(params, torch.float64), neval, SEED, t, BETA,
           dev(edges, torch.float64), dev(offsets, torch.int64), ell, bins, res, flags, scratch, problem_id=pid,
           tile_log2=tile_log2)
    torch.cuda.synchronize()
    return float(res[0]), float(res[1]), bins.cpu().numpy().reshape(d, G), int(flags[0])


def test_iteration0_matches_single_fill_and_oracle(V, orc):
    b = V.Batch(as_dicts(PROBLEMS), nbins=G, alpha=ALPHA, beta=BETA, seed=SEED)
    out, nrun, _ = b.integrate(1)
    assert nrun == 1
    for p, (d, iid, params, neval) in enumerate(PROBLEMS):
        inf = b.info(p)
        ns, nh = inf["nstrat"], inf["ncubes"]
        assert ns == orc.default_nstrat(neval, d) and nh == ns ** d and inf["nitn_run"] == 1
        assert out[p]["status"] == V.OK and out[p]["nitn_run"] == 1
        off = b.get(p, V.BATCH_OFFSETS)
        assert np.array_equal(off, orc.allocate(None, nh, neval, BETA))  # uniform counts, bit-exact
        est = b.get(p, V.BATCH_ITER_EST)[0]
        var = b.get(p, V.BATCH_ITER_SIG)[0] ** 2
        bins = b.get(p, V.BATCH_BINS)
        cfg = orc.Config(d, G, ns, ALPHA, BETA, points_f32=True, problem_id=p)
        edges = cfg.uniform_edges()
        s_est, s_var, s_bins, s_flags = single_fill(V, d, ns, iid, params, neval, 0, edges, off, p, inf["tile_log2"])
        assert s_flags == 0
        assert est == pytest.approx(s_est, rel=1e-12, abs=1e-13)  # oscillatory sums cancel; |f| <= 1
        assert var == pytest.approx(s_var, rel=1e-12)
        assert np.allclose(bins, s_bins, rtol=0, atol=1e-12 * s_bins.max())
        r = orc.iteration(cfg, iid, params, neval, 0, SEED, edges, off)
        assert est == pytest.approx(r["est"], rel=2e-5), p
        assert var == pytest.approx(r["var"], rel=2e-3), p
        assert np.allclose(bins, r["bins"], rtol=0, atol=1e-3 * r["bins"].max()), p
        # the combination of one iteration is that iteration
        assert out[p]["estimate"] == pytest.approx(est, rel=1e-15)
        assert out[p]["sigma"] == pytest.approx(math.sqrt(var), rel=1e-15)


def test_every_iteration_from_the_batch_state(V, orc):
    """counts bit-exact and I_t against the oracle at every iteration, from the batch's own map and weights"""
    probs = [PROBLEMS[1], PROBLEMS[4], PROBLEMS[6]]
    b = V.Batch(as_dicts(probs), nbins=G, alpha=ALPHA, beta=BETA, seed=SEED)
    prev_ell = [None] * len(probs)
    for t in range(4):
        edges = [b.get(p, V.BATCH_EDGES) for p in range(len(probs))]
        out, nrun, _ = b.integrate(1)
        assert nrun == 1
        for p, (d, iid, params, neval) in enumerate(probs):
            ns = b.info(p)["nstrat"]
            nh = ns ** d
            cfg = orc.Config(d, G, ns, ALPHA, BETA, points_f32=True, problem_id=p)
            off = b.get(p, V.BATCH_OFFSETS)
            want_off = orc.allocate(prev_ell[p], nh, neval, BETA)
            assert np.array_equal(off, want_off), (t, p)
            r = orc.iteration(cfg, iid, params, neval, t, SEED, edges[p], off)
            est = b.get(p, V.BATCH_ITER_EST)
            assert len(est) == t + 1
            assert est[t] == pytest.approx(r["est"], rel=2e-5), (t, p)
            sig = b.get(p, V.BATCH_ITER_SIG)
            assert sig[t] ** 2 == pytest.approx(r["var"], rel=2e-3), (t, p)
            bins = b.get(p, V.BATCH_BINS)
            e_new = b.get(p, V.BATCH_EDGES)
            for k in range(d):
                want, _ = orc.refine_axis(bins[k], edges[p][k], ALPHA)
                assert np.allclose(e_new[k], want, rtol=0, atol=1e-13), (t, p, k)
            ell = b.get(p, V.BATCH_ELL)
            assert np.all(np.isfinite(ell) | (ell == -np.inf))
            prev_ell[p] = ell
            c = orc.combine(est, sig)
            assert out[p]["estimate"] == pytest.approx(c["estimate"], rel=1e-14)
            assert out[p]["sigma"] == pytest.approx(c["sigma"], rel=1e-14)


def test_batch_reaches_closed_forms(V):
    rng = np.random.default_rng(5)
    probs = []
    for i in range(24):
        d = int(rng.integers(2, 13))
        fam = [W.GAUSS_SUM, W.PRODUCT_PEAK, W.OSCILLATORY][i % 3]
        params = (W.ridge(d, 3, 0.1) if fam == W.GAUSS_SUM else
                  W.product_peak(d, seed=i) if fam == W.PRODUCT_PEAK else W.oscillatory(d, seed=i))
        probs.append((d, fam, params, int(10 ** rng.uniform(5, 6.3))))
    b = V.Batch(as_dicts(probs), nbins=G, alpha=ALPHA, beta=BETA, seed=7)
    out, nrun, ms = b.integrate(8)
    assert nrun == 8 and ms > 0
    for p, (d, iid, params, neval) in enumerate(probs):
        exact = W.exact(iid, d, params)
        r = out[p]
        assert r["status"] == V.OK and r["nitn_run"] == 8 and r["n_used"] == 8
        assert abs(r["estimate"] - exact) < 5 * r["sigma"], (p, d, iid, r, exact)
        assert r["sigma"] < 0.1 * abs(exact) + 1e-2


def test_rtol_stops_each_integral(V, orc):
    probs = [(4, W.GAUSS_SUM, W.ridge(4, 3, 0.1), 200_000), (2, W.OSCILLATORY, W.oscillatory(2, seed=3), 100_000),
             (10, W.PRODUCT_PEAK, W.product_peak(10, seed=4), 20_000)]
    b = V.Batch(as_dicts(probs), nbins=G, seed=1)
    out, nrun, _ = b.integrate(30, rtol=1e-3)
    for p, r in enumerate(out):
        if r["converged"]:
            assert r["sigma"] <= 1e-3 * abs(r["estimate"])
            # it stopped at the first iteration that met the target
            sig = b.get(p, V.BATCH_ITER_SIG)
            est = b.get(p, V.BATCH_ITER_EST)
            assert len(est) == r["nitn_run"]
            for k in range(1, len(est)):
                c = orc.combine(est[:k], sig[:k])
                assert c["sigma"] > 1e-3 * abs(c["estimate"]), (p, k)
        else:
            assert r["nitn_run"] == nrun
    assert out[0]["converged"] and out[1]["converged"]
    if all(r["converged"] for r in out):
        assert nrun == max(r["nitn_run"] for r in out) < 30
    # a second call continues the same records
    out2, nrun2, _ = b.integrate(2)
    assert nrun2 == 2 and all(r2["nitn_run"] == r["nitn_run"] + 2 for r, r2 in zip(out, out2))


def test_nonfinite_integral_stops_alone(V):
    bad = W.gauss_sum(3, [[0.5, 0.5, 0.5]], 0.1, math.inf)
    probs = [(3, W.GAUSS_SUM, W.ridge(3, 2, 0.1), 20_000), (3, W.GAUSS_SUM, bad, 20_000),
             (5, W.OSCILLATORY, W.oscillatory(5, seed=2), 20_000)]
    b = V.Batch(as_dicts(probs), nbins=G, seed=3)
    out, nrun, _ = b.integrate(4)
    assert nrun == 4
    assert out[1]["status"] == V.ENONFINITE and out[1]["nitn_run"] == 1
    for p in (0, 2):
        assert out[p]["status"] == V.OK and out[p]["nitn_run"] == 4
        assert abs(out[p]["estimate"] - W.exact(probs[p][1], probs[p][0], probs[p][2])) < 5 * out[p]["sigma"]


def test_launch_shapes_agree_and_tune(V):
    b = V.Batch(as_dicts(PROBLEMS), nbins=G, seed=SEED)
    ref = None
    for variant, cps, chunk in [(0, 0, 4), (0, 1, 1), (1, 2, 16), (1, 1, 3)]:
        b.reset()
        b.set_launch(variant, cps, chunk)
        out, _, _ = b.integrate(2)
        est = np.array([r["estimate"] for r in out])
        if ref is None:
            ref = est
        else:
            assert np.allclose(est, ref, rtol=1e-9, atol=0)
    tile0 = b.info(0)["tile_log2"]
    t = b.tune()
    assert t["variant"] in (0, 1) and t["ctas_per_sm"] >= 1 and t["chunk_tiles"] in (1, 4, 16) and t["ms"] > 0
    assert t["tile_log2"] in (10, 11) and all(b.info(p)["tile_log2"] == t["tile_log2"] for p in range(len(PROBLEMS)))
    # tune resets the batch; on the starting tile the tuned shape gives the same iterations
    assert b.info(0)["nitn_run"] == 0
    b.set_tile(tile0)
    out, _, _ = b.integrate(2)
    assert np.allclose([r["estimate"] for r in out], ref, rtol=1e-9, atol=0)


def test_tile_sizes(V, orc):
    """both tile sizes: each integral's first iteration equals the single fill on the same tiles, and the two
    tile sizes agree to the FP32 form's rounding; an unknown tile is EINVAL"""
    b = V.Batch(as_dicts(PROBLEMS), nbins=G, alpha=ALPHA, beta=BETA, seed=SEED)
    est = {}
    for tl in (10, 11):
        b.reset()
        b.set_tile(tl)
        out, _, _ = b.integrate(1)
        est[tl] = np.array([r["estimate"] for r in out])
        for p, (d, iid, params, neval) in enumerate(PROBLEMS):
            inf = b.info(p)
            assert inf["tile_log2"] == tl
            off = b.get(p, V.BATCH_OFFSETS)
            cfg = orc.Config(d, G, inf["nstrat"], ALPHA, BETA, points_f32=True, problem_id=p)
            s_est, _, s_bins, _ = single_fill(V, d, inf["nstrat"], iid, params, neval, 0, cfg.uniform_edges(), off,
                                              p, tl)
            assert est[tl][p] == pytest.approx(s_est, rel=1e-12, abs=1e-13)
            bins = b.get(p, V.BATCH_BINS)
            assert np.allclose(bins, s_bins, rtol=0, atol=1e-12 * s_bins.max())
    # cubes that cross a tile edge are merged from other parts: the estimates differ at FP32 rounding
    assert np.allclose(est[10], est[11], rtol=1e-6, atol=1e-9)
    for bad in (9, 12):
        with pytest.raises(V.VegasError) as e:
            b.set_tile(bad)
        assert e.value.status == V.EINVAL
    b.close()


def test_argument_errors(V):
    ok = as_dicts(PROBLEMS[:1])
    for bad in ({"dim": 17}, {"dim": 0}, {"integrand": W.LINEAR, "params": []}, {"neval": 1},
                {"params": [1.0, 2.0]}, {"nstrat": 100}):
        q = dict(ok[0])
        q.update(bad)
        with pytest.raises(V.VegasError) as e:
            V.Batch([q], nbins=G)
        assert e.value.status == V.EINVAL, bad
    with pytest.raises(V.VegasError):
        V.Batch(ok, nbins=257)
    with pytest.raises(V.VegasError):
        V.Batch(ok, nbins=G, beta=1.5)
    b = V.Batch(ok, nbins=G)
    with pytest.raises(V.VegasError) as e:
        b.set_launch(2, 0, 4)
    assert e.value.status == V.EINVAL
    import ctypes
    small = np.zeros(3)
    st = V.lib.vegas_batch_get(b._h, 0, V.BATCH_EDGES, small.ctypes.data_as(ctypes.c_void_p), 3)
    assert st == V.ENOSPACE
    assert V.lib.vegas_batch_get(b._h, 1, V.BATCH_EDGES, small.ctypes.data_as(ctypes.c_void_p), 3) == V.EINVAL
