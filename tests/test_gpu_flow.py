"""The learned proposal's coupling flow on the GPU (vegas_flow_*), against
the oracle (oracle/flow.py) and against its own invariants.

Tolerances.  The CUDA path rounds the weights, the conditioner input and the
hidden activations to bf16 (8 significant bits) and accumulates in FP32; the
oracle rounds the same quantities to bf16 and computes in FP64.  The two
then differ only where an FP32 rounding moves a value across a bf16 rounding
boundary, which changes one hidden unit by one bf16 ulp (2^-8 relative):
outputs agree to ~1e-5 typically and to 5e-3 at worst.  The backward pass also
rounds the gradients of the layer outputs and hidden units to bf16, so the
gradient of each parameter block agrees with the oracle's FP64 gradient to a
few percent of its norm.  Checks that need no tolerance argument: the
change of variables (Monte Carlo within 5 standard errors), the round trip,
Adam against its definition, and that training lowers the loss.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import flow as F  # noqa: E402
from paper_2408_09229_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def V():
    import __graft_entry__ as g
    g.build()
    from paper_2408_09229_gb300 import vegas
    assert torch.cuda.is_available()
    return vegas


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()


def gpu_apply(V, d, direction, th, x):
    xi = dev(x)
    xo = torch.empty_like(xi)
    ld = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
    V.flow_apply(d, direction, dev(th), xi, xo, ld)
    torch.cuda.synchronize()
    return xo.cpu().numpy().astype(np.float64), ld.cpu().numpy().astype(np.float64)


def test_param_count_matches_layout(V):
    for d in range(2, 33):
        assert V.flow_param_count(d) == F.param_count(d)
    assert V.flow_param_count(1) == 0 and V.flow_param_count(33) == 0


@pytest.mark.parametrize("d", [2, 5, 12, 16, 17, 27, 30, 32])
def test_apply_matches_oracle(V, d):
    """the tensor-core transform against the oracle's bf16 path; d = 17..32 take the 32-axis kernel, and from
    d = 27 on the first GEMM has two k-steps"""
    th = W.flow_params(d, seed=d, out_scale=0.05)
    n = 1037  # 8 full tiles of 128 points and a ragged one
    x = np.random.default_rng(d).uniform(0.01, 0.99, (n, d)).astype(np.float32).astype(np.float64)
    for direction, fn in ((V.FLOW_NORMALISE, F.normalise), (V.FLOW_SAMPLE, F.sample)):
        gx, gl = gpu_apply(V, d, direction, th, x)
        ox, ol = fn(th, x, d, bf16_path=True)
        ex, el = np.abs(gx - ox), np.abs(gl - ol)
        assert np.median(ex) < 2e-5 and ex.max() < 5e-3, (direction, np.median(ex), ex.max())
        assert np.median(el) < 2e-4 and el.max() < 5e-2, (direction, np.median(el), el.max())
        # the flow moves the points: the comparison is not of two identities
        assert np.abs(ox - x).max() > 0.02


@pytest.mark.parametrize("d", [3, 16, 17])
@pytest.mark.parametrize("n", [1, 127, 128, 129])
def test_apply_small_and_ragged_sizes(V, d, n):
    """a single point, one short of a tile, exactly one tile and one over, on both tensor-core kernels (up to 16
    axes and above); rows past n are never written"""
    th = W.flow_params(d, seed=20 + d, out_scale=0.05)
    x = np.random.default_rng(n).uniform(0.01, 0.99, (n, d)).astype(np.float32)
    xi = dev(x)
    xo = torch.full((n + 5, d), -3.0, dtype=torch.float32, device="cuda")
    ld = torch.full((n + 5,), -3.0, dtype=torch.float32, device="cuda")
    V.flow_apply(d, V.FLOW_SAMPLE, dev(th), xi, xo[:n], ld[:n])
    V.flow_check()
    ox, ol = F.sample(th, x.astype(np.float64), d, bf16_path=True)
    got = xo.cpu().numpy()
    assert np.abs(got[:n] - ox).max() < 5e-3 and np.abs(ld.cpu().numpy()[:n] - ol).max() < 5e-2
    assert (got[n:] == -3.0).all() and (ld.cpu().numpy()[n:] == -3.0).all()


def test_apply_many_tiles_and_check(V):
    """more tiles than the resident warpgroups: every warpgroup loops over several tiles; in place; the
    bounded waits all completed"""
    d = 12
    th = W.flow_params(d, seed=11, out_scale=0.05)
    n = 2 * 152 * 4 * 128 + 77
    x = np.random.default_rng(12).uniform(0.01, 0.99, (n, d)).astype(np.float32)
    xd = torch.as_tensor(x).cuda()
    ld = torch.empty(n, dtype=torch.float32, device="cuda")
    V.flow_apply(d, V.FLOW_SAMPLE, dev(th), xd, xd, ld)
    V.flow_check()
    ox, ol = F.sample(th, x.astype(np.float64), d, bf16_path=True)
    ex = np.abs(xd.cpu().numpy() - ox)
    el = np.abs(ld.cpu().numpy() - ol)
    # a rare bf16 rounding that falls the other way moves one point further: bound the far tail separately
    assert np.median(ex) < 2e-5 and np.quantile(ex, 0.9999) < 5e-3 and ex.max() < 5e-2, (np.median(ex), ex.max())
    assert np.median(el) < 2e-4 and np.quantile(el, 0.9999) < 5e-2, (np.median(el), el.max())


@pytest.mark.parametrize("direction", ["normalise", "sample"])
def test_apply_extreme_inputs_stay_finite(V, direction):
    """exact 0, denormal-sized and 1 - 2^-24 coordinates through a strongly scaled flow: the logit clamp,
    the soft clamp and the sigmoid keep x in [0, 1] and the log-determinant finite"""
    d = 12
    th = W.flow_params(d, seed=13, out_scale=2.0)
    rng = np.random.default_rng(14)
    x = rng.uniform(0.0, 1.0, (4096, d)).astype(np.float32)
    specials = np.array([0.0, 1e-30, 2.0 ** -24, 0.5, 1.0 - 2.0 ** -24], dtype=np.float32)
    x[::7] = rng.choice(specials, size=x[::7].shape)
    dirn = V.FLOW_NORMALISE if direction == "normalise" else V.FLOW_SAMPLE
    gx, gl = gpu_apply(V, d, dirn, th, x)
    assert np.isfinite(gx).all() and np.isfinite(gl).all()
    assert gx.min() >= 0.0 and gx.max() <= 1.0


def test_bounded_wait_reports_timeout(V):
    """failure detection without a fault: an mbarrier that nothing arrives on runs out its poll budget and the
    host reads VEGAS_ETIMEOUT; the report is cleared, the context stays usable, and a wait that is satisfied
    returns OK"""
    V.flow_check()
    assert V.flow_wait_selftest(1000, 0) == V.ETIMEOUT
    V.flow_check()  # cleared: no error
    assert V.flow_wait_selftest(1000, 1) == V.OK
    assert V.flow_wait_selftest(0, 1) == V.EINVAL
    x = torch.rand((300, 6), device="cuda")
    xo, ld = torch.empty_like(x), torch.empty(300, device="cuda")
    V.flow_apply(6, V.FLOW_SAMPLE, dev(W.flow_params(6, seed=1, out_scale=0.0)), x, xo, ld)
    V.flow_check()
    assert torch.allclose(xo, x, atol=1e-6)


def test_identity_flow_on_gpu(V):
    d = 7
    th = W.flow_params(d, seed=1, out_scale=0.0)
    x = np.random.default_rng(0).uniform(0.001, 0.999, (500, d)).astype(np.float32).astype(np.float64)
    gx, gl = gpu_apply(V, d, V.FLOW_SAMPLE, th, x)
    assert np.abs(gx - x).max() < 1e-6 and np.abs(gl).max() < 1e-5


def test_round_trip_and_logdet_sign(V):
    d = 12
    th = W.flow_params(d, seed=3, out_scale=0.05)
    x = np.random.default_rng(4).uniform(0.01, 0.99, (4096, d))
    xp, ln = gpu_apply(V, d, V.FLOW_NORMALISE, th, x)
    xb, ls = gpu_apply(V, d, V.FLOW_SAMPLE, th, xp)
    err = np.abs(xb - x.astype(np.float32))
    assert np.quantile(err, 0.99) < 1e-5 and err.max() < 1e-2
    assert np.quantile(np.abs(ls + ln), 0.99) < 1e-4


@pytest.mark.parametrize("d", [3, 12])
def test_change_of_variables_on_gpu(V, d):
    """the GPU's sampling map with its own log-determinant: the integral of |det dF/dx'| over the cube is 1
    and a Gaussian keeps its integral (Monte Carlo within 5 standard errors)"""
    th = W.flow_params(d, seed=7, out_scale=0.05)
    n = 1 << 22
    xp = torch.rand((n, d), dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    xo = torch.empty_like(xp)
    ld = torch.empty(n, dtype=torch.float32, device="cuda")
    V.flow_apply(d, V.FLOW_SAMPLE, dev(th), xp, xo, ld)
    jac = torch.exp(ld.double())
    m, s = float(jac.mean()), float(jac.std())
    assert abs(m - 1.0) < 5 * s / math.sqrt(n) and s > 0.02
    mu, sg = 0.45, 0.3
    f = torch.exp(-((xo.double() - mu) ** 2).sum(dim=1) / (2 * sg * sg)) * jac
    one = math.sqrt(math.pi / 2) * sg * (math.erf((1 - mu) / (sg * math.sqrt(2))) + math.erf(mu / (sg * math.sqrt(2))))
    assert abs(float(f.mean()) - one ** d) < 5 * float(f.std()) / math.sqrt(n)


def _gpu_grad(V, d, th, x, w):
    n = x.shape[0]
    grad = torch.zeros(th.size, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    scratch = torch.empty(V.flow_grad_scratch_bytes(d, n), dtype=torch.uint8, device="cuda")
    V.flow_grad(d, dev(th), dev(x), dev(w), grad, loss, scratch)
    V.flow_check()
    return float(loss[0]), grad.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("d,n", [(2, 128), (4, 1), (5, 1000), (8, 4096), (12, 777), (12, 4096), (16, 300)])
def test_tensor_core_gradient_matches_oracle_elementwise(V, d, n):
    """the tcgen05 gradient (up to 16 axes) against the oracle rounding the same operands to bf16 (weights,
    conditioner input, hidden activations, and the backward pass's gradients of (s, t) and of the hidden
    pre-activations), element by element.  The bound: FP32 accumulation over at most 128 samples per tile and
    the partials of the tiles (~1e-5 of the sum of magnitudes), plus rare bf16 rounding decisions that fall the
    other way on the two sides (one operand of one sample moves by 2^-8 relative), plus the z before each
    layer, which the GPU recomputes by inverting the layer: |g - g_oracle| <= 2e-3 max|block| + 1e-2 |g_oracle|"""
    th = W.flow_params(d, seed=11 + d, out_scale=0.05)
    rng = np.random.default_rng(d + n)
    x = rng.uniform(0.02, 0.98, (n, d)).astype(np.float32).astype(np.float64)
    w = rng.exponential(1.0, n).astype(np.float32).astype(np.float64)
    lg, gg = _gpu_grad(V, d, th, x, w)
    L, g = F.grad(th, x, w, d, bf16_path=True, bf16_grad=True)
    assert lg == pytest.approx(L, rel=1e-4, abs=1e-4)
    off = 0
    worst = 0.0
    for l in range(F.LAYERS):
        for name, shape in F.layer_sizes(d, l):
            k = int(np.prod(shape))
            a, b = gg[off:off + k], g[off:off + k]
            bound = 2e-3 * np.abs(b).max() + 1e-2 * np.abs(b) + 1e-9
            worst = max(worst, float((np.abs(a - b) / bound).max()))
            assert np.all(np.abs(a - b) <= bound), (l, name, np.abs(a - b).max(), np.abs(b).max())
            off += k
    print(f"d={d} n={n}: worst error / bound = {worst:.3f}")


@pytest.mark.parametrize("d,n", [(5, 1000), (12, 777), (30, 333)])
def test_gradient_matches_oracle(V, d, n):
    th = W.flow_params(d, seed=11 + d, out_scale=0.05)
    rng = np.random.default_rng(d)
    x = rng.uniform(0.02, 0.98, (n, d)).astype(np.float32).astype(np.float64)
    w = rng.exponential(1.0, n).astype(np.float32).astype(np.float64)
    grad = torch.zeros(th.size, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    scratch = torch.empty(V.flow_grad_scratch_bytes(d, n), dtype=torch.uint8, device="cuda")
    V.flow_grad(d, dev(th), dev(x), dev(w), grad, loss, scratch)
    torch.cuda.synchronize()
    L, g = F.grad(th, x, w, d, bf16_path=True)
    assert float(loss[0]) == pytest.approx(L, rel=2e-3, abs=2e-3)
    gg = grad.cpu().numpy().astype(np.float64)
    off = 0
    for l in range(F.LAYERS):
        for name, shape in F.layer_sizes(d, l):
            k = int(np.prod(shape))
            a, b = gg[off:off + k], g[off:off + k]
            assert np.linalg.norm(a - b) <= 0.05 * np.linalg.norm(b) + 1e-6, (l, name)
            off += k


def test_adam_matches_definition(V):
    rng = np.random.default_rng(2)
    n = 10_001
    th, g = rng.normal(size=n), rng.normal(size=n)
    m, v = rng.normal(size=n) * 0.1, rng.uniform(0, 0.1, n)
    tt, gt, mt, vt = dev(th), dev(g), dev(m), dev(v)
    V.flow_adam(tt, gt, mt, vt, 7, lr=2e-3, beta1=0.9, beta2=0.99, eps=1e-6)
    torch.cuda.synchronize()
    want, wm, wv = F.adam(th, g, m, v, 7, lr=2e-3, beta1=0.9, beta2=0.99, eps=1e-6)
    assert np.allclose(tt.cpu().numpy(), want, rtol=1e-5, atol=1e-6)
    assert np.allclose(mt.cpu().numpy(), wm, rtol=1e-5, atol=1e-7)
    assert np.allclose(vt.cpu().numpy(), wv, rtol=1e-5, atol=1e-8)


def test_training_on_gpu_lowers_the_loss(V):
    """GPU forward/backward and Adam on samples of a diagonal ridge in d = 2 (the oracle's training pin)"""
    d, n = 2, 4096
    rng = np.random.default_rng(7)
    xs = rng.uniform(0, 1, (n, d))
    w = np.exp(-((xs[:, 0] - xs[:, 1]) ** 2) / (2 * 0.05 ** 2))
    th = dev(W.flow_params(d, seed=1))
    m, v = torch.zeros_like(th), torch.zeros_like(th)
    grad = torch.zeros_like(th)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    scratch = torch.empty(V.flow_grad_scratch_bytes(d, n), dtype=torch.uint8, device="cuda")
    X, Wt = dev(xs), dev(w)
    losses = []
    for step in range(1, 201):
        V.flow_grad(d, th, X, Wt, grad, loss, scratch)
        V.flow_adam(th, grad, m, v, step, lr=3e-3)
        if step in (1, 200):
            torch.cuda.synchronize()
            losses.append(float(loss[0]))
    assert losses[1] < losses[0] - 0.3
    # the oracle's loss of the GPU-trained parameters agrees
    assert F.loss(th.cpu().numpy().astype(np.float64), xs, w, d) < losses[0] - 0.3


# ---------------------------------------------------------------------------
# the flow inside the VEGAS+ iteration (vegas_set_flow / vegas_set_flow_training)
# ---------------------------------------------------------------------------
def test_identity_flow_reproduces_plain_vegas(V):
    """with F = identity the points and weights of the first iteration are those of the plain FP32 form up
    to the FP32 rounding of logit / sigmoid (1e-6); later iterations start from allocation weights that
    differ in their last bits, so their counts differ and they agree statistically"""
    d, neval = 4, 200_000
    p = W.ridge(4, 3, 0.1)
    plain = V.Vegas(d, 50, 0, 0.5, 0.75, precision=V.FP32).integrate(W.GAUSS_SUM, p, neval, 5, seed=3)
    v = V.Vegas(d, 50, 0, 0.5, 0.75, precision=V.FP32)
    v.set_flow(W.flow_params(d, seed=0, out_scale=0.0))
    r = v.integrate(W.GAUSS_SUM, p, neval, 5, seed=3)
    assert r["it_est"][0] == pytest.approx(plain["it_est"][0], rel=1e-6)
    assert r["it_sig"][0] == pytest.approx(plain["it_sig"][0], rel=1e-4)
    assert np.all(np.abs(r["it_est"] - plain["it_est"]) < 3 * plain["it_sig"])


@pytest.mark.parametrize("name,iid,d,params", [
    ("ridge d6", W.GAUSS_SUM, 6, W.ridge(6, 3, 0.1)),
    ("product peak d5", W.PRODUCT_PEAK, 5, W.product_peak(5, seed=2)),
    ("oscillatory d4", W.OSCILLATORY, 4, W.oscillatory(4, seed=1)),
])
def test_random_flow_keeps_the_estimate_unbiased(V, name, iid, d, params):
    """any flow: g = f(F(x')) |det dF/dx'| has the integral of f"""
    v = V.Vegas(d, 50, 0, 0.5, 0.75, precision=V.FP32)
    v.set_flow(W.flow_params(d, seed=5, out_scale=0.05))
    r = v.integrate(iid, params, 300_000, 8, seed=1)
    exact = W.exact(iid, d, params)
    assert r["status"] == 0
    assert abs(r["estimate"] - exact) < 5 * r["sigma"], (r["estimate"], r["sigma"], exact)


def test_flow_handle_combines_with_lagged_weights(V, orc):
    """with a flow the handle's default combination weights iteration t by 1/sigma_{t-1}^2 (R20); the
    setter restores Eq. (8), and plain VEGAS+ keeps Eq. (8) by default"""
    d = 4
    p = W.ridge(4, 3, 0.1)
    v = V.Vegas(d, 50, 0, 0.5, 0.75, precision=V.FP32)
    v.set_flow(W.flow_params(d, seed=5, out_scale=0.05))
    r = v.integrate(W.GAUSS_SUM, p, 100_000, 6, seed=2)
    want = orc.combine(r["it_est"], r["it_sig"], 0, lagged=True)
    assert r["estimate"] == pytest.approx(want["estimate"], rel=1e-13)
    assert r["sigma"] == pytest.approx(want["sigma"], rel=1e-13)
    assert r["chi2_dof"] == pytest.approx(want["chi2_dof"], rel=1e-11)
    v.set_weighting(V.WEIGHT_INVERSE_VARIANCE)
    r = v.integrate(W.GAUSS_SUM, p, 100_000, 4, seed=3)
    assert r["estimate"] == pytest.approx(orc.combine(r["it_est"], r["it_sig"], 0)["estimate"], rel=1e-13)
    q = V.Vegas(d, 50, 0, 0.5, 0.75, precision=V.FP32).integrate(W.GAUSS_SUM, p, 100_000, 4, seed=3)
    assert q["estimate"] == pytest.approx(orc.combine(q["it_est"], q["it_sig"], 0)["estimate"], rel=1e-13)


def test_online_training_in_the_loop(V):
    """training between iterations lowers the flow's loss; the trained proposal integrates the ridge with a
    lower variance per iteration than plain VEGAS+ and an estimate within 5 sigma.  (Trained on its own
    samples alone the flow drains density from the regions it rarely samples; sigma_t then correlates with
    I_t and the inverse-variance combination of Eq. (8) leans low.  The uniform floor keeps it covering the
    cube: the flow's Jacobian averages to 1 over uniform x'.)"""
    d, neval = 4, 200_000
    p = W.ridge(4, 3, 0.05)
    v = V.Vegas(d, 50, 0, 0.5, 0.75, precision=V.FP32)
    v.set_flow(W.flow_params(d, seed=2))
    v.set_flow_training(iterations=8, steps_per_iteration=100, samples=32768, batch=4096, lr=1e-3, temper=0.5,
                        floor=0.03)
    v.set_skip(7)  # the estimate combines the iterations after training
    v.integrate(W.GAUSS_SUM, p, neval, 1, seed=4)
    _, loss1 = v.get_flow()
    r = v.integrate(W.GAUSS_SUM, p, neval, 15, seed=5)
    th, loss2 = v.get_flow()
    assert loss2 < loss1
    assert np.abs(th - W.flow_params(d, seed=2)).max() > 1e-3
    assert abs(r["estimate"] - 1.0) < 5 * r["sigma"], (r["estimate"], r["sigma"], r["chi2_dof"])
    xq = torch.rand((1 << 20, d), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    xo, lq = torch.empty_like(xq), torch.empty(1 << 20, device="cuda")
    V.flow_apply(d, V.FLOW_SAMPLE, torch.as_tensor(th).cuda(), xq, xo, lq)
    assert abs(float(torch.exp(lq.double()).mean()) - 1.0) < 0.15
    plain = V.Vegas(d, 50, 0, 0.5, 0.75, precision=V.FP32).integrate(W.GAUSS_SUM, p, neval, 15, seed=5)
    rel = lambda q: np.median(q["it_sig"][7:] / q["it_est"][7:])  # noqa: E731
    assert rel(r) < 0.7 * rel(plain)


# ---------------------------------------------------------------------------
# plain VEGAS+ as the fallback and judge of the learned proposal (vegas_set_flow_judge)
# ---------------------------------------------------------------------------
def test_judge_turns_an_idle_flow_off(V):
    """the identity flow costs time and removes no variance: beside it, plain VEGAS+ reaches a given error
    sooner, the judge turns the flow off and the result is the plain iterations'"""
    d = 4
    p = W.ridge4_params()
    v = V.Vegas(d, 50, 0, 0.5, 0.75, precision=V.FP32)
    v.set_flow(W.flow_params(d, seed=0, out_scale=0.0))
    v.set_flow_judge(3)
    r = v.integrate(W.GAUSS_SUM, p, 100_000, 20, seed=0)
    assert r["flags"] & V.RESULT_FLOW_OFF and not r["flags"] & V.RESULT_FLOW_KEPT
    assert 0.0 < r["judge_ratio"] <= 1.0
    assert r["nitn_judge"] == 8  # 5 iterations to adapt plain VEGAS+'s map, then the window of 3
    assert r["nitn_run"] == 20 and r["neval_total"] == 100_000 * 28
    assert abs(r["estimate"] - 1.0) < 5 * r["sigma"]
    # the result is plain VEGAS+ (Eq. (8), the plain arm's own records)
    assert r["estimate"] > 0
    r2 = v.integrate(W.GAUSS_SUM, p, 100_000, 4, seed=1)  # later calls stay plain, with no judge
    assert r2["nitn_judge"] == 0 and not r2["flags"] & (V.RESULT_FLOW_OFF | V.RESULT_FLOW_KEPT)
    # a new flow starts the judge over
    v.set_flow(W.flow_params(d, seed=0, out_scale=0.0))
    r3 = v.integrate(W.GAUSS_SUM, p, 100_000, 3, seed=2)
    assert r3["nitn_judge"] == 3 and not r3["flags"] & (V.RESULT_FLOW_OFF | V.RESULT_FLOW_KEPT)


def test_judge_keeps_a_flow_that_wins(V):
    """the paper's Ridge (Table 3 (8)) with 100 Gaussians along the diagonal of the 8-cube at 1e6 evaluations
    per iteration: a separable map cannot follow the tube and the trained flow can; the judge keeps it"""
    d = 8
    tube = W.paper_ridge(d, 100)
    v = V.Vegas(d, 50, 0, 0.5, 0.75, precision=V.FP32)
    v.set_flow(W.flow_params(d, seed=0))
    v.set_flow_training(iterations=10, steps_per_iteration=200, samples=65536, batch=4096, lr=1e-3, temper=0.5,
                        floor=0.03)
    v.set_skip(10)
    v.set_flow_judge(3)
    r = v.integrate(W.GAUSS_SUM, tube, 1_000_000, 16, seed=0)
    assert r["flags"] & V.RESULT_FLOW_KEPT and not r["flags"] & V.RESULT_FLOW_OFF
    assert r["judge_ratio"] > 3.0
    assert r["nitn_judge"] == 13  # 10 training iterations, then the window of 3
    exact = W.exact(W.GAUSS_SUM, d, tube)
    assert abs(r["estimate"] - exact) < 5 * r["sigma"]
