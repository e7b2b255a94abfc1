"""The handle's memory hooks, its chi^2 flag and the status codes that need a GPU.

* Memory hooks (vegas_set_allocator, vegas_batch_create_ex): every device
  allocation goes through the caller's hooks; a hook that fails on its k-th call
  makes the asking call return VEGAS_ENOMEM, the handle or batch keeps working
  once the hook succeeds again, and after destroy every allocation has been
  given back (the hooks track what is live).  With torch's caching allocator
  the results equal those of cudaMalloc memory.
* chi^2/dof (Sec. 2.1.3, Eqs. (8)-(9)): iterations that disagree beyond their
  sigmas raise VEGAS_RESULT_CHI2_HIGH.  The 12-dimensional ridge of four narrow
  peaks, where plain VEGAS+ finds and loses peaks from one iteration to the
  next, raises it; the 4-dimensional ridge it integrates well does not.
* VEGAS_ECUDA: a CUDA call that fails without any device fault.  A stream
  synchronisation is not allowed while the stream is being captured into a CUDA
  graph; the handle's vegas_reset_map synchronises its stream, so on a
  capturing stream it returns VEGAS_ECUDA (run in a child process, so that the
  broken capture stays out of this one).
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2408_09229_gb300 import workloads as W  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def V():
    import __graft_entry__ as g
    g.build()
    from paper_2408_09229_gb300 import vegas
    assert torch.cuda.is_available()
    return vegas


class Hooks:
    """torch caching-allocator hooks that count calls, fail on call number fail_at and track live memory"""

    def __init__(self, fail_at=None):
        self.calls = 0
        self.fail_at = fail_at
        self.live = {}

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return 0
        p = torch.cuda.caching_allocator_alloc(nbytes, stream=stream)
        self.live[p] = nbytes
        return p

    def free(self, ptr, nbytes, stream):
        assert self.live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)


def test_torch_hooks_give_the_same_results(V):
    p = W.ridge4_params()
    a = V.Vegas(4, 50, 0, 0.5, 0.75, precision=V.FP32)
    ra = a.integrate(W.GAUSS_SUM, p, 100_000, 5, seed=3)
    hk = Hooks()
    b = V.Vegas(4, 50, 0, 0.5, 0.75, precision=V.FP32)
    b.set_allocator(hk.alloc, hk.free)
    rb = b.integrate(W.GAUSS_SUM, p, 100_000, 5, seed=3)
    assert hk.calls > 6 and len(hk.live) > 6
    np.testing.assert_allclose(rb["it_est"], ra["it_est"], rtol=1e-12)
    # moving back to cudaMalloc keeps the map: the next iteration continues alike
    b.set_allocator(None, None)
    assert not hk.live
    ra2 = a.integrate(W.GAUSS_SUM, p, 100_000, 2, seed=3)
    rb2 = b.integrate(W.GAUSS_SUM, p, 100_000, 2, seed=3)
    np.testing.assert_allclose(rb2["it_est"], ra2["it_est"], rtol=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "fp32_flow"])
def test_failing_hook_returns_enomem_and_leaks_nothing(V, precision):
    p = W.ridge4_params()
    ref = V.Vegas(4, 50, 0, 0.5, 0.75, precision=V.FP64 if precision == "fp64" else V.FP32)
    if precision == "fp32_flow":
        ref.set_flow(W.flow_params(4, seed=0))
        ref.set_flow_training(1, 2, 4096, batch=1024)
    want = ref.integrate(W.GAUSS_SUM, p, 50_000, 2, seed=1)
    total = None
    k = 1
    while total is None or k <= total:
        hk = Hooks(fail_at=k)
        v = V.Vegas(4, 50, 0, 0.5, 0.75, precision=V.FP64 if precision == "fp64" else V.FP32)
        statuses = []
        for step in ("hook", "flow", "integrate"):
            try:
                if step == "hook":
                    v.set_allocator(hk.alloc, hk.free)
                elif step == "flow" and precision == "fp32_flow":
                    v.set_flow(W.flow_params(4, seed=0))
                    v.set_flow_training(1, 2, 4096, batch=1024)
                elif step == "integrate":
                    got = v.integrate(W.GAUSS_SUM, p, 50_000, 2, seed=1)
                statuses.append(V.OK)
            except V.VegasError as e:
                statuses.append(e.status)
        if hk.calls < k:  # the hook was never asked k times: every call succeeded
            total = hk.calls
            assert statuses == [V.OK] * 3
            np.testing.assert_allclose(got["it_est"], want["it_est"], rtol=1e-12)
        else:
            assert V.ENOMEM in statuses, (k, statuses)
            assert all(st in (V.OK, V.ENOMEM) for st in statuses)
            # the hook works again: the handle recovers and runs
            hk.fail_at = None
            if precision == "fp32_flow" and statuses[1] != V.OK:
                v.set_flow(W.flow_params(4, seed=0))
            r = v.integrate(W.GAUSS_SUM, p, 50_000, 2, seed=1)
            assert abs(r["estimate"] - 1.0) < 5 * r["sigma"]
        v.close()
        assert not hk.live, (k, len(hk.live))  # everything given back
        k += 1
    assert total >= 8


def test_batch_hooks(V):
    probs = W.batch_problems(12, seed=1, neval_range=(1e5, 1e6))
    ref = V.Batch(probs, 50, 0.5, 0.75, seed=0)
    want, _, _ = ref.integrate(3)
    hk = Hooks()
    b = V.Batch(probs, 50, 0.5, 0.75, seed=0, alloc=hk.alloc, free=hk.free)
    got, _, _ = b.integrate(3)
    assert hk.live
    for g, w in zip(got, want):
        assert g["estimate"] == pytest.approx(w["estimate"], rel=1e-12)
    # the records grow past their first capacity through the hook
    b.integrate(40)
    b.close()
    assert not hk.live
    # failures at create and at the growth of the records
    for k in (1, 2, 3):
        hk = Hooks(fail_at=k)
        try:
            b = V.Batch(probs, 50, 0.5, 0.75, seed=0, alloc=hk.alloc, free=hk.free)
        except V.VegasError as e:
            assert e.status == V.ENOMEM
            assert not hk.live
            continue
        with pytest.raises(V.VegasError) as e:
            b.integrate(40)
        assert e.value.status == V.ENOMEM
        hk.fail_at = None
        out, n, _ = b.integrate(2)
        assert n == 2 and all(r["status"] == V.OK for r in out)
        b.close()
        assert not hk.live


def test_chi2_flag(V):
    v = V.Vegas(12, 50, 0, 0.5, 0.75, precision=V.FP32)
    r = v.integrate(W.GAUSS_SUM, W.ridge(12, 4, 0.03), 10_000_000, 40, seed=0)
    assert r["chi2_dof"] > 10 and r["flags"] & V.RESULT_CHI2_HIGH
    w = V.Vegas(4, 50, 0, 0.5, 0.75)
    r = w.integrate(W.GAUSS_SUM, W.ridge4_params(), 100_000, 10, seed=0)
    assert r["chi2_dof"] < 3 and not r["flags"] & V.RESULT_CHI2_HIGH
    # an explicit bound: below the run's chi2/dof raises the flag, one iteration never does
    w.set_chi2_bound(r["chi2_dof"] / 2 if r["chi2_dof"] > 0 else 1e-300)
    w.reset_map()
    r = w.integrate(W.GAUSS_SUM, W.ridge4_params(), 100_000, 10, seed=0)
    assert r["flags"] & V.RESULT_CHI2_HIGH
    r = w.integrate(W.GAUSS_SUM, W.ridge4_params(), 100_000, 1, seed=0)
    assert not r["flags"] & V.RESULT_CHI2_HIGH


def test_fp32_rounding_floor(V):
    """the FP32 form: a sigma below 2^-20 |I| is flagged and the rtol stop counts the floor; FP64 is not floored.
    The linear integrand x_0 + x_1 (I = 1) on 1e6 cubes of 2 evaluations has sigma_t about 3e-7 an iteration
    (cube variance 2 (1e-3)^2 / 12), about 1.2e-7 over six, well under the floor 2^-20 = 9.5e-7"""
    v = V.Vegas(2, 50, 0, 0.5, 0.75, precision=V.FP32, rtol=1e-7)
    r = v.integrate(W.LINEAR, [], 2_000_000, 6, seed=0)
    assert r["nitn_run"] == 6  # 1e-7 is below the floor: never reached
    assert r["sigma"] < 2.0 ** -20 * abs(r["estimate"])
    assert r["flags"] & V.RESULT_FP32_FLOOR
    assert abs(r["estimate"] - 1.0) < 3.0 * max(r["sigma"], 2.0 ** -20)
    w = V.Vegas(2, 50, 0, 0.5, 0.75, precision=V.FP64, rtol=1e-7)
    q = w.integrate(W.LINEAR, [], 2_000_000, 6, seed=0)
    assert not q["flags"] & V.RESULT_FP32_FLOOR
    u = V.Vegas(4, 50, 0, 0.5, 0.75, precision=V.FP32)
    q = u.integrate(W.GAUSS_SUM, W.ridge4_params(), 100_000, 3, seed=0)
    assert not q["flags"] & V.RESULT_FP32_FLOOR  # sigma/I ~ 1e-3


def test_batch_chi2_flag(V):
    probs = [dict(dim=12, integrand=W.GAUSS_SUM, params=W.ridge(12, 4, 0.03), neval=10_000_000, exact=1.0),
             dict(dim=4, integrand=W.GAUSS_SUM, params=W.ridge4_params(), neval=100_000, exact=1.0)]
    b = V.Batch(probs, 50, 0.5, 0.75, seed=0)
    out, _, _ = b.integrate(40)
    assert out[0]["flags"] & V.RESULT_CHI2_HIGH
    assert not out[1]["flags"] & V.RESULT_CHI2_HIGH


def test_ecuda_from_a_capturing_stream():
    code = textwrap.dedent("""
        import sys, torch
        sys.path.insert(0, %r)
        from paper_2408_09229_gb300 import vegas as V, workloads as W
        s = torch.cuda.Stream()
        v = V.Vegas(4, 50, 0, 0.5, 0.75, stream=s)
        v.integrate(W.GAUSS_SUM, W.ridge4_params(), 100_000, 1)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        status = None
        try:
            with torch.cuda.graph(g, stream=s):
                status = V.lib.vegas_reset_map(v._h)
        except RuntimeError:
            pass
        torch.cuda.synchronize()
        # the handle is still usable on its own stream afterwards
        v.set_stream(None)
        v.reset_map()
        r = v.integrate(W.GAUSS_SUM, W.ridge4_params(), 100_000, 3)
        print("STATUS", status, abs(r["estimate"] - 1.0) < 5 * r["sigma"])
    """ % ROOT)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("STATUS")][-1]
    assert line == "STATUS -3 True", r.stdout + r.stderr[-2000:]
