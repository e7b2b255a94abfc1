"""The bounds-checking build (VEGAS_BOUNDS_CHECK), the substitute for a memory
sanitizer: every index that the fill derives from data (an interval from a
point, a cube from the offsets, a slot of the tile's shared arrays, a bin of
the histogram) is checked on the device, and a failed check sets bit 3 of the
caller's flag word and is replaced by a safe index.  The workloads below cover
the fill's paths (FP64 and FP32, the exact-width and general array paths, the
streamed 16- and 32-axis paths with the map table in shared and in global
memory, the step entry point at both tile sizes, the learned proposal's points
and tabulated passes, the batched fill, cubes longer than a tile, ragged last
tiles) and must run with no check failing.  They run in a child process that
loads libvegas_gb300_check.so through VEGAS_GB300_LIB.
"""
import json
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import json, sys
    import numpy as np
    import torch
    sys.path.insert(0, %r)
    from paper_2408_09229_gb300 import vegas as V, workloads as W
    assert V.LIB_PATH.endswith("libvegas_gb300_check.so"), V.LIB_PATH
    out = []

    def run(name, d, iid, params, neval, nitn, precision, nstrat_axes=None, nbins=50, flow=False):
        v = V.Vegas(d, nbins, 0, 0.5, 0.75, precision=precision, nstrat_axes=nstrat_axes)
        if flow:
            v.set_flow(W.flow_params(d, seed=0, out_scale=0.05))
            v.set_flow_training(2, 5, 4096, batch=1024)
        r = v.integrate(iid, params, neval, nitn, seed=1, check=False)
        out.append({"name": name, "status": r["status"]})

    run("fp64 ridge d4", 4, W.GAUSS_SUM, W.ridge4_params(), 100_003, 4, V.FP64)
    run("fp32 ridge d4", 4, W.GAUSS_SUM, W.ridge4_params(), 100_003, 4, V.FP32)
    run("fp64 product peak d8", 8, W.PRODUCT_PEAK, W.product_peak(8, 0), 1_000_001, 3, V.FP64)
    run("fp32 ridge d8", 8, W.GAUSS_SUM, W.ridge8_params(), 2_000_000, 3, V.FP32)
    run("fp64 d5 general path", 5, W.OSCILLATORY, W.oscillatory(5, 1), 300_007, 3, V.FP64)
    run("fp32 d12 streamed", 12, W.GAUSS_SUM, W.ridge(12, 3, 0.1), 1_000_000, 3, V.FP32)
    # 2^20 cubes: at least 2^21 evaluations (two a cube)
    run("fp32 d30 streamed", 30, W.GAUSS_SUM, W.two_diagonal_ridge(30, 0.1), 3_000_000, 3, V.FP32,
        nstrat_axes=[2] * 20 + [1] * 10)
    run("fp32 N_g 1024", 4, W.LINEAR, [], 500_000, 3, V.FP32, nbins=1024)
    run("fp64 one long cube", 2, W.GAUSS_SUM, W.ridge(2, 3, 0.1), 50_000, 2, V.FP64, nstrat_axes=[1, 1])
    run("flow d6", 6, W.GAUSS_SUM, W.ridge(6, 3, 0.1), 200_000, 3, V.FP32, flow=True)
    b = V.Batch(W.batch_problems(24, seed=3, neval_range=(1e5, 3e6)), 50, 0.5, 0.75, seed=0)
    res, _, _ = b.integrate(3)
    out.append({"name": "batched", "status": max((r["status"] for r in res), key=abs)})
    b.reset()
    b.set_tile(10)
    res, _, _ = b.integrate(3)
    out.append({"name": "batched, tiles of 1024", "status": max((r["status"] for r in res), key=abs)})
    # the step entry point: the caller's flag word itself
    cfg_d, G, neval = 4, 50, 100_000
    nh = 14 ** 4
    sb = V.fill_scratch_bytes(cfg_d, G, [14] * 4, neval)
    scratch = torch.empty(sb, dtype=torch.uint8, device="cuda")
    off = torch.empty(nh + 1, dtype=torch.int64, device="cuda")
    asc = torch.empty(V.allocate_scratch_bytes(nh), dtype=torch.uint8, device="cuda")
    V.allocate(None, nh, neval, True, off, asc)
    edges = torch.tensor(np.tile(np.linspace(0, 1, G + 1), (cfg_d, 1)), dtype=torch.float64, device="cuda")
    ell = torch.empty(nh, dtype=torch.float32, device="cuda")
    bins = torch.zeros(cfg_d * G, dtype=torch.float64, device="cuda")
    result = torch.zeros(2, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = torch.tensor(W.ridge4_params(), dtype=torch.float64, device="cuda")
    for prec in (V.FP64, V.FP32):
        for tl in (0, 10, 11):  # the library's tile, then each tile size forced (both exact-d instances)
            V.fill(cfg_d, G, [14] * 4, prec, W.GAUSS_SUM, p, neval, 0, 0, 0.75, edges, off, ell, bins, result, flags,
                   scratch, tile_log2=tl)
    torch.cuda.synchronize()
    out.append({"name": "step fill flags", "status": int(flags[0])})
    print("RESULT " + json.dumps(out))
""") % ROOT


def test_bounds_checking_build_runs_every_path_clean():
    from paper_2408_09229_gb300 import build_lib
    lib = build_lib.build(check=True)
    env = dict(os.environ, VEGAS_GB300_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    rows = json.loads(line[len("RESULT "):])
    assert len(rows) == 13
    bad = [row for row in rows if row["status"] != 0]
    assert not bad, bad
