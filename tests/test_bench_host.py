"""Host logic of bench.py that needs no GPU: the all-cores CPU baseline runs the oracle's iterations with the
fill's evaluation range split over threads, and must reproduce the single-threaded oracle's iterations."""
import numpy as np
import pytest

import bench
from paper_2408_09229_gb300 import workloads as W


def test_threaded_oracle_iterations_match_the_oracle(orc):
    neval, nitn = 60_000, 3
    _, est = bench.oracle_iterations_threaded(neval, nitn, 3)
    cfg = orc.Config(bench.D, bench.NBINS, orc.default_nstrat(neval, bench.D), bench.ALPHA, bench.BETA)
    ref = orc.integrate(cfg, W.GAUSS_SUM, W.ridge8_params(), neval, nitn, seed=bench.SEED)
    # the same samples, cubes and map; only the order of the per-cube sums differs
    assert np.allclose(est, ref["it_est"], rtol=1e-12, atol=0)


def test_measured_hbm_peak_is_positive():
    gbs, basis = bench.measured_hbm_gbs()
    assert gbs > 0 and basis in ("measured", "fallback")


def test_reference_arm_under_torchrun_prints_once():
    """two ranks launched as the driver launches them: rank 0 alone runs the oracle and prints one JSON line,
    the other rank exits 0 without work"""
    import json
    import os
    import socket
    import subprocess
    import sys

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
