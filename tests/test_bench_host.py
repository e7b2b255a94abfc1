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
