"""World-size-2 gloo tests of the multi-process paths, on CPU.

* Sharding of an iteration over evaluation ranges (Sec. 3.4 of the paper: the
  evaluations are split evenly across devices and the fill results merged):
  each rank fills its half of [0, neval) with the oracle, the ranks gather
  the per-cube partial statistics and merge them in rank order, and sum the
  map weights.  The merged result equals the single-process fill.
* The benchmark's replica timing: the job time is the maximum over ranks.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _merge(n1, m1, q1, n2, m2, q2):
    n = n1 + n2
    delta = m2 - m1
    safe = np.maximum(n, 1)
    mean = np.where(n > 0, m1 + delta * n2 / safe, 0.0)
    q = q1 + q2 + np.where(n > 0, delta * delta * n1 * n2 / safe, 0.0)
    return n, mean, q


def _worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2408_09229_gb300 import workloads as W
    import bench
    cfg = oracle.Config(4, 20, 5, 0.5, 0.75)
    neval = 20_001
    ell = np.random.default_rng(0).normal(0, 3, cfg.ncubes).astype(np.float32)
    off = oracle.allocate(ell, cfg.ncubes, neval, 0.75)
    edges = cfg.uniform_edges()
    params = W.ridge(4, 3, 0.1)
    lo, hi = rank * neval // world, (rank + 1) * neval // world
    cnt, mean, m2, bins = oracle.fill_range(cfg, W.GAUSS_SUM, params, neval, 1, 3, edges, off, lo, hi)
    parts = [torch.zeros(3, cfg.ncubes, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, torch.tensor(np.stack([cnt.astype(np.float64), mean, m2])))
    b = torch.tensor(bins.ravel())
    dist.all_reduce(b)
    n, mu, q = parts[0][0].numpy(), parts[0][1].numpy(), parts[0][2].numpy()
    for r in range(1, world):
        n, mu, q = _merge(n, mu, q, parts[r][0].numpy(), parts[r][1].numpy(), parts[r][2].numpy())
    t = bench.max_over_ranks(float(rank + 1), world, device="cpu")
    if rank == 0:
        np.savez(out_path, n=n, mean=mu, m2=q, bins=b.numpy(), tmax=t)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_fill_equals_single_fill(tmp_path, orc):
    from paper_2408_09229_gb300 import workloads as W
    out = str(tmp_path / "merged.npz")
    port = 29500 + os.getpid() % 1000
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    got = np.load(out)
    cfg = orc.Config(4, 20, 5, 0.5, 0.75)
    neval = 20_001
    ell = np.random.default_rng(0).normal(0, 3, cfg.ncubes).astype(np.float32)
    off = orc.allocate(ell, cfg.ncubes, neval, 0.75)
    cnt, mean, m2, bins = orc.fill_range(cfg, W.GAUSS_SUM, W.ridge(4, 3, 0.1), neval, 1, 3, cfg.uniform_edges(),
                                         off, 0, neval)
    assert np.array_equal(got["n"], cnt)
    assert np.allclose(got["mean"], mean, rtol=1e-13)
    assert np.allclose(got["m2"], m2, rtol=1e-9, atol=1e-12 * m2.max())
    assert np.allclose(got["bins"], bins.ravel(), rtol=1e-13)
    assert float(got["tmax"]) == 2.0
