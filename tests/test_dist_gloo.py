"""World-size-2 gloo tests of the multi-process paths, on CPU.

* Sharding of an iteration over evaluation ranges (Sec. 3.4 of the paper: the
  evaluations are split evenly across devices and the fill results merged):
  each rank fills its half of [0, neval) with the oracle, the ranks gather
  the per-cube partial statistics and merge them in rank order, and sum the
  map weights.  The merged result equals the single-process fill.
* The benchmark's replica timing: the job time is the maximum over ranks.
* Failure detection on the host: a rank that leaves between steps makes the
  other rank's next collective end with an error within the process group's
  timeout (no device is involved).
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


def _leaver(rank, world, port, out_path):
    """rank 1 leaves between steps (after the first step's collective, with nothing in flight); rank 0 learns of
    it on the host: its next collective ends with an error within the process group's short timeout instead of
    waiting forever"""
    import datetime
    import time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=3))
    t = torch.ones(4)
    dist.all_reduce(t)  # step 1: both ranks
    if rank == 1:
        os._exit(0)  # leaves without a goodbye
    t0 = time.perf_counter()
    err = ""
    try:
        dist.all_reduce(t)  # step 2: the peer is gone
    except Exception as e:  # gloo reports a closed connection or a timeout
        err = type(e).__name__ + ": " + str(e)[:200]
    np.savez(out_path, err=np.array(err), dt=time.perf_counter() - t0, first=t.numpy())


def test_rank_that_leaves_is_detected_on_the_host(tmp_path):
    out = str(tmp_path / "leave.npz")
    port = 29700 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_leaver, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = np.load(out)
    assert str(got["err"]), "the collective with a departed rank returned without an error"
    assert float(got["dt"]) < 60.0
    assert np.all(got["first"] == 2.0)
