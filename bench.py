"""Benchmark of the GB300 VEGAS+ iteration loop.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Workload: plain VEGAS+ on the d = 8 unit cube.  The integrand is a sum of 5
isotropic Gaussians (sigma 0.05) on the main diagonal, normalised to an
integral of exactly 1.  The run uses 50 intervals per axis, 9 strata per axis
(9^8 = 43,046,721 hypercubes, about 2 evaluations each), beta = 0.75 and
alpha = 0.5, with 1e8 evaluations per iteration and Philox seed 0.  A step is
one whole iteration (allocation, fill, map refinement, combination) over 1e8
evaluations.
The headline line times plain VEGAS+ in FP64 throughout, the paper's
precision.  The chosen form, FP32 evaluation with compensated FP32 cube sums
and FP64 across cubes, is timed beside it with its error against the FP64
oracle on the same points, together with the time each takes to reach a
relative error of 1e-4.

Timing: W warm-up iterations, then K timed iterations in one integrate call.
The call sits between a barrier and a device synchronisation on both sides.
Per-iteration device time comes from CUDA events that the library records on
its stream.  The per-cube arrays (0.5 GB) are larger than L2.  --gpus N > 1
runs N independent replicas, one process per GPU under torchrun.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "evals/s and time to 1e-4 rel. error, chosen form vs plain VEGAS+, 1 GB300"
D, NBINS, NSTRAT, ALPHA, BETA, NEVAL, NITN, SEED, K_PEAKS, SIGMA = 8, 50, 9, 0.5, 0.75, 100_000_000, 15, 0, 5, 0.05
WORKLOAD = ("plain VEGAS+ d=8, ridge of 5 Gaussians (s=0.05) on the diagonal, Ng=50, 9^8 cubes, "
            "1e8 evals/iteration, beta=0.75, alpha=0.5, Philox seed 0")
# nominal SM facts of GB300 (152 SMs, 128 FP32 lanes per SM, 2070 MHz maximum SM clock)
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) of one launch of the dominant kernel on this workload, from one ncu capture of
# that kernel (dram__bytes_read.sum + dram__bytes_write.sum): the per-cube offsets and weights
FILL_TRAFFIC_BYTES = (345.26 + 144.44) * 1e6
# the same for the FP64 form's fill kernel (profiles/fill_kernel_ridge8_fp64.md)
FILL64_TRAFFIC_BYTES = (350.64 + 145.65) * 1e6
# the same capture: issue slots busy and warp instructions x 32 per evaluation (1.685e9 x 32 / 1e8)
FILL_ISSUE_ACTIVE = 0.679
FILL_INSTR_PER_EVAL = 539
# the FP32 form's evaluation-rounding floor relative to |I| (the library flags results below it)
FP32_FLOOR = 2.0 ** -20


def measured_hbm_gbs():
    """HBM copy bandwidth measured on the GB300s (MEASURED_PEAKS.json at the repository root), else the
    fallback figure of one earlier GB300 measurement"""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def pipe_ops_per_eval(d=D, K=K_PEAKS):
    """FMA-pipe operations the method needs per evaluation of the d-dimensional ridge, counted from the
    algorithm; the same count holds for the FP32 pipe in the FP32 form and the FP64 pipe in the FP64 form, which
    adds K exp() calls (the FP32 form's K ex2 run on the special-function unit):
      point + map, per axis: c+u, *g, z-i, fma(dz,dx,e), J*=jk        -> 5 d
      integrand, per peak:   per axis x-mu, fma(dx,dx,r2); r2*c; acc+= -> K (2 d + 2)
      A*acc, v = J f, v*v, *1/n_h                                      -> 4"""
    return 5 * d + K * (2 * d + 2) + 4


def sample_clocks(stop, out):
    cmd = ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-i", str(int(os.environ.get("LOCAL_RANK", 0))), "-lms", "100"]
    try:
        p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return
    def reader():
        for line in p.stdout:
            out.append(line.strip())
    th = threading.Thread(target=reader, daemon=True)
    th.start()
    stop.wait()
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    th.join(timeout=2)


def summarize_clocks(lines):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 7:
            continue
        try:
            sm.append(float(f[0]))
            mx.append(float(f[1]))
        except ValueError:
            continue
        for name, v in zip(names, f[3:7]):
            if v.lower().startswith("active"):
                reasons.add(name)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def _json_default(o):
    """numpy scalars and arrays in the bench line"""
    if isinstance(o, np.generic):
        return o.item()
    if isinstance(o, np.ndarray):
        return o.tolist()
    raise TypeError(f"not JSON serialisable: {type(o).__name__}")


def dist_setup(gpus):
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if gpus > 0 else "gloo"
        dist.init_process_group(backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def stress_d30(V, W, stream, rank):
    """The high-dimensional workload: d = 30, 6 Gaussian peaks (s = 0.1) on the main and the anti-diagonal,
    2 strata on axes 0-19 and 1 on axes 20-29 (2^20 cubes), 4e8 evaluations per iteration, 20 iterations,
    FP32 form: plain VEGAS+ and with the learned proposal (trained online over the first 10 iterations,
    the estimate combining the last 10); plain FP64 timed for 2 iterations beside them, and run to 20
    iterations at 4e7 evaluations (the FP64 reference of what plain VEGAS+ converges to here)."""
    import torch
    d, neval, nitn = 30, 400_000_000, 20
    ns = [2] * 20 + [1] * 10
    params = W.two_diagonal_ridge(d, 0.1)
    out = {"workload": "d=30, 6 peaks (s=0.1) on two diagonals, strata 2 on axes 0-19, 1 on 20-29, "
                       "4e8 evals/iteration, Ng=50, beta=0.75, alpha=0.5"}
    arms = (("fp32_form", V.FP32, nitn, neval), ("learned_proposal", V.FP32, nitn, neval),
            ("learned_proposal_judged", V.FP32, nitn, neval), ("plain_fp64", V.FP64, 2, neval),
            ("plain_fp64_4e7x20", V.FP64, nitn, neval // 10))
    for pname, prec, its, ne in arms:
        v = V.Vegas(d, NBINS, 0, ALPHA, BETA, precision=prec, nstrat_axes=ns, stream=stream)
        flow = pname.startswith("learned_proposal")
        if flow:
            v.set_flow(W.flow_params(d, seed=0))
        v.integrate(W.GAUSS_SUM, params, ne, 1, seed=5)  # sizes the buffers outside the clock
        v.reset_map()
        if flow:
            v.set_flow(W.flow_params(d, seed=0))  # untrained again: the sizing call above ran no training
            v.set_flow_training(**FLOW_TRAIN)
            v.set_skip(FLOW_TRAIN["iterations"])
            if pname == "learned_proposal_judged":
                v.set_flow_judge(JUDGE_WINDOW)
        torch.cuda.synchronize()
        r = v.integrate(W.GAUSS_SUM, params, ne, its, seed=SEED + rank)
        it_ms, fill_ms = v.timings()
        pull = (r["estimate"] - 1.0) / r["sigma"] if r["sigma"] > 0 else None
        out[pname] = {"evals_per_s": r["neval_total"] / (float(np.sum(it_ms)) / 1e3), "iterations": its,
                      "neval_per_iteration": ne,
                      "ms_per_iteration": float(np.mean(it_ms)), "fill_ms": float(np.mean(fill_ms)),
                      "estimate": r["estimate"], "sigma": r["sigma"], "chi2_dof": r["chi2_dof"],
                      "pull_from_exact": pull, "chi2_high": bool(r["flags"] & V.RESULT_CHI2_HIGH),
                      "judge": judge_summary(V, r),
                      # correct: within 3 sigma of the exact integral, with chi2/dof under its bound
                      "correct": bool(pull is not None and abs(pull) <= 3 and not r["flags"] & V.RESULT_CHI2_HIGH)}
        v.close()
    out["note"] = ("no form finds every peak of this integrand: a run is correct only when its estimate lies "
                   "within 3 sigma of 1 and its chi2/dof is under the bound")
    return out


def judge_summary(V, r):
    """the judge's decision in a result (vegas_set_flow_judge), or None when it made none"""
    if not r["flags"] & (V.RESULT_FLOW_OFF | V.RESULT_FLOW_KEPT):
        return None
    return {"kept": "learned_proposal" if r["flags"] & V.RESULT_FLOW_KEPT else "plain",
            "variance_time_ratio_plain_over_flow": r["judge_ratio"], "plain_iterations_beside": r["nitn_judge"]}


FLOW_TRAIN = dict(iterations=10, steps_per_iteration=200, samples=65536, batch=4096, lr=1e-3, temper=0.5, floor=0.03)
# a slower anneal for the narrow 4-peak ridge in d = 12: the training target starts at |f|^0.03 (peaks about six
# times wider) and sharpens over 20 iterations of 500 steps, so that the flow can reach peaks that plain VEGAS+
# never samples
FLOW_TRAIN_TEMPERED = dict(iterations=20, steps_per_iteration=500, samples=65536, batch=4096, lr=2e-3, temper=0.03,
                           floor=0.03)
# exploration before the run (vegas_flow_explore): 16 VEGAS+ maps adapted from uniform with their own seeds, 10
# iterations each at the run's budget, 32768 samples of each pooled by the balance heuristic, 2000 Adam steps; then
# two rounds of 2000 steps on as many samples of the flow itself
FLOW_EXPLORE = dict(iterations=10, maps=16, samples_per_map=32768, steps=2000, batch=4096, lr=1e-3, floor=0.03,
                    rounds=3)
FLOW_EXPLORE_CAP = 400
# the exploration's seeds (+ rank): the first is the arm `flow_explored`, the others `flow_explored_seed<s>`
FLOW_EXPLORE_SEEDS = (100, 200, 300, 400)
# iterations after training over which the judge compares the learned proposal with plain VEGAS+
JUDGE_WINDOW = 3


def learned_proposal(V, W, stream, rank):
    """The learned proposal against plain VEGAS+ (both FP32 form) on diagonal ridges: in d = 12 the
    4-peak ridge of width 0.03 (1e7 evaluations per iteration) and a 3-peak ridge of width 0.1 (1e6),
    and in d = 8 the 5-peak ridge of width 0.05 of the main workload (1e7), from a fresh map, until
    the combined sigma <= 1e-4 |I| or the iteration cap.  The flow trains for 2000 Adam steps
    (10 iterations x 200, minibatches of 4096 from 65536 weighted evaluations per iteration); its
    estimate combines the iterations after training (lagged weights, the handle default with a flow); the
    3-peak ridge runs up to 1200 iterations, enough
    for the flow to reach 1e-4 where plain VEGAS+ stops at a wrong value.  variance_time_ratio compares the steady state:
    (sigma_t^2 x iteration time) of plain VEGAS+ over that of the flow, above 1 where the flow reaches
    a given error sooner once trained.  The last two rows are the paper's Ridge integrand (Table 3 (8), 100
    Gaussians along the diagonal of the 8-cube) at 1e6 and 1e7 evaluations per iteration.  On the 4-peak ridge
    the flow is also trained by exploration alone (vegas_flow_explore: 16 maps with their own seeds, pooled by the
    balance heuristic, two more rounds on the flow's own samples, then the run under the fixed flow), once per
    exploration seed, exploration inside the timed region."""
    import torch
    out = {"training": dict(FLOW_TRAIN, adam_steps=FLOW_TRAIN["iterations"] * FLOW_TRAIN["steps_per_iteration"]),
           "training_tempered": FLOW_TRAIN_TEMPERED, "exploration": dict(FLOW_EXPLORE, seeds=FLOW_EXPLORE_SEEDS)}
    tube = W.paper_ridge(8, 100)
    cases = [("d12_4peaks_s0.03", 12, W.ridge(12, 4, 0.03), 1.0, 10_000_000, 40, 40),
             ("d12_3peaks_s0.1", 12, W.ridge(12, 3, 0.1), 1.0, 1_000_000, 1200, 1200),
             ("d8_5peaks_s0.05", 8, W.ridge(8, 5, 0.05), 1.0, 10_000_000, 60, 60),
             # the paper's Ridge (Table 3 (8)) with 100 Gaussians in d = 8: a thin tube along the diagonal that a
             # separable map cannot follow; both budgets, plain run until it reaches 1e-4
             ("d8_paper_ridge_N100_1e6", 8, tube, W.exact(W.GAUSS_SUM, 8, tube), 1_000_000, 9000, 400),
             ("d8_paper_ridge_N100_1e7", 8, tube, W.exact(W.GAUSS_SUM, 8, tube), 10_000_000, 300, 300)]
    for name, d, params, exact, neval, cap_plain, cap_flow in cases:
        row = {}
        forms = ("plain", "flow", "flow_judged") + (
            ("flow_tempered",) + tuple("flow_explored" + ("" if i == 0 else f"_seed{sd}")
                                       for i, sd in enumerate(FLOW_EXPLORE_SEEDS))
            if name.startswith("d12_4peaks") else ())
        for form in forms:
            cap = cap_plain if form == "plain" else cap_flow
            train = FLOW_TRAIN_TEMPERED if form == "flow_tempered" else FLOW_TRAIN
            if form == "flow_tempered":
                cap = train["iterations"] + 30
            explored = form.startswith("flow_explored")
            if explored:
                cap = FLOW_EXPLORE_CAP
                ex_seed = FLOW_EXPLORE_SEEDS[0] if form == "flow_explored" else int(form.rsplit("seed", 1)[1])
            v = V.Vegas(d, NBINS, 0, ALPHA, BETA, precision=V.FP32, rtol=1e-4, stream=stream)
            if form != "plain":
                v.set_flow(W.flow_params(d, seed=0))
            if form != "plain" and not explored:
                v.set_flow_training(**train)
                v.set_skip(train["iterations"])
                if form == "flow_judged":
                    v.set_flow_judge(JUDGE_WINDOW)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if explored:  # exploration and training inside the timed region
                v.flow_explore(W.GAUSS_SUM, params, neval, seed=ex_seed + rank, **FLOW_EXPLORE)
            r = v.integrate(W.GAUSS_SUM, params, neval, cap, seed=SEED + rank)
            dt = time.perf_counter() - t0
            it_ms, _ = v.timings()
            k = train["iterations"] if form != "plain" and not explored else min(10, r["nitn_run"] - 1)
            late = r["it_sig"][k:] / np.abs(r["it_est"][k:])
            pull = (r["estimate"] - exact) / r["sigma"]
            row[form] = {"seconds": dt, "iterations": r["nitn_run"], "estimate": r["estimate"], "sigma": r["sigma"],
                         "chi2_dof": r["chi2_dof"], "pull_from_exact": pull,
                         "chi2_high": bool(r["flags"] & V.RESULT_CHI2_HIGH), "judge": judge_summary(V, r),
                         "correct": bool(abs(pull) <= 3 and not r["flags"] & V.RESULT_CHI2_HIGH),
                         "reached_rtol": r["sigma"] <= 1e-4 * abs(r["estimate"]),
                         # the metric's time to a relative error of 1e-4: sigma <= 1e-4 |I| with the
                         # estimate within 3 sigma of the exact integral, else never reached (None)
                         "time_to_rtol_correct": dt if (r["sigma"] <= 1e-4 * abs(r["estimate"]) and
                                                        abs(r["estimate"] - exact) <= 3 * r["sigma"]) else None,
                         "rel_sigma_per_iteration_after_adaptation": float(np.median(late)),
                         "ms_per_iteration_after_adaptation": float(np.median(it_ms[k:]))}
            v.close()
        row["variance_per_iteration_ratio"] = (row["plain"]["rel_sigma_per_iteration_after_adaptation"] /
                                               row["flow"]["rel_sigma_per_iteration_after_adaptation"]) ** 2
        row["variance_time_ratio"] = row["variance_per_iteration_ratio"] * (
            row["plain"]["ms_per_iteration_after_adaptation"] / row["flow"]["ms_per_iteration_after_adaptation"])
        row["neval_per_iteration"] = neval
        # the learned proposal's objective: a correct 1e-4 (sigma <= 1e-4 |I| within 3 sigma of the exact
        # value) sooner than plain VEGAS+, or at all where plain VEGAS+ never gets there
        t_plain = row["plain"]["time_to_rtol_correct"]
        t_flow = [row[k]["time_to_rtol_correct"] for k in row if isinstance(row[k], dict) and k != "plain" and
                  "time_to_rtol_correct" in row[k] and row[k]["time_to_rtol_correct"] is not None]
        row["objective_met"] = bool(t_flow and (t_plain is None or min(t_flow) < t_plain))
        ex = [row[k] for k in row if k.startswith("flow_explored")]
        if ex:  # how many of the exploration seeds reach a correct 1e-4 sooner than plain VEGAS+
            row["objective_met_explored_seeds"] = "%d of %d" % (
                sum(1 for e in ex if e["time_to_rtol_correct"] is not None and
                    (t_plain is None or e["time_to_rtol_correct"] < t_plain)), len(ex))
        out[name] = row
    return out


SWEEP_DEFAULT = {"neval": 10 ** 9, "dim": 8, "nbins": 1024}
SWEEP_AXES = {"neval": [10 ** 5, 10 ** 6, 10 ** 7, 10 ** 8, 10 ** 9], "dim": [2, 4, 8, 16, 32],
              "nbins": [16, 64, 256, 1024, 4096]}


def fill_sweep(V, W, stream, args):
    """The paper's vegasFill scaling test (Sec. 4.2, its Table 4): the linear integrand, one parameter
    changed at a time around evaluations 2e10 over 20 iterations (1e9 per iteration), d = 8, N_g = 1024.
    Per point: mean fill-kernel and iteration times over the timed iterations, both forms."""
    import torch
    rows = []
    for axis, values in SWEEP_AXES.items():
        for val in values:
            cfg = dict(SWEEP_DEFAULT, **{axis: val})
            for pname, prec in (("fp32_form", V.FP32), ("plain_fp64", V.FP64)):
                v = V.Vegas(cfg["dim"], cfg["nbins"], 0, ALPHA, BETA, precision=prec, stream=stream)
                v.integrate(W.LINEAR, [], cfg["neval"], 2, seed=SEED)
                torch.cuda.synchronize()
                r = v.integrate(W.LINEAR, [], cfg["neval"], args.steps, seed=SEED + 1)
                it_ms, fill_ms = v.timings()
                rows.append({"vary": axis, **cfg, "form": pname, "fill_ms": float(np.mean(fill_ms)),
                             "iteration_ms": float(np.mean(it_ms)),
                             "fill_ns_per_eval": float(np.mean(fill_ms)) * 1e6 / cfg["neval"],
                             "rel_err": abs(r["estimate"] / (cfg["dim"] / 2.0) - 1), "sigma": r["sigma"]})
                v.close()
    return {"sweep": "fill scaling, linear integrand", "iterations_timed": args.steps, "rows": rows}


BATCH_N, BATCH_CAP, BATCH_ITERS = 256, 30, 3


def batched_form(V, W, stream, rank):
    """The batched form on 256 integrals (d uniform over 2-12, budgets log-uniform over 1e5-1e8
    evaluations per iteration, diagonal ridge / product peak / oscillatory), FP32 evaluation:
    evaluations per second and the wall time until every integral reaches sigma <= 1e-4 |I| or
    BATCH_CAP iterations, against the same integrals run one after another through vegas_integrate."""
    import torch
    probs = W.batch_problems(BATCH_N, seed=0)
    total = sum(p["neval"] for p in probs)
    b = V.Batch(probs, NBINS, ALPHA, BETA, seed=SEED + rank, stream=stream)
    tune = b.tune()
    b.reset()
    b.integrate(1)  # warm
    b.reset()
    torch.cuda.synchronize()
    _, n, ms = b.integrate(BATCH_ITERS)
    rate_batch = total * n / (ms / 1e3)
    b.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out, n_rtol, ms_rtol = b.integrate(BATCH_CAP, rtol=1e-4)
    t_batch = time.perf_counter() - t0
    pulls = np.array([(r["estimate"] - p["exact"]) / r["sigma"] for r, p in zip(out, probs) if r["sigma"] > 0])

    def err(r):  # the FP32 form's error: sigma, or its evaluation-rounding floor 2^-20 |I| where larger
        return max(r["sigma"], FP32_FLOOR * abs(r["estimate"]))
    pulls_err = np.array([(r["estimate"] - p["exact"]) / err(r) for r, p in zip(out, probs) if err(r) > 0])
    names = {W.GAUSS_SUM: "ridge", W.PRODUCT_PEAK: "product_peak", W.OSCILLATORY: "oscillatory"}
    outliers = [{"i": i, "d": p["dim"], "family": names[p["integrand"]], "neval": p["neval"],
                 "pull": (r["estimate"] - p["exact"]) / r["sigma"],
                 "pull_with_floor": (r["estimate"] - p["exact"]) / err(r),
                 "fp32_floor_flag": bool(r["flags"] & V.RESULT_FP32_FLOOR),
                 "rel_err": abs(r["estimate"] / p["exact"] - 1), "iterations": r["nitn_run"]}
                for i, (r, p) in enumerate(zip(out, probs)) if r["sigma"] > 0 and
                abs(r["estimate"] - p["exact"]) > 3 * r["sigma"]]
    evals_batch = sum(r["nitn_run"] * p["neval"] for r, p in zip(out, probs))
    conv_batch = sum(r["converged"] for r in out)
    b.close()
    # the same integrals through the plain FP64 path, for comparison
    for o in outliers[:6]:
        p = probs[o["i"]]
        v = V.Vegas(p["dim"], NBINS, 0, ALPHA, BETA, precision=V.FP64, rtol=1e-4, stream=stream)
        r = v.integrate(p["integrand"], p["params"], p["neval"], BATCH_CAP, seed=SEED + rank)
        o["plain_fp64_pull"] = (r["estimate"] - p["exact"]) / r["sigma"]
        o["plain_fp64_rel_err"] = abs(r["estimate"] / p["exact"] - 1)
        v.close()
    # the same integrals one after another through the single-integral handle
    hs = []
    for p in probs:
        v = V.Vegas(p["dim"], NBINS, 0, ALPHA, BETA, precision=V.FP32, rtol=0.0, stream=stream)
        v.integrate(p["integrand"], p["params"], p["neval"], 1, seed=5)  # sizes the buffers outside the clock
        v.reset_map()
        hs.append(v)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for v, p in zip(hs, probs):
        v.integrate(p["integrand"], p["params"], p["neval"], BATCH_ITERS, seed=SEED + rank)
    torch.cuda.synchronize()
    rate_plain = total * BATCH_ITERS / (time.perf_counter() - t0)
    for v in hs:
        v.reset_map()
        v.set_rtol(1e-4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    conv_plain, evals_plain = 0, 0
    for v, p in zip(hs, probs):
        r = v.integrate(p["integrand"], p["params"], p["neval"], BATCH_CAP, seed=SEED + 1000 + rank)
        conv_plain += r["sigma"] <= 1e-4 * abs(r["estimate"])
        evals_plain += r["neval_total"]
    t_plain = time.perf_counter() - t0
    for v in hs:
        v.close()
    return {"workload": "%d integrals, d ~ U{2..12}, neval ~ logU[1e5, 1e8] per iteration (%.3g in all), "
                        "ridge (3 peaks, s = 0.1) / product peak / oscillatory, seed 0; FP32 evaluation" % (BATCH_N, total),
            "evals_per_s": rate_batch, "plain_evals_per_s": rate_plain, "iterations_timed": BATCH_ITERS,
            "launch": tune,
            "time_to_rtol": {"rtol": 1e-4, "cap_iterations": BATCH_CAP,
                             "batched": {"seconds": t_batch, "device_ms": ms_rtol, "iterations": n_rtol,
                                         "converged": conv_batch, "evals": evals_batch},
                             "plain_one_by_one": {"seconds": t_plain, "converged": int(conv_plain),
                                                  "evals": evals_plain}},
            "pulls_from_exact": {"within_3_sigma": int((np.abs(pulls) <= 3).sum()), "n": int(len(pulls)),
                                 "within_3_errors": int((np.abs(pulls_err) <= 3).sum()),
                                 "error": "max(sigma, 2^-20 |I|): the FP32 form's rounding floor (VEGAS_RESULT_FP32_FLOOR)",
                                 "outside_3_sigma": outliers},
            "gpu_launches_per_iteration": 10}


def run_ours(args, rank, world):
    import torch
    from paper_2408_09229_gb300 import vegas as V
    from paper_2408_09229_gb300 import workloads as W

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    params = W.ridge8_params()

    def timed_run(precision, iid=W.GAUSS_SUM, prm=params):
        v = V.Vegas(D, NBINS, NSTRAT, ALPHA, BETA, precision=precision, stream=stream)
        v.integrate(iid, prm, NEVAL, args.warmup, seed=SEED + rank)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = v.integrate(iid, prm, NEVAL, args.steps, seed=SEED + rank)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        outer_ms = e0.elapsed_time(e1)
        it_ms, fill_ms = v.timings()
        return v, r, outer_ms, it_ms, fill_ms

    if args.sweep:
        if rank == 0:
            print(json.dumps(fill_sweep(V, W, stream, args)))
        return
    if args.profile_stress:
        d, neval = 30, int(args.profile_stress)
        v = V.Vegas(d, NBINS, 0, ALPHA, BETA, precision=V.FP32, nstrat_axes=[2] * 20 + [1] * 10, stream=stream)
        prm = W.two_diagonal_ridge(d, 0.1)
        v.integrate(W.GAUSS_SUM, prm, neval, args.warmup, seed=SEED)
        r = v.integrate(W.GAUSS_SUM, prm, neval, args.steps, seed=SEED + 1)
        it_ms, fill_ms = v.timings()
        if rank == 0:
            print(json.dumps({"profile": "d30 stress", "evals_per_s": neval * args.steps / (float(np.sum(it_ms)) / 1e3),
                              "iteration_ms": [float(x) for x in it_ms], "fill_ms": [float(x) for x in fill_ms]}))
        return
    if args.profile_ridge:
        # the paper's Ridge with 1000 Gaussians in d = 4 under the "def" configuration (N_g = 1024), FP32 form
        d, neval = 4, int(args.profile_ridge)
        v = V.Vegas(d, 1024, 0, 0.5, 0.75, precision=V.FP32, stream=stream)
        prm = W.paper_ridge(d, 1000)
        v.integrate(W.GAUSS_SUM, prm, neval, args.warmup, seed=5)
        r = v.integrate(W.GAUSS_SUM, prm, neval, args.steps, seed=SEED)
        it_ms, fill_ms = v.timings()
        if rank == 0:
            print(json.dumps({"profile": "ridge d4 N1000", "evals_per_s": neval * args.steps / (float(np.sum(it_ms)) / 1e3),
                              "iteration_ms": [float(x) for x in it_ms], "fill_ms": [float(x) for x in fill_ms],
                              "estimate": r["estimate"], "sigma": r["sigma"]}))
        return
    if args.profile_flow:
        d, neval = 12, 10_000_000
        v = V.Vegas(d, NBINS, 0, ALPHA, BETA, precision=V.FP32, stream=stream)
        v.set_flow(W.flow_params(d, seed=0, out_scale=0.05))
        prm = W.ridge(d, 4, 0.03)
        v.integrate(W.GAUSS_SUM, prm, neval, args.warmup, seed=SEED)
        r = v.integrate(W.GAUSS_SUM, prm, neval, args.steps, seed=SEED + 1)
        it_ms, fill_ms = v.timings()
        if rank == 0:
            print(json.dumps({"profile": "learned proposal", "evals_per_s": neval * args.steps / (float(np.sum(it_ms)) / 1e3),
                              "iteration_ms": [float(x) for x in it_ms], "fill_ms": [float(x) for x in fill_ms],
                              "estimate": r["estimate"], "sigma": r["sigma"]}))
        return
    if args.profile_grad:
        # the learned proposal's training gradient alone: 4096 seeded samples in the d-cube, exponential weights,
        # a seeded flow; 3 warm-up calls, then 200 timed ones (CUDA events)
        d, n = args.profile_grad, 4096
        th = torch.as_tensor(W.flow_params(d, seed=0, out_scale=0.05), dtype=torch.float32).cuda()
        gen = torch.Generator("cuda").manual_seed(0)
        x = torch.rand((n, d), device="cuda", generator=gen)
        wts = torch.rand(n, device="cuda", generator=gen)
        grad, loss = torch.empty_like(th), torch.empty(1, device="cuda")
        sc = torch.empty(V.flow_grad_scratch_bytes(d, n), dtype=torch.uint8, device="cuda")
        for _ in range(3):
            V.flow_grad(d, th, x, wts, grad, loss, sc)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(200):
            V.flow_grad(d, th, x, wts, grad, loss, sc)
        e1.record()
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile": "flow gradient", "dim": d, "samples": n,
                              "ms_per_gradient": e0.elapsed_time(e1) / 200}))
        return
    if args.profile_batch:
        probs = W.batch_problems(args.profile_batch, seed=0, neval_range=(1e5, args.batch_max_neval))
        b = V.Batch(probs, NBINS, ALPHA, BETA, seed=SEED, stream=stream)
        b.integrate(args.warmup)
        _, n, ms = b.integrate(args.steps)
        total = sum(p["neval"] for p in probs)
        if rank == 0:
            print(json.dumps({"profile": "batched", "integrals": len(probs), "evals_per_iteration": total,
                              "evals_per_s": total * n / (ms / 1e3), "ms_per_iteration": ms / n}))
        return
    if args.profile:
        v, r, outer_ms, it_ms, fill_ms = timed_run(V.FP32 if args.precision == "fp32" else V.FP64)
        if rank == 0:
            print(json.dumps({"profile": True, "evals_per_s": NEVAL * args.steps / (float(np.sum(it_ms)) / 1e3),
                              "fill_ms": [float(x) for x in fill_ms], "iteration_ms": [float(x) for x in it_ms],
                              "estimate": r["estimate"], "sigma": r["sigma"]}))
        return

    stop = threading.Event()
    clock_lines = []
    th = threading.Thread(target=sample_clocks, args=(stop, clock_lines), daemon=True)
    th.start()
    time.sleep(0.3)
    # the headline: plain VEGAS+ in FP64 throughout, the paper's precision
    v64, r64, outer64, it64, fill64 = timed_run(V.FP64)
    # the chosen form: FP32 evaluation with compensated cube sums, FP64 across cubes
    v32, r32, outer32, it32, fill32 = timed_run(V.FP32)
    # the second integrand of the same configuration: the product peak
    pp = W.product_peak8_params()
    pp_exact = W.exact(W.PRODUCT_PEAK, D, pp)
    pp_lines = {}
    for name, prec in (("plain_fp64", V.FP64), ("fp32_form", V.FP32)):
        _, rp, _, itp, flp = timed_run(prec, W.PRODUCT_PEAK, pp)
        pp_lines[name] = {"value": NEVAL * args.steps * world / max_over_ranks(float(np.sum(itp)) / 1e3, world),
                          "unit": "evals/s", "ms_per_step": float(np.mean(itp)), "fill_ms": float(np.mean(flp)),
                          "rel_err": rp["sigma"] / abs(rp["estimate"]),
                          "pulls_from_exact": (rp["estimate"] - pp_exact) / rp["sigma"]}
    stop.set()
    th.join(timeout=10)
    clocks = summarize_clocks(clock_lines)

    # end to end through the public call: host params in, host results out, one call per step
    def e2e(precision):
        v = V.Vegas(D, NBINS, NSTRAT, ALPHA, BETA, precision=precision, stream=stream)
        v.integrate(W.GAUSS_SUM, params, NEVAL, args.warmup, seed=SEED + rank)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            v.integrate(W.GAUSS_SUM, params, NEVAL, 1, seed=SEED + rank)
        dt = max_over_ranks(time.perf_counter() - t0, world)
        v.close()
        return {"value": NEVAL * args.steps * world / dt, "unit": "evals/s",
                # per step: the parameters in; the result (4 doubles), I_t and sigma_t and the status flag out
                "h2d_bytes_per_step": 8 * len(params), "d2h_bytes_per_step": 8 * 4 + 2 * 8 + 4}

    e2e64 = e2e(V.FP64)
    e2e32 = e2e(V.FP32)

    # time to a relative error of 1e-4 from a fresh map, both forms
    def time_to_rtol(precision):
        v = V.Vegas(D, NBINS, NSTRAT, ALPHA, BETA, precision=precision, rtol=1e-4, stream=stream)
        v.integrate(W.GAUSS_SUM, params, NEVAL, 1, seed=99)  # sizes the buffers outside the clock
        v.reset_map()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = v.integrate(W.GAUSS_SUM, params, NEVAL, 60, seed=SEED + 1000 + rank)
        dt = time.perf_counter() - t0
        return {"seconds": dt, "iterations": r["nitn_run"], "evals": r["neval_total"], "estimate": r["estimate"],
                "sigma": r["sigma"], "rel_err_reached": r["sigma"] / abs(r["estimate"]),
                "within_3_sigma_of_exact": abs(r["estimate"] - 1.0) <= 3 * r["sigma"],
                "chi2_dof": r["chi2_dof"], "chi2_high": bool(r["flags"] & V.RESULT_CHI2_HIGH)}

    ttr64 = time_to_rtol(V.FP64)
    ttr32 = time_to_rtol(V.FP32)

    # context: the paper's Table 1 workloads under its "def" configuration (Table 2: 20 iterations,
    # N_g = 1024, alpha = 0.5, beta = 0.75); "integrand evaluations" there are the run total
    sm_mhz = clocks["sm_mhz"] or 2070.0
    table1 = {}
    for name, iid, d, prm in (("roos_arnold_d10", W.ROOS_ARNOLD, 10, []),
                              ("ridge_d4_N1000", W.GAUSS_SUM, 4, W.paper_ridge(4, 1000))):
        row = {}
        for total in (10 ** 7, 10 ** 8):
            for pname, prec in (("fp32_form", V.FP32), ("plain_fp64", V.FP64)):
                if prec == V.FP64 and iid == W.GAUSS_SUM and total > 10 ** 7:
                    continue  # 1000 FP64 exponentials per evaluation: about 4 s per 1e8 on this GPU
                v = V.Vegas(d, 1024, 0, 0.5, 0.75, precision=prec, stream=stream)
                v.integrate(iid, prm, total // 20, 1, seed=5)  # sizes the buffers outside the clock
                v.reset_map()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = v.integrate(iid, prm, total // 20, 20, seed=SEED)
                dt = time.perf_counter() - t0
                _, fl = v.timings()
                cell = {"ms": dt * 1e3, "estimate": r["estimate"], "sigma": r["sigma"],
                        "fill_ms_mean": float(np.mean(fl))}
                if iid == W.GAUSS_SUM and prec == V.FP32:
                    # the evaluation kernel on a compute-heavy integrand: 1000 Gaussians, FP32-pipe roofline
                    ops = pipe_ops_per_eval(d, int(prm[2]))
                    ach = ops * (total // 20) / (float(np.mean(fl)) / 1e3) / 1e12
                    pk = FP32_LANES_PER_SM * torch.cuda.get_device_properties(local).multi_processor_count * \
                        sm_mhz * 1e6 / 1e12
                    cell["fill_fp32_roofline"] = {"ops_per_eval": ops, "achieved_tops": ach, "peak_tops": pk,
                                                  "frac": ach / pk, "peak_clock_mhz": sm_mhz}
                row[f"{pname}_{total:.0e}"] = cell
        table1[name] = row

    batched = batched_form(V, W, stream, rank)
    stress = stress_d30(V, W, stream, rank)
    learned = learned_proposal(V, W, stream, rank)

    t_dev32 = max_over_ranks(float(np.sum(it32)) / 1e3, world)
    t_dev64 = max_over_ranks(float(np.sum(it64)) / 1e3, world)
    fill_mean32 = float(np.mean(fill32)) / 1e3
    fill_mean64 = float(np.mean(fill64)) / 1e3
    evals = NEVAL * args.steps * world
    rates = V.probe_pipes()
    exp_rate = V.probe_exp64()
    atom_rate = V.probe_shared_atomics()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    hbm = measured_hbm_gbs()
    clk_hz = sm_mhz * 1e6
    # FP64 form: the FP64-pipe roofline.  The evaluation needs fp64_ops FP64-pipe operations and K exp() calls;
    # an exp costs dfma_rate / exp_rate FMA issue slots of that pipe (both rates measured on this GPU)
    ops64 = pipe_ops_per_eval()
    exp_cost = rates[1] / exp_rate
    ops64_equiv = ops64 + K_PEAKS * exp_cost
    achieved64 = ops64_equiv * NEVAL / fill_mean64 / 1e12
    peak64 = rates[1] * sms * clk_hz / 1e12
    ops32 = pipe_ops_per_eval()
    achieved32 = ops32 * NEVAL / fill_mean32 / 1e12
    peak32 = FP32_LANES_PER_SM * sms * clk_hz / 1e12
    # per steady iteration: allocation 3 (q sums, their scan, offsets; the max of the weights comes from
    # the fill), fill 6 (tile search, fill, carry runs, fix-up, results, map weights), refinement 1,
    # combination 1
    launches_per_it = 11
    line = {
        "metric": METRIC, "value": evals / t_dev64, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_dev64 / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "plain VEGAS+, FP64 throughout (the paper's precision)",
                   "neval_per_step": NEVAL, "ncubes": NSTRAT ** D, "l2": "per-cube arrays 0.5 GB > L2; no flush",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "result": {"estimate": r64["estimate"], "sigma": r64["sigma"], "chi2_dof": r64["chi2_dof"],
                   "chi2_high": bool(r64["flags"] & V.RESULT_CHI2_HIGH)},
        "e2e": e2e64,
        "roofline": {"bound": "alu", "kernel": "fill_kernel<GAUSS_SUM, double, 8, exact>", "achieved": achieved64,
                     "peak": peak64, "unit": "Tops/s (FP64-pipe FMA issue slots; one exp() = %.1f, measured)"
                     % exp_cost, "frac": achieved64 / peak64, "traffic": FILL64_TRAFFIC_BYTES,
                     "ops_per_eval": ops64, "exp_per_eval": K_PEAKS, "fill_ms": fill_mean64 * 1e3,
                     "peak_basis": "FP64 FMA rate of vegas_probe_pipes (%.2f per SM per clock) x %d SMs x %.0f MHz "
                                   "(median SM clock sampled during the run)" % (rates[1], sms, sm_mhz),
                     "probe_ops_per_sm_clk": {"ffma": rates[0], "dfma": rates[1], "exp64": exp_rate,
                                              "mufu_ex2": rates[2], "imad_hi": rates[3],
                                              "shared_atomic_add": atom_rate}},
        "chosen_form": {
            "form": "FP32 evaluation, compensated cube sums, FP64 across cubes, map refinement and combination",
            "dtype": "f32", "value": evals / t_dev32, "unit": "evals/s", "ms_per_step": t_dev32 / args.steps * 1e3,
            "result": {"estimate": r32["estimate"], "sigma": r32["sigma"], "chi2_dof": r32["chi2_dof"],
                       "chi2_high": bool(r32["flags"] & V.RESULT_CHI2_HIGH)},
            "e2e": e2e32,
            "roofline": {"bound": "alu", "kernel": "fill_kernel<GAUSS_SUM, float, 8, exact>", "achieved": achieved32,
                         "peak": peak32, "unit": "Tops/s (FP32-pipe operations, FMA = 1)", "frac": achieved32 / peak32,
                         "traffic": FILL_TRAFFIC_BYTES,
                         "issue": {"slots_busy": FILL_ISSUE_ACTIVE, "instructions_per_eval": FILL_INSTR_PER_EVAL,
                                   "source": "ncu capture of this kernel (profiles/fill_kernel_ridge8_fp32.md)"},
                         "ops_per_eval": ops32, "fill_ms": fill_mean32 * 1e3,
                         "peak_basis": "FP32 FMA pipe: 128 lanes x %d SMs x %.0f MHz (median SM clock sampled "
                                       "during the run)" % (sms, sm_mhz),
                         # the accumulation's own bounds: d shared 32-bit atomic adds per evaluation into the
                         # fixed-point histogram against the probe's rate, and the kernel's DRAM traffic
                         "accumulation": {
                             "shared_atomics_per_eval": D,
                             "achieved_per_sm_clk": D * NEVAL / (fill_mean32 * clk_hz * sms),
                             "peak_per_sm_clk": atom_rate,
                             "frac": D * NEVAL / (fill_mean32 * clk_hz * sms) / atom_rate,
                             "dram_gbs": FILL_TRAFFIC_BYTES / fill_mean32 / 1e9,
                             "dram_frac": FILL_TRAFFIC_BYTES / fill_mean32 / 1e9 / hbm[0],
                             "dram_peak_gbs": hbm[0], "dram_peak_basis": hbm[1]}},
            "speedup_over_plain_fp64": t_dev64 / t_dev32},
        "product_peak": dict(pp_lines, workload="product peak prod 1/(c^-2 + (x - w)^2), c ~ U[5,15], "
                                                "w ~ U[0.2,0.8], seed 0; same d, cubes and evaluations"),
        "time_to_rtol": {"rtol": 1e-4, "plain_fp64": ttr64, "fp32_form": ttr32},
        "batched": batched,
        "stress_d30": stress,
        "learned_proposal": learned,
        "paper_table1_context": dict(table1, note="total wall ms of 20 iterations (def configuration) through "
                                     "vegas_integrate; the paper reports 29.0/91.5 ms (Roos&Arnold) and "
                                     "149.4/1123.1 ms (Ridge) for 1e7/1e8 evaluations on one A100 in FP64"),
        "clocks": clocks,
        "gpu_launches": launches_per_it * args.steps,
        "timing_check": {"outer_event_ms": outer64, "sum_iteration_ms": float(np.sum(it64))},
    }
    if rank == 0:
        try:
            base, err = fp32_form_against_the_oracle(V, W, stream)
            line["cpu_baseline"] = base
            line["chosen_form"]["error_vs_fp64_oracle"] = err
            line["cpu_baseline_all_cores"] = cpu_baseline_all_cores()
        except Exception as e:  # the oracle build needs gcc; report instead of failing the bench
            line["cpu_baseline"] = {"error": str(e)[:200]}
        print(json.dumps(line, default=_json_default))


def fp32_form_against_the_oracle(V, W, stream):
    """The CPU baseline leg: the oracle, as it stands and single-threaded, computes in FP64 on the FP32 form's own
    points (its FP32-point mode, reading R3) from the FP32 form's own map and allocation, one iteration at a time.
    Its timing on the full-size iteration is the CPU baseline; the difference between the two iteration
    estimates is the FP32 form's error against the FP64 oracle, stated per result:
      - the 4-d ridge (3 peaks, s = 0.05), 1e5 evaluations x 10 iterations from a fresh map, every iteration
        and the combined estimate (Eq. (8) over both sides' iterations);
      - the headline workload at full size (1e8 evaluations, 9^8 cubes): the iteration after three that adapt
        the map."""
    import oracle

    def one(v, cfg, iid, prm, neval, seed):
        st = v.state_arrays()
        off = oracle.allocate(st["ell"], cfg.ncubes, neval, BETA)  # the GPU's counts: integer, bit-exact
        t0 = time.perf_counter()
        o = oracle.iteration(cfg, iid, prm, neval, st["iteration"], seed, st["edges"], off)
        dt = time.perf_counter() - t0
        g = v.integrate(iid, prm, neval, 1, seed=seed)
        return g["it_est"][0], g["it_sig"][0], o["est"], math.sqrt(o["var"]), dt

    err = {}
    d4, n4 = 4, 100_000
    p4 = W.ridge4_params()
    cfg4 = oracle.Config(d4, NBINS, oracle.default_nstrat(n4, d4), ALPHA, BETA, points_f32=True)
    v = V.Vegas(d4, NBINS, 0, ALPHA, BETA, precision=V.FP32, stream=stream)
    rows = [one(v, cfg4, W.GAUSS_SUM, p4, n4, SEED) for _ in range(10)]
    v.close()
    gI, gS, oI, oS = (np.array([r[k] for r in rows]) for k in range(4))
    cg, co = oracle.combine(gI, gS), oracle.combine(oI, oS)
    err["ridge4_1e5x10"] = {
        "iteration_rel_diff": [float(x) for x in np.abs(gI - oI) / np.abs(oI)],
        "iteration_rel_sigma": [float(x) for x in gS / np.abs(gI)],
        "combined": {"fp32_form": cg["estimate"], "fp64_oracle": co["estimate"],
                     "rel_diff": abs(cg["estimate"] - co["estimate"]) / abs(co["estimate"]),
                     "rel_sigma": cg["sigma"] / abs(cg["estimate"])}}
    cfg8 = oracle.Config(D, NBINS, NSTRAT, ALPHA, BETA, points_f32=True)
    v = V.Vegas(D, NBINS, NSTRAT, ALPHA, BETA, precision=V.FP32, stream=stream)
    v.integrate(W.GAUSS_SUM, W.ridge8_params(), NEVAL, 3, seed=SEED)
    gI8, gS8, oI8, oS8, dt = one(v, cfg8, W.GAUSS_SUM, W.ridge8_params(), NEVAL, SEED)
    v.close()
    err["ridge8_1e8_one_iteration"] = {"fp32_form": gI8, "fp64_oracle": oI8, "rel_diff": abs(gI8 - oI8) / abs(oI8),
                                       "rel_sigma": gS8 / abs(gI8), "sigma_rel_diff": abs(gS8 - oS8) / oS8}
    base = {"value": NEVAL / dt, "unit": "evals/s", "cores": 1, "kind": "oracle",
            "sample": f"one full iteration of the headline workload ({NEVAL:.0e} evals, {NSTRAT}^{D} cubes) on the "
                      f"FP32 form's adapted map and counts, FP64 arithmetic on the same points; {dt:.1f} s"}
    return base, err


def oracle_iterations_threaded(neval, nitn, threads):
    """The oracle's iterations with the fill on all host cores: each iteration splits the evaluation range into
    `threads` contiguous parts, runs the oracle's range fill on each in its own thread (ctypes releases the GIL
    for the C call), merges the partial cube statistics in range order with Chan's update and sums the map
    weights; then the oracle's cube finish, map refinement and allocation, as one oracle iteration does.
    Returns the per-iteration estimates."""
    import concurrent.futures as cf
    import oracle
    from paper_2408_09229_gb300 import workloads as W
    cfg = oracle.Config(D, NBINS, oracle.default_nstrat(neval, D), ALPHA, BETA)
    params = W.ridge8_params()
    edges = cfg.uniform_edges()
    off = oracle.allocate(None, cfg.ncubes, neval, BETA)
    est = []
    bounds = [neval * r // threads for r in range(threads + 1)]
    with cf.ThreadPoolExecutor(threads) as ex:
        for t in range(nitn):
            parts = list(ex.map(lambda r: oracle.fill_range(cfg, W.GAUSS_SUM, params, neval, t, SEED, edges, off,
                                                              bounds[r], bounds[r + 1]), range(threads)))
            n, mu, q, bins = parts[0][0].astype(np.float64), parts[0][1], parts[0][2], parts[0][3].copy()
            for n2, mu2, q2, b2 in parts[1:]:
                n2 = n2.astype(np.float64)
                nt = n + n2
                delta = mu2 - mu
                with np.errstate(invalid="ignore", divide="ignore"):
                    f = np.where(nt > 0, n2 / np.where(nt > 0, nt, 1.0), 0.0)
                mu = mu + delta * f
                q = q + q2 + delta * delta * n * f
                n = nt
                bins += b2
            I, _, ell = oracle.finish_cubes(cfg, off, mu, q)
            est.append(I)
            edges = np.stack([oracle.refine_axis(bins[k], edges[k], ALPHA)[0] for k in range(D)])
            off = oracle.allocate(ell, cfg.ncubes, neval, BETA)
    return cfg, est


def cpu_baseline_all_cores(neval=10_000_000, nitn=4):
    """the oracle's iterations with the fill split over every host core (see oracle_iterations_threaded)"""
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    cfg, _ = oracle_iterations_threaded(neval, nitn, threads)
    dt = time.perf_counter() - t0
    return {"value": neval * nitn / dt, "unit": "evals/s", "cores": threads, "kind": "oracle",
            "sample": f"{nitn} iterations x {neval:.0e} evals, the fill's evaluation range split over {threads} "
                      f"threads; {int(cfg.nstrat[0])}^8 cubes; {dt:.1f} s"}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle, as it stands, one bounded-sample iteration per step"""
    if rank != 0:
        return
    import oracle
    from paper_2408_09229_gb300 import workloads as W
    neval = 1_000_000
    cfg = oracle.Config(D, NBINS, oracle.default_nstrat(neval, D), ALPHA, BETA)
    params = W.ridge8_params()
    oracle.integrate(cfg, W.GAUSS_SUM, params, neval, max(args.warmup, 1), seed=SEED)
    t0 = time.perf_counter()
    r = oracle.integrate(cfg, W.GAUSS_SUM, params, neval, args.steps, seed=SEED)
    dt = time.perf_counter() - t0
    value = neval * args.steps / dt
    sample = (f"each step one oracle iteration of {neval:.0e} evals of the same integrand, d, Ng, alpha, beta "
              f"({int(cfg.nstrat[0])}^8 cubes); single-threaded")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "CPU oracle (plain FP64 VEGAS+)", "neval_per_step": neval},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "result": {"estimate": r["estimate"], "sigma": r["sigma"]},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=NITN)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile", action="store_true",
                    help="profiling run: only the warm-up and timed iterations of one form, a short JSON line")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="the form a --profile run times")
    ap.add_argument("--sweep", action="store_true",
                    help="fill scaling sweep of the paper's Table 4 parameters on the linear integrand")
    ap.add_argument("--profile-stress", type=float, default=0.0, metavar="NEVAL",
                    help="profiling run of the d = 30 workload (FP32 form) at NEVAL evaluations per iteration")
    ap.add_argument("--profile-ridge", type=float, default=0.0, metavar="NEVAL",
                    help="profiling run of the paper's Ridge, 1000 Gaussians in d = 4 (FP32 form), NEVAL per iteration")
    ap.add_argument("--profile-flow", action="store_true",
                    help="profiling run of the learned proposal: d = 12 ridge, 1e7 evaluations, a fixed flow")
    ap.add_argument("--profile-grad", type=int, default=0, metavar="D",
                    help="profiling run of the learned proposal's training gradient in D dimensions (4096 samples)")
    ap.add_argument("--profile-batch", type=int, default=0, metavar="N",
                    help="profiling run of the batched form on the first N integrals of the batched workload")
    ap.add_argument("--batch-max-neval", type=float, default=1e8,
                    help="upper end of the log-uniform budgets of a --profile-batch run")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank, world = dist_setup(args.gpus if args.impl == "ours" else 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        import __graft_entry__
        __graft_entry__.build()
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
