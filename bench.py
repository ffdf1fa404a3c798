#!/usr/bin/env python
"""Benchmark: space-time DOF/s of a full MGRIT solve on one GB300, against
GPU sequential time-stepping and the CPU oracle.

Default line (one "step" = one whole solve, every row of the hot path):
  1D periodic advection, nx = 16384, nt = 65536, 5th-order upwind + 3-stage
  SDIRK3 (c = 4), V-cycle MGRIT with m = 16 and 5 levels, FCF relaxation,
  corrected semi-Lagrangian coarse operators (two-term correction for
  q != p), smooth random IC (20 Fourier modes), random initial iterate
  (seed 0).  `value` is the FP64 solve; FP32-relaxation variants, GPU
  sequential stepping, the 512-solve batch and a bounded window of the
  served Poisson stream are sub-records of the same line.

  The stop tolerance is 1e-11: a 1e-10 relative residual leaves an error of
  about 1.7e-10 against sequential stepping on this problem (the error is
  bounded only by ||A^{-1}|| ||r||), and every C-point is meant to be within
  1e-10 of it; the line reports that error over all C-points.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs are independent replicas (one solve per rank): value = N *
DOF / max-over-ranks time; with --sharded, one solve is time-sharded over
the ranks (strong scaling).
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # 16384 x 65536, U5 + SDIRK3 (c = 4), m = 16, 5 levels: the largest
    # single-GPU configuration, solved in FP64 (the variants add FP32
    # relaxation in FP64 refinement)
    "c3": dict(name="advection1d_sdirk3u5_vcycle", nx=16384, nt=65536, p=5, kind="sdirk", q=3,
               cfl=4.0, m=16, levels=5, nu=1, tol=1e-11, max_iter=40, seed=0, ic="fourier20",
               precision="fp64"),
    # 4096 x 16384, ERK3+U3, FP64, 4-level V-cycle (m = 8)
    "c2": dict(name="advection1d_erk3u3_vcycle", nx=4096, nt=16384, p=3, kind="erk", q=3, cfl=0.85,
               m=8, levels=4, nu=1, tol=1e-11, max_iter=40, seed=0, ic="sin4_noise", precision="fp64"),
    # 256 x 1024, ERK1+U1, FP64, two-level m = 4
    "c1": dict(name="advection1d_erk1u1_twolevel", nx=256, nt=1024, p=1, kind="erk", q=1, cfl=0.85,
               m=4, levels=2, nu=1, tol=1e-11, max_iter=40, seed=0, ic="sin4", precision="fp64"),
}
WORKLOAD = WORKLOADS["c3"]
METRIC = "space-time DOF/s to 1e-10 residual vs GPU seq. stepping; p50/p99 latency"
UNIT = "DOF/s"
# FP64 FMA pipe: 152 SMs x 2 FP64 FMA/clk/SM (4 flop/clk/SM) x 2.07 GHz
FP64_PEAK_FLOPS = 152 * 4 * 2.07e9
# FP32 FMA pipe: 152 SMs x 128 FP32 FMA/clk/SM (256 flop/clk/SM) x 2.07 GHz
FP32_PEAK_FLOPS = 152 * 256 * 2.07e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (ms): every rank gets the max (an all-reduce on
    `device`; NCCL on GPUs, gloo on CPU).  Without a process group: ms."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(dof_per_rank, steps, max_ms, ws):
    """Whole-job throughput of replicas (weak scaling): the DOF every rank
    solved in `steps` steps, over the slowest rank's time."""
    return ws * dof_per_rank * steps / (max_ms / 1e3)


def clocks_sampler_start(path):
    try:
        f = open(path, "w")
        p = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def clocks_sampler_stop(p, f, path, device):
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    f.close()
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(device):
            continue
        try:
            sm.append(float(parts[1]))
            mx = float(parts[2])
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def make_ic(w, seed=None):
    from workloads import ic_fourier, ic_sin4, ic_sin4_noise
    seed = w["seed"] if seed is None else seed
    if w["ic"] == "sin4_noise":
        return ic_sin4_noise(w["nx"], seed=seed)
    if w["ic"] == "fourier20":
        return ic_fourier(w["nx"], seed=seed)
    return ic_sin4(w["nx"])


def _oracle_sample(job):
    """One oracle solve (plain numpy FP64 MGRIT, as it stands) on a bounded
    sample of a workload: the same nx, scheme, m and tolerance over the
    first `nt` steps.  Runs in a pool worker; returns (DOF, seconds,
    iterations)."""
    from oracle import mgrit as omg
    w, nt, levels, seed = job
    h = omg.Hierarchy(w["p"], w["kind"], w["q"], w["cfl"], w["m"], levels)
    u0 = make_ic(w, seed)
    t = time.perf_counter()
    r = omg.solve(h, u0, nt, nu=w["nu"], tol=w["tol"], max_iter=w["max_iter"], seed=w["seed"])
    return w["nx"] * nt, time.perf_counter() - t, r["iterations"]


def _oracle_import(_):
    from oracle import mgrit  # noqa: F401
    return 0


def _sample_levels(w, nt):
    levels = w["levels"]
    while levels > 2 and nt % (w["m"] ** (levels - 1)):
        levels -= 1
    return levels


def cpu_baseline(w, sample_nt, workers=None):
    """The CPU oracle on the host cores: one independent sample solve per
    core (a process pool, spawn start method, one BLAS/OpenMP thread per
    worker), each the workload's nx, scheme, m and tolerance over the first
    sample_nt steps with its own IC seed.  value = the DOF all workers
    solved / the wall time of the round."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    workers = workers or cores
    sample_nt = min(sample_nt, w["nt"])
    levels = _sample_levels(w, sample_nt)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    jobs = [(w, sample_nt, levels, w["seed"] + i) for i in range(workers)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_import, range(workers))  # start the workers and import, untimed
        t = time.perf_counter()
        res = pool.map(_oracle_sample, jobs)
        wall = time.perf_counter() - t
    dof = sum(r[0] for r in res)
    its = sorted(r[2] for r in res)
    return {"value": dof / wall, "unit": UNIT, "cores": workers, "kind": "oracle",
            "host_cpu_count": cores,
            "sample": "%d independent solves (one per core, spawn pool), each nx=%d, nt=%d (the first %d of %d "
                      "steps), same scheme/m/tol, %d levels, %d-%d iterations; %.1f s wall"
                      % (workers, w["nx"], sample_nt, sample_nt, w["nt"], levels, its[0], its[-1], wall)}


def batched_record(count, steps, warmup, tol=1e-11, implicit=False):
    """The batched workload: `count` independent solves (nx, nt, p, c, m
    mixed; ERK of matching order, or with implicit=True SDIRK of order
    min(p, 3)), FP32 relaxation in FP64 refinement, captured into one CUDA
    graph and run with one launch; against GPU sequential stepping of the
    same problems, all at once over the batch's streams, and against FP64
    single-solve MGRIT of a sample.  value = total DOF / batch time."""
    import torch
    import paper_2209_06916_gb300 as pkg
    from workloads import batch_mix, batch_mix_sdirk, ic_fourier, ic_sin4_noise
    kind = pkg.SDIRK if implicit else pkg.ERK
    if implicit:
        mix = batch_mix_sdirk(count, seed=3000)
        u0h = [ic_fourier(d["nx"], seed=d["seed"]) for d in mix]
    else:
        mix = batch_mix(count, seed=1000)
        u0h = [ic_sin4_noise(d["nx"], seed=d["seed"]) for d in mix]
    prms = [pkg.make_params(d["nx"], d["nt"], d["cfl"], d["p"], kind=kind, q=d.get("q", d["p"]), m=d["m"], levels=0,
                            nu=1, tol=tol, max_iter=60, precision=pkg.MIXED, seed=d["seed"]) for d in mix]
    u0s = [torch.tensor(u, dtype=torch.float64, device="cuda") for u in u0h]
    t0 = time.perf_counter()
    b = pkg.Batch(prms, nstreams=32)
    setup_s = time.perf_counter() - t0
    dof = b.dof()
    for _ in range(warmup):
        b.solve(u0s, allow_unconverged=True)
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        st = b.solve(u0s, allow_unconverged=True)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    dt = float(np.median(ts))
    its = [x["iterations"] for x in st]
    conv = sum(1 for x in st if x["converged"])
    outs = [torch.empty(d["nx"], dtype=torch.float64, device="cuda") for d in mix]
    b.sequential(u0s, outs)
    torch.cuda.synchronize()
    sts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        b.sequential(u0s, outs)
        torch.cuda.synchronize()
        sts.append(time.perf_counter() - t0)
    sdt = float(np.median(sts))
    # accuracy: the final C-point row of a sample of the solves against their
    # sequential stepping
    err = 0.0
    for i in range(0, count, max(1, count // 8)):
        last = b.get(i)[-1]
        ref = outs[i].cpu().numpy()
        err = max(err, float(np.max(np.abs(last - ref)) / np.max(np.abs(ref))))
    b.close()
    # plain FP64 single-solve MGRIT on a sample of the same problems (every
    # 8th), one solve at a time after a warm-up solve of each
    single_dof, single_s = 0, 0.0
    for i in range(0, count, 8):
        d = mix[i]
        p64 = pkg.make_params(d["nx"], d["nt"], d["cfl"], d["p"], kind=kind, q=d.get("q", d["p"]), m=d["m"], levels=0,
                              nu=1, tol=tol, max_iter=60, precision=pkg.FP64, seed=d["seed"])
        s = pkg.Solver(p64)
        out = torch.empty((d["nt"] // d["m"] + 1, d["nx"]), dtype=torch.float64, device="cuda")
        s.solve(u0s[i], out, allow_unconverged=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.solve(u0s[i], out, allow_unconverged=True)
        torch.cuda.synchronize()
        single_s += time.perf_counter() - t0
        single_dof += d["nx"] * d["nt"]
        s.close()
    single_rate = single_dof / single_s
    # FP64 floor: every refinement step needs one FP64 level-0 residual, the
    # composite stencil Phi^m over all intervals; for ERKp+Up its flops per
    # space-time point equal those of one explicit step (2 p^2 taps' worth,
    # m p^2 + 1 taps per m steps), i.e. a residual sweep costs the flops of
    # the whole sequential solve.  At the stencil kernel's 0.8 of the FP64
    # peak this bounds the batch time from below whatever the FP32 and coarse
    # work cost.
    sweeps = [x["outer_iterations"] + 1 for x in st]
    if implicit:  # the explicit-step argument does not apply
        floor = {"median": float(np.median(sweeps)), "max": int(max(sweeps)), "floor_ms": None,
                 "floor_over_sequential": None, "note": "implicit steps: a residual sweep costs far less than the "
                                                       "sequential solve's dependent stage solves"}
    else:
        fl = [2.0 * min(d["m"] * d["p"] ** 2 + 1, d["nx"]) * d["nx"] * (d["nt"] // d["m"]) for d in mix]
        floor_s = sum(k * f for k, f in zip(sweeps, fl)) / (0.8 * FP64_PEAK_FLOPS)
        floor = {"median": float(np.median(sweeps)), "max": int(max(sweeps)), "floor_ms": floor_s * 1e3,
                 "floor_over_sequential": (floor_s * 1e3) / (sdt * 1e3),
                 "note": "FP64 residual sweeps alone at 0.8 of the FP64 peak; each sweep has the flops of the whole "
                         "sequential solve"}
    return {"workload": "advection1d_batched_%d_%s_mixed" % (count, "sdirk" if implicit else "erk"),
            "value": dof / dt, "unit": UNIT,
            "fp64_residual_sweeps": floor,
            "ms_per_batch": dt * 1e3, "batches_timed": steps, "solves": count, "dof_total": dof,
            "converged": conv, "iterations_median": float(np.median(its)), "iterations_max": int(max(its)),
            "tol": tol, "setup_s": setup_s, "launch": "one CUDA graph, one branch per solve",
            "max_rel_err_final_row_vs_sequential": err, "err_sample": "every %d-th solve" % max(1, count // 8),
            "sequential": {"value": dof / sdt, "unit": UNIT, "ms": sdt * 1e3,
                           "kernel": "one sequential-stepping cluster per solve, all solves over the 32 streams"},
            "mgrit_over_sequential": sdt / dt,
            "fp64_single_solve": {"value": single_rate, "unit": UNIT, "sample": "every 8th problem, %d solves "
                                  "one at a time in FP64" % len(range(0, count, 8)), "seconds": single_s},
            "mgrit_over_fp64_single_solve": (dof / dt) / single_rate}


def run_batched(args, implicit=False):
    import torch
    torch.cuda.set_device(0)
    count = 128 if implicit and args.count == 512 else args.count
    rec = batched_record(count, args.steps, args.warmup, implicit=implicit)
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rec["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 relax / f64 residual", "data": "synthetic",
            "config": {"workload": rec["workload"]}, "batched": rec}
    print(json.dumps(line))
    return 0


def pretune_shapes(prms, max_s):
    """Set up one handle per distinct launch-geometry shape of a request
    stream (the tuner's keys: sizes, orders, m, precision and, for SDIRK,
    log2 c to one digit) on the idle GPU, so their measured geometries are
    cached before the serving clock starts; stops after max_s seconds.
    Returns (shapes tuned, shapes seen, seconds)."""
    import math
    import paper_2209_06916_gb300 as pkg
    seen, t0, tuned = {}, time.perf_counter(), 0
    for p in prms:
        key = (p.nx, p.nt, p.order_p, p.rk_kind, p.rk_order_q, p.m, p.precision,
               round(math.log2(p.cfl)) if p.rk_kind == pkg.SDIRK else 0)
        seen.setdefault(key, p)
    for p in seen.values():
        if time.perf_counter() - t0 > max_s:
            break
        pkg.Solver(p).close()
        tuned += 1
    return tuned, len(seen), time.perf_counter() - t0


def served_sequential(prms, u0s, chunk=64, nstreams=32):
    """GPU sequential stepping of the given requests (the served solves'
    baseline): chunks of `chunk` requests, each chunk's solves stepped at
    once over the batch's streams, chunks back to back.  Returns (DOF/s,
    seconds)."""
    import torch
    import paper_2209_06916_gb300 as pkg
    dof, secs = 0, 0.0
    for i in range(0, len(prms), chunk):
        ps = prms[i:i + chunk]
        us = [torch.tensor(u, dtype=torch.float64, device="cuda") for u in u0s[i:i + chunk]]
        outs = [torch.empty(p.nx, dtype=torch.float64, device="cuda") for p in ps]
        b = pkg.Batch(ps, nstreams=nstreams)
        b.sequential(us, outs)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.sequential(us, outs)
        torch.cuda.synchronize()
        secs += time.perf_counter() - t0
        dof += sum(p.nx * p.nt for p in ps)
        b.close()
    return (dof / secs if secs > 0 else None), secs


def alone_equals_in_mix(prms, u0s, res, u_outs, idx):
    """Each served request of idx that completed, solved again alone (same
    parameters, measured tuning off as inside the server, so both take the
    same launch geometry): are the C-points bitwise equal?"""
    import paper_2209_06916_gb300 as pkg
    old = os.environ.get("MGRIT_AUTOTUNE")
    os.environ["MGRIT_AUTOTUNE"] = "0"
    checked, equal = [], True
    try:
        for i in idx:
            if res[i]["status"] != 0:
                continue
            s = pkg.Solver(prms[i])
            want = np.zeros_like(u_outs[i])
            s.solve(u0s[i], want, allow_unconverged=True)
            s.close()
            same = bool(np.array_equal(want, u_outs[i]))
            equal = equal and same
            checked.append({"request": int(i), "nx": int(prms[i].nx), "nt": int(prms[i].nt), "equal": same})
    finally:
        if old is None:
            os.environ.pop("MGRIT_AUTOTUNE", None)
        else:
            os.environ["MGRIT_AUTOTUNE"] = old
    return {"all_equal": equal if checked else None, "checked": checked,
            "note": "bitwise, C-points of each request served in the mix against a standalone solve"}


def serving_record(duration, drain, inflight, rate=2000.0, budget_gb=80, tol=1e-11, seed=2000, pretune_s=0.0):
    """A Poisson stream of mixed solves (the batched mix plus 10% SDIRK5+U5
    at c in [2, 8]) through the native continuous-batching server with an
    HBM budget: arrival-to-completion latency p50/p99, service time and the
    completed DOF/s over the window (arrivals for `duration` s, the server
    stops `drain` s later).  With pretune_s > 0 the stream's shapes are tuned
    first (at most that many seconds, before the clock starts); the server
    itself never times launch candidates."""
    import paper_2209_06916_gb300 as pkg
    from workloads import ic_fourier, ic_sin4_noise, serving_stream
    arrivals, reqs = serving_stream(rate=rate, duration=duration, seed=seed)
    prms, u0s = [], []
    for d in reqs:
        kind = pkg.ERK if d["kind"] == "erk" else pkg.SDIRK
        prms.append(pkg.make_params(d["nx"], d["nt"], d["cfl"], d["p"], kind=kind, q=d["q"], m=d["m"], levels=0,
                                    nu=1, tol=tol, max_iter=60, precision=pkg.MIXED, seed=d["seed"]))
        u0s.append(ic_sin4_noise(d["nx"], seed=d["seed"]) if d["kind"] == "erk" else ic_fourier(d["nx"], d["seed"]))
    pre = pretune_shapes(prms, pretune_s) if pretune_s > 0 else (0, 0, 0.0)
    # alone == in mix: the C-points of a few small early requests come back
    # from the server and are compared with standalone solves below
    early = sorted(range(min(64, len(prms))), key=lambda i: prms[i].nx * prms[i].nt)[:4]
    u_outs = [None] * len(prms)
    for i in early:
        u_outs[i] = np.zeros((prms[i].nt // prms[i].m + 1, prms[i].nx))
    res, st = pkg.serve(prms, u0s, arrivals, budget_gb * 10 ** 9, max_inflight=inflight,
                        time_limit_s=duration + drain, u_outs=u_outs)
    alone = alone_equals_in_mix(prms, u0s, res, u_outs, early)
    ok = [r for r in res if r["status"] == 0]
    lat = np.array([r["latency_ms"] for r in ok])
    svc = np.array([(r["finish_s"] - r["start_s"]) * 1e3 for r in ok])
    statuses = {}
    for r in res:
        if r["status"] not in (0, 1):
            nm = pkg.ERRORS.get(r["status"], str(r["status"]))
            statuses[nm] = statuses.get(nm, 0) + 1
    offered = float(sum(d["nx"] * d["nt"] for d in reqs))
    # the completed requests stepped sequentially on the same GPU
    done = [i for i, r in enumerate(res) if r["status"] == 0]
    seq_rate, seq_s = served_sequential([prms[i] for i in done], [u0s[i] for i in done]) if done else (None, 0.0)
    served_rate = st["dof_completed"] / st["wall_s"]
    return {"workload": "advection1d_serving_poisson%d" % int(rate), "value": st["dof_completed"] / st["wall_s"],
            "unit": UNIT, "arrival_rate_per_s": rate, "arrivals_s": duration, "window_s": st["wall_s"],
            "requests": len(reqs), "offered_dof_per_s": offered / duration, "hbm_budget_gb": budget_gb,
            "max_inflight": inflight, "tol": tol,
            "serving": {k: st[k] for k in ("arrived", "admitted", "completed", "failed", "rejected", "backlog_end",
                                           "max_backlog", "max_mem_bytes", "max_inflight", "wall_s", "setup_s")},
            "pretune": {"shapes_tuned": pre[0], "shapes": pre[1], "seconds": pre[2],
                        "note": "measured geometries cached before the clock; none timed while serving"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)) if lat.size else None,
                           "p99": float(np.percentile(lat, 99)) if lat.size else None,
                           "completed": int(lat.size), "note": "arrival to completion"},
            "service_ms": {"p50": float(np.percentile(svc, 50)) if svc.size else None,
                           "p99": float(np.percentile(svc, 99)) if svc.size else None,
                           "note": "admission to completion"},
            "failures": statuses,
            "sequential": {"value": seq_rate, "unit": UNIT, "seconds": seq_s, "requests": len(done),
                           "note": "the completed requests by GPU sequential stepping, 64 at a time over 32 "
                                   "streams"},
            "served_over_sequential": (served_rate / seq_rate) if seq_rate else None,
            "alone_equals_in_mix": alone}


def run_serving(args):
    import torch
    torch.cuda.set_device(0)
    rec = serving_record(args.duration, args.drain, args.inflight, pretune_s=args.pretune)
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": rec["window_s"] * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 relax / f64 residual", "data": "synthetic", "config": {"workload": rec["workload"]},
            "serving_record": rec}
    print(json.dumps(line))
    return 0


def run_coarse_ops(args):
    """Coarse-grid operator comparison (Sec. 5.3 and Sec. 6.3.4 settings):
    two-level MGRIT at n_x x n_t = 2^10 x 2^12, stop at 1e-10 or 20
    iterations, random initial iterate, IC sin^4.  Per case: iterations,
    the measured final-iteration factor and the time per solve.
    Rediscretised vs corrected SL for SDIRK1+U1 and
    SDIRK3+U3 (FCF); F- vs FCF-relaxation with the corrected SL operator
    for ERK3+U3 at 0.85 c_max; the dispersive schemes of Sec. 6.4 (even p,
    corrected SL operator, FCF, at most 30 iterations as in Sec. 6.3); the
    approach to the CFL limit of ERK3+U3 and ERK5+U5 (Sec. 6.3.3)."""
    import torch
    import paper_2209_06916_gb300 as pkg
    from workloads import ic_sin4
    torch.cuda.set_device(0)
    nx, nt = 1 << 10, 1 << 12
    u0 = torch.tensor(ic_sin4(nx), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rows = []

    def case(kind, p, c, m, op, nu, max_iter=20):
        prm = pkg.make_params(nx, nt, c, p, kind=kind, m=m, levels=2, nu=nu, tol=1e-10, max_iter=max_iter, seed=0,
                              coarse_op=op)
        s = pkg.Solver(prm, stream=stream.cuda_stream)
        out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
        st = s.solve(u0, out, allow_unconverged=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            st = s.solve(u0, out, allow_unconverged=True)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / max(1, args.steps)
        s.close()
        kname = "erk" if kind == pkg.ERK else "sdirk"
        opname = {pkg.SL_CORRECTED: "sl_corrected", pkg.SL: "sl", pkg.REDISC: "redisc"}[op]
        rows.append({"scheme": "%s%d+U%d" % (kname.upper(), p, p), "c": round(c, 5), "m": m, "nu": nu,
                     "coarse_op": opname, "iterations": st["iterations"], "converged": st["converged"],
                     "factor": st["conv_factor"], "ms": ms})

    for p in (1, 3):
        for m in (2, 4, 8, 16):
            for c in (1.0, 4.0):
                for op in (pkg.REDISC, pkg.SL_CORRECTED):
                    case(pkg.SDIRK, p, c, m, op, 1)
    cmax = 1.62589  # ERK3 + U3 stability limit (Table 2)
    for m in (2, 4, 8, 16):
        for nu in (0, 1):
            case(pkg.ERK, 3, 0.85 * cmax, m, pkg.SL_CORRECTED, nu)
    # dispersive schemes (Sec. 6.4): ERK2+U2, ERK4+U4 over c / c_max (Table 2:
    # 1/2 and 1.04449), including both sides of the ERK4+U4 jump at 0.24 for
    # m = 2; SDIRK2+U2, SDIRK4+U4 over c
    for p, cm in ((2, 0.5), (4, 1.04449)):
        for m in (2, 4):
            for frac in (0.1, 0.23, 0.25, 0.5, 0.85):
                case(pkg.ERK, p, frac * cm, m, pkg.SL_CORRECTED, 1, max_iter=30)
    for p in (2, 4):
        for m in (2, 4):
            for c in (0.5, 1.0, 2.0):
                case(pkg.SDIRK, p, c, m, pkg.SL_CORRECTED, 1, max_iter=30)
    # convergence near the CFL limit (Sec. 6.3.3): ERK3+U3 and ERK5+U5, m = 4,
    # over c / c_max (ERK5: c_max = 1.9399 of the stability polynomial that
    # Table 1's error constant fixes)
    for p, cm, fracs in ((3, 1.62589, (0.5, 0.7, 0.85, 0.95, 0.99)), (5, 1.9399, (0.3, 0.5, 0.6, 0.7, 0.8))):
        for frac in fracs:
            case(pkg.ERK, p, frac * cm, 4, pkg.SL_CORRECTED, 1, max_iter=30)
    line = {"metric": "two-level MGRIT convergence factor, measured vs LFA", "unit": "factor", "n_gpus": 1,
            "steps": args.steps, "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "advection1d_coarse_operator_comparison", "nx": nx, "nt": nt, "levels": 2,
                       "tol": 1e-10, "max_iter": "20 (Sec. 5.3 cases), 30 (even p)"}, "cases": rows}
    print(json.dumps(line))
    return 0


def run_table3(args):
    """Table 3 (Sec. 6.3.1): two-level and V-cycle iteration counts of the
    paper's setup (ERK3+U3 at 0.85 c_max, SDIRK3+U3 at c = 5, FCF, stop at
    a 1e-10 residual reduction, random initial iterate, IC sin^4), beside
    the printed counts (tests/golden/table3_iterations.txt); the ERK V-cycles
    also with GMRES correction solves, as the paper ran them."""
    import torch
    import paper_2209_06916_gb300 as pkg
    from workloads import ic_sin4
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "table3_iterations.txt")) as f:
        table = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    t0 = time.perf_counter()
    for kname, nx, nt, m, two, vc in table:
        nx, nt, m = int(nx), int(nt), int(m)
        kind = pkg.ERK if kname == "erk" else pkg.SDIRK
        c = 0.85 * 1.62589 if kind == pkg.ERK else 5.0   # Table 2: c_max of ERK3+U3

        def its(levels, cs=pkg.DIRECT):
            prm = pkg.make_params(nx, nt, c, 3, kind=kind, m=m, levels=levels, nu=1, tol=1e-10, max_iter=40,
                                  seed=0, coarse_solve=cs)
            s = pkg.Solver(prm, stream=stream.cuda_stream)
            u0 = torch.tensor(ic_sin4(nx), dtype=torch.float64, device="cuda")
            out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
            st = s.solve(u0, out, allow_unconverged=True)
            s.close()
            return st["iterations"] if st["converged"] else None

        row = {"scheme": kname.upper() + "3+U3", "nx": nx, "nt": nt, "m": m,
               "two_level": its(2), "paper_two_level": int(two), "vcycle": its(0), "paper_vcycle": int(vc)}
        if kind == pkg.ERK:
            row["vcycle_gmres"] = its(0, pkg.GMRES)
        rows.append(row)
    line = {"metric": "MGRIT iterations to a 1e-10 residual reduction (Table 3)", "unit": "iterations",
            "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "advection1d_table3_iterations", "seconds": time.perf_counter() - t0},
            "rows": rows}
    print(json.dumps(line))
    return 0


def run_parallel_problems(args):
    """The problems of the paper's parallel results (Sec. 6.3.2): n_x x n_t =
    2^12 x 2^14, V-cycles with m = 16 on the first level and 4 below
    (coarsening until fewer than two time points), stop at a 1e-10 residual
    reduction; ERK1+U1 and ERK3+U3 at 0.85 c_max, SDIRK1+U1 at c = 1,
    SDIRK3+U3 at c = 5.  Per problem: FP64 MGRIT (exact correction solves;
    ERK also with GMRES ones, the paper's choice), MIXED, and GPU sequential
    stepping of the same problem, each the mean of the timed solves."""
    import torch
    import paper_2209_06916_gb300 as pkg
    from workloads import ic_sin4_noise
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    nx, nt = 1 << 12, 1 << 14
    u0 = torch.tensor(ic_sin4_noise(nx, seed=0), dtype=torch.float64, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    rows = []
    problems = [("ERK1+U1", pkg.ERK, 1, 0.85 * 1.0), ("ERK3+U3", pkg.ERK, 3, 0.85 * 1.62589),
                ("SDIRK1+U1", pkg.SDIRK, 1, 1.0), ("SDIRK3+U3", pkg.SDIRK, 3, 5.0)]
    for name, kind, p, c in problems:
        row = {"scheme": name, "c": round(c, 5)}
        variants = [("fp64", pkg.FP64, pkg.DIRECT), ("mixed", pkg.MIXED, pkg.DIRECT)]
        if kind == pkg.ERK:
            variants.append(("fp64_gmres", pkg.FP64, pkg.GMRES))
        seq_ms = None
        for vname, prec, cs in variants:
            prm = pkg.make_params(nx, nt, c, p, kind=kind, m=16, m_coarse=4, levels=0, nu=1, tol=1e-10,
                                  max_iter=30, seed=0, precision=prec, coarse_solve=cs)
            s = pkg.Solver(prm, stream=stream.cuda_stream)
            out = torch.empty((nt // 16 + 1, nx), dtype=torch.float64, device="cuda")
            st = s.solve(u0, out, allow_unconverged=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                st = s.solve(u0, out, allow_unconverged=True)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            if seq_ms is None:
                seq = torch.empty(nx, dtype=torch.float64, device="cuda")
                s.fine_propagate(u0, seq, nt)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(args.steps):
                    s.fine_propagate(u0, seq, nt)
                e1.record(stream)
                torch.cuda.synchronize()
                seq_ms = e0.elapsed_time(e1) / args.steps
                row["levels"] = st["levels"]
                row["sequential_ms"] = seq_ms
            err = float((out[-1] - seq).abs().max().item() / seq.abs().max().item())
            row[vname] = {"ms": ms, "iterations": st["iterations"], "converged": st["converged"],
                          "max_rel_err_vs_sequential": err, "over_sequential": seq_ms / ms}
            s.close()
        rows.append(row)
    line = {"metric": "space-time DOF/s to 1e-10 residual vs GPU seq. stepping; p50/p99 latency", "unit": "DOF/s",
            "n_gpus": 1, "steps": args.steps, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "advection1d_parallel_problems_4096x16384_m16_4", "nx": nx, "nt": nt,
                       "m": 16, "m_coarse": 4, "levels": "until fewer than two time points"},
            "rows": rows}
    print(json.dumps(line))
    return 0


def run_reference(args):
    """The oracle timed as it stands on the host cores (the one place this
    repository has no reference implementation to install: the paper has
    no code).  Each step is one round of independent bounded samples of the
    workload, one per core.  Under torchrun only rank 0 runs it."""
    ws, rank = _dist()
    if rank != 0:
        return 0
    w = WORKLOAD
    sample_nt = args.reference_nt or (128 if w["kind"] == "sdirk" else 512)
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    levels = _sample_levels(w, sample_nt)
    jobs = [(w, sample_nt, levels, w["seed"] + i) for i in range(cores)]
    times, its = [], []
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_import, range(cores))
        for i in range(args.warmup + args.steps):
            t = time.perf_counter()
            res = pool.map(_oracle_sample, jobs)
            dt = time.perf_counter() - t
            if i >= args.warmup:
                times.append(dt)
                its += [r[2] for r in res]
    dof = cores * w["nx"] * sample_nt
    value = dof * len(times) / sum(times)
    sample = ("%d independent solves per step (one per core, spawn pool), each nx=%d, nt=%d (the first %d of %d "
              "steps), same scheme/m/tol, %d levels, %d-%d iterations"
              % (cores, w["nx"], sample_nt, sample_nt, w["nt"], levels, min(its), max(its)))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "nx": w["nx"], "nt": sample_nt,
                       "note": "CPU oracle (numpy FP64 MGRIT) on %d-step samples of the %d-step workload"
                               % (sample_nt, w["nt"])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_sharded(args):
    """One solve of the workload time-sharded over the torchrun ranks (one
    GPU each, NCCL): the level-0 CF-intervals in contiguous blocks per rank,
    one boundary row per C-relaxation, the residual norm all-reduced, the
    coarse levels on rank 0.  Strong scaling: the whole job is one solve."""
    import torch
    import torch.distributed as dist
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl" if ws > 1 else "gloo")
    import paper_2209_06916_gb300 as pkg
    from paper_2209_06916_gb300.sharded import ShardedSolver
    w = dict(WORKLOAD)
    if args.nt > 0:
        w["nt"] = args.nt
        while w["levels"] > 2 and args.nt % (w["m"] ** (w["levels"] - 1)):
            w["levels"] -= 1
    kind = pkg.ERK if w["kind"] == "erk" else pkg.SDIRK
    prm = pkg.make_params(w["nx"], w["nt"], w["cfl"], w["p"], kind=kind, q=w["q"], m=w["m"], levels=w["levels"],
                          nu=w["nu"], tol=w["tol"], max_iter=w["max_iter"], seed=w["seed"], precision=pkg.FP64)
    s = ShardedSolver(prm, comm_device="cuda" if ws > 1 else "cpu")
    u0 = make_ic(w)
    for _ in range(args.warmup):
        s.solve(u0)
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    its = []
    for _ in range(args.steps):
        out, st = s.solve(u0)
        its.append(st["iterations"])
    torch.cuda.synchronize()
    dist.barrier()
    ms = (time.perf_counter() - t0) * 1e3
    ms = max_over_ranks(ms, dist, "cuda" if ws > 1 else "cpu")
    dof = w["nx"] * w["nt"]
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": dof * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": ws,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                          "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic",
                          "config": {"workload": w["name"] + "_time_sharded", "nx": w["nx"], "nt": w["nt"],
                                     "parallelism": "time-sharded x%d (level-0 CF-interval blocks per rank, "
                                                    "coarse levels on rank 0)" % ws, "iterations": its,
                                     "timing": "host clock around the solves, max over ranks"}}))
    s.close()
    dist.destroy_process_group()
    return 0


def _max_rel_err(out, ref_rows, u0):
    """max |out - ref| / max |ref| over every C-point row (device tensors;
    row 0 of `out` against u0, rows 1.. against the sequential trajectory)."""
    e = max(float((out[0] - u0).abs().max().item()), float((out[1:] - ref_rows).abs().max().item()))
    scale = max(float(u0.abs().max().item()), float(ref_rows.abs().max().item()))
    return e / scale


def run_single(args):
    import torch
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import paper_2209_06916_gb300 as pkg

    w = dict(WORKLOAD)
    if args.nt > 0:
        w["nt"] = args.nt
        w["name"] += "_nt%d" % args.nt
        while w["levels"] > 2 and args.nt % (w["m"] ** (w["levels"] - 1)):
            w["levels"] -= 1
    if args.precision:
        w["precision"] = args.precision
    if args.tol > 0:
        w["tol"] = args.tol
    nx, nt, m = w["nx"], w["nt"], w["m"]
    stream = torch.cuda.current_stream()
    kind = pkg.ERK if w["kind"] == "erk" else pkg.SDIRK
    prec = {"fp64": pkg.FP64, "mixed": pkg.MIXED, "mixed_fast": pkg.MIXED_FAST}[w["precision"]]

    def make(precision, coarse_solve=pkg.DIRECT):
        prm = pkg.make_params(nx, nt, w["cfl"], w["p"], kind=kind, q=w["q"], m=m, levels=w["levels"], nu=w["nu"],
                              tol=w["tol"], max_iter=w["max_iter"], seed=w["seed"], precision=precision,
                              coarse_solve=coarse_solve)
        if args.inner > 0:
            prm.inner_cycles = args.inner
        return pkg.Solver(prm, stream=stream.cuda_stream)

    main_solve = pkg.GMRES if args.coarse_solve == "gmres" else pkg.DIRECT
    if main_solve == pkg.GMRES:
        w["name"] += "_gmres"
    t0 = time.perf_counter()
    s = make(prec, main_solve)
    setup_s = time.perf_counter() - t0
    u0_h = make_ic(w)
    u0 = torch.tensor(u0_h, dtype=torch.float64, device="cuda")
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")

    for _ in range(args.warmup):
        st = s.solve(u0, out)
    torch.cuda.synchronize()

    # raw nvidia-smi samples of the timed region (BENCH_CLOCKS_DIR, else the
    # system's temporary directory); the JSON line carries their summary
    import tempfile
    clk_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
    clk_path = os.path.join(clk_dir, "bench_clocks_rank%d.csv" % rank)
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    cp, cf = clocks_sampler_start(clk_path)
    time.sleep(0.5)

    # the timed region: K solves, with the library's per-launch CUDA events on
    # the handle's stream (the roofline's kernel times come from these same
    # launches)
    s.profile(True)
    launches0 = s.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = []
    for _ in range(args.steps):
        st = s.solve(u0, out)
        iters.append(st["iterations"])
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = s.launch_count() - launches0
    prof = s.profile_read()
    s.profile(False)
    ms = max_over_ranks(ms, dist, "cuda")

    # end to end through the C ABI with host buffers (pinned), copies inside
    e2e_steps = min(args.steps, args.e2e_steps)
    u0_pin = torch.tensor(u0_h, dtype=torch.float64).pin_memory()
    out_pin = torch.empty((nt // m + 1, nx), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.solve(u0_pin, out_pin)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3
    e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")

    # GPU sequential time-stepping of the same problem (the baseline), with
    # every C-point row kept: the error of the MGRIT solution over all
    # C-points against it
    seq_ms, err, sprof = None, None, {"sequential": (0, 0.0, 0.0)}
    seq_rows = None
    if not args.no_sequential:
        seq_out = torch.empty(nx, dtype=torch.float64, device="cuda")
        seq_rows = torch.empty((nt // m, nx), dtype=torch.float64, device="cuda")
        s.fine_propagate(u0, seq_out, nt, m, seq_rows)
        s.profile(True)
        torch.cuda.synchronize()
        seq_steps = min(args.steps, args.seq_steps)
        e0.record(stream)
        for _ in range(seq_steps):
            s.fine_propagate(u0, seq_out, nt)
        e1.record(stream)
        torch.cuda.synchronize()
        seq_ms = e0.elapsed_time(e1) / seq_steps
        sprof = s.profile_read()
        s.profile(False)
        s.solve(u0, out)
        torch.cuda.synchronize()
        err = _max_rel_err(out, seq_rows, u0)
    dof = nx * nt
    variants = {}
    # the same workload with other choices of the method:
    #   "mixed" / "mixed_fast"  FP32 relaxation inside FP64 refinement ("mixed"
    #                           keeps every correction solve in FP64,
    #                           "mixed_fast" runs the well-conditioned ones,
    #                           kappa <= 1e3, in FP32)
    #   "gmres"                 the coarse correction systems solved by GMRES
    #                           (rel. 1e-2, at most 20 iterations, Sec. 6.3)
    #                           instead of the exact banded solve (explicit
    #                           workloads: on the implicit one capped GMRES
    #                           stalls MGRIT near a 1e-3 residual)
    vlist = []
    if not args.no_variants:
        if prec == pkg.FP64:
            vlist += [("mixed", pkg.MIXED, pkg.DIRECT), ("mixed_fast", pkg.MIXED_FAST, pkg.DIRECT)]
        if main_solve == pkg.DIRECT and kind == pkg.ERK:
            vlist.append(("gmres", prec, pkg.GMRES))
    vsteps = max(1, min(args.steps, args.variant_steps))
    for vname, vprec, vsolve in vlist:
        sm = make(vprec, vsolve)
        outm = torch.empty_like(out)
        stm = sm.solve(u0, outm, allow_unconverged=True)
        torch.cuda.synchronize()
        g0 = [sm.gmres_stats(l) for l in range(1, w["levels"])]
        sm.profile(True)
        e0.record(stream)
        for _ in range(vsteps):
            stm = sm.solve(u0, outm, allow_unconverged=True)
        e1.record(stream)
        torch.cuda.synchronize()
        vprof = sm.profile_read()
        sm.profile(False)
        mms = e0.elapsed_time(e1) / vsteps
        errm = _max_rel_err(outm, seq_rows, u0) if seq_rows is not None else None
        v = {"value": dof / (mms / 1e3), "unit": UNIT, "ms": mms, "converged": stm["converged"],
             "rel_residual": stm["rnorm"] / stm["rnorm0"] if stm["rnorm0"] > 0 else 0.0,
             "iterations": stm["iterations"],
             "outer_iterations": stm["outer_iterations"], "inner_cycles": stm["inner_cycles"],
             "max_rel_err_vs_sequential": errm, "err_over": "all C-points",
             "over_sequential": seq_ms / mms if seq_ms is not None else None,
             "over_fp64": (ms / args.steps) / mms, "solves_timed": vsteps,
             "kernel_ms": {k: vv[1] / vsteps for k, vv in vprof.items()}}
        n32, ms32, fl32 = vprof.get("level0_fp32", (0, 0.0, 0.0))
        if ms32 > 0:
            v["fp32_level0_kernel"] = {"launches": n32, "ms_per_launch": ms32 / max(1, n32),
                                       "achieved_tflops": fl32 / (ms32 / 1e3) / 1e12,
                                       "frac_of_derived_fp32_peak": fl32 / (ms32 / 1e3) / FP32_PEAK_FLOPS}
        if vsolve == pkg.GMRES:
            g1 = [sm.gmres_stats(l) for l in range(1, w["levels"])]
            v["gmres_iterations_per_solve"] = [
                (b[0] - a[0]) / max(1, b[1] - a[1]) for a, b in zip(g0, g1)]
        variants[vname] = v
        sm.close()
    clocks = clocks_sampler_stop(cp, cf, clk_path, local)
    scnt, sms, sfl = sprof["sequential"]
    del seq_rows

    value = whole_job_value(dof, args.steps, ms, ws)
    cnt, kms, kfl = prof["stencil0"]
    achieved = kfl / (kms / 1e3) if kms > 0 else 0.0
    info0 = s.level_info(0)
    if w["kind"] == "erk":
        kname = "%s<double,%d> (level-0 composite Phi^m)" % (
            "stencil_rows_persistent" if info0[4] else "stencil_rows_kernel", int(info0[6]))
    elif info0[4] == 2:
        kname = ("sdirk_seg_kernel<%d,%d,128> (level-0 SDIRK stages in FP64: one CTA per interval, 128-point "
                 "segments per thread, warm-up recurrences, stage right-hand sides from the solves)"
                 % ((w["p"] + 1) // 2, (w["p"] - 1) // 2))
    else:
        kname = ("sdirk_kernel<double,%d,%d> (level-0 SDIRK stages: banded solves, stage derivatives from the "
                 "solves), clusters of %d" % (int(info0[6]), w["p"] + 1, int(info0[7])))
    roof = {"bound": "alu", "kernel": kname,
            "achieved": achieved / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_FLOPS, "traffic": None,
            "traffic_note": "DRAM bytes come from ncu captures, not from this run; the kernel is FP64-pipe bound "
                            "(DRAM below 2% of peak)",
            "peak_source": "derived FP64 FMA pipe: 152 SMs x 4 flop/clk x 2.07 GHz",
            "launches": cnt, "ms_per_launch": kms / max(1, cnt),
            "share_of_step": kms / ms if ms > 0 else None,
            "timing": "per-launch CUDA events on the handle's stream inside the timed region"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == pkg.FP64 else "f32 relax / f64 residual", "data": "synthetic",
            "config": {"workload": w["name"], "nx": nx, "nt": nt,
                       "scheme": "%s%d+U%d" % (w["kind"].upper(), w["q"], w["p"]), "cfl": w["cfl"],
                       "m": m, "levels": w["levels"], "relax": "FCF", "tol": w["tol"],
                       "tol_note": "stop at 1e-11: every C-point within 1e-10 of sequential stepping "
                                   "(a 1e-10 residual leaves ~1.7e-10 on the 16384 x 65536 workload)",
                       "precision": w["precision"], "coarse_solve": args.coarse_solve,
                       "iterations": iters, "parallelism": "replicas" if ws > 1 else "single",
                       "setup_s": setup_s,
                       "l2": "working set %.0f MB > 129 MB L2 (no flush)" % (
                           (2 * (nt // m + 1) + (nt // m + 1) + 2 * (nt // m ** 2 + 1)) * nx * 8 / 1e6)},
            "roofline": roof,
            "e2e": {"value": whole_job_value(dof, e2e_steps, e2e_ms, ws), "unit": UNIT,
                    "h2d_bytes_per_step": nx * 8, "d2h_bytes_per_step": (nt // m + 1) * nx * 8,
                    "steps": e2e_steps},
            "gpu_launches": launches, "clocks": clocks,
            "sequential": None if seq_ms is None else {
                "value": dof / (seq_ms / 1e3), "unit": UNIT, "ms": seq_ms,
                "kernel": ("seq_kernel (thread-block cluster, DSMEM halos, composite Phi^B)" if w["kind"] == "erk"
                           else "sdirk_kernel<double> on one cluster (K = 1)"),
                "achieved_tflops": sfl / (sms / 1e3) / 1e12 if sms > 0 else None,
                "frac": (sfl / (sms / 1e3)) / FP64_PEAK_FLOPS if sms > 0 else None},
            "mgrit_over_sequential": seq_ms / (ms / args.steps) if seq_ms is not None else None,
            "max_rel_err_vs_sequential": err, "err_over": "all C-points",
            "variants": variants,
            "kernel_ms": {k: v[1] / args.steps for k, v in prof.items()}}
    s.close()
    del out
    torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not args.no_c4:
        line["batched"] = batched_record(args.count, 1, 1)
    if rank == 0 and ws == 1 and not args.no_c5:
        line["served"] = serving_record(args.c5_duration, args.c5_drain, args.inflight)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, sample_nt=args.cpu_nt or (256 if w["kind"] == "sdirk" else 2048))
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS) + ["c4", "c4_sdirk", "c5", "coarse_ops", "table3",
                                                                      "parallel_problems"])
    ap.add_argument("--count", type=int, default=512, help="c4: number of solves")
    ap.add_argument("--duration", type=float, default=60.0, help="c5: seconds of arrivals")
    ap.add_argument("--drain", type=float, default=30.0, help="c5: extra seconds before the server stops")
    ap.add_argument("--inflight", type=int, default=64, help="c5: concurrent solves")
    ap.add_argument("--pretune", type=float, default=0.0, help="c5: seconds of shape tuning before the clock")
    ap.add_argument("--no-c4", action="store_true", help="skip the batched sub-record")
    ap.add_argument("--no-c5", action="store_true", help="skip the served sub-record")
    ap.add_argument("--c5-duration", type=float, default=3.0, help="served sub-record: seconds of arrivals")
    ap.add_argument("--c5-drain", type=float, default=12.0, help="served sub-record: seconds after the arrivals")
    ap.add_argument("--no-variants", action="store_true", help="skip the mixed-precision sub-measurement")
    ap.add_argument("--variant-steps", type=int, default=3, help="timed solves per variant")
    ap.add_argument("--e2e-steps", type=int, default=5, help="solves of the end-to-end measurement")
    ap.add_argument("--seq-steps", type=int, default=2, help="timed runs of sequential stepping")
    ap.add_argument("--nt", type=int, default=0, help="override n_t of c1-c3 (small profiling cases)")
    ap.add_argument("--tol", type=float, default=0.0, help="override the stop tolerance")
    ap.add_argument("--cpu-nt", type=int, default=0, help="time steps of the CPU baseline's sample")
    ap.add_argument("--reference-nt", type=int, default=0, help="time steps of the reference arm's sample")
    ap.add_argument("--no-sequential", action="store_true", help="skip the sequential-stepping baseline")
    ap.add_argument("--sharded", action="store_true",
                    help="under torchrun: one time-sharded solve over the ranks (default: independent replicas)")
    ap.add_argument("--precision", default="", choices=["", "fp64", "mixed", "mixed_fast"],
                    help="override the workload's")
    ap.add_argument("--inner", type=int, default=0, help="MIXED: FP32 V-cycles per FP64 residual (0: library default)")
    ap.add_argument("--coarse-solve", default="direct", choices=["direct", "gmres"],
                    help="correction solves of the coarse operator (gmres: Sec. 6.3's GMRES)")
    args = ap.parse_args()
    global WORKLOAD
    if args.workload in ("c4", "c4_sdirk") and args.impl == "ours":
        return run_batched(args, implicit=args.workload == "c4_sdirk")
    if args.workload == "c5" and args.impl == "ours":
        return run_serving(args)
    if args.workload == "coarse_ops" and args.impl == "ours":
        return run_coarse_ops(args)
    if args.workload == "table3" and args.impl == "ours":
        return run_table3(args)
    if args.workload == "parallel_problems" and args.impl == "ours":
        return run_parallel_problems(args)
    WORKLOAD = WORKLOADS.get(args.workload, WORKLOADS["c3"])
    if args.impl == "reference":
        return run_reference(args)
    if args.sharded:
        return run_sharded(args)
    return run_single(args)


if __name__ == "__main__":
    sys.exit(main())
