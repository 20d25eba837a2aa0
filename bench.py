"""Benchmark of the moving-boundary cut-cell sweep on GB300.

Workload (default): 64 independent Euler instances on uneven grids drawn
uniformly from 128^2 to 1024^2 (seeded), bodies mixed from cylinder,
equilateral triangle and piston-in-tube, seeded shock Mach numbers in
[1.2, 3.0]; FP32 bulk arithmetic with FP64 geometry and stabilisation
weights; each instance at its own CFL time step computed on the device; one
CUDA-graph replay per time step.  A "step" is one time step of every
instance = two directional sweeps, each running all five stages of the
sweep (geometry, standard fluxes, stabilised and wall fluxes, conservative
update with covering/uncovering, CFL reduction).

Metric: cell-updates per second per sweep (grid cells of all instances times
sweeps, divided by the device time).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mb|reference]

Multi-GPU (torchrun, one rank per GPU): every rank advances its own seeded
batch of independent instances (weak scaling, no collective on the data
path); value = cells updated by all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per sweep (FP32 batched vs plain FP64, same GB300, stated L1 err); p50/p99"
UNIT = "cell-updates/s"
BYTES_PER_CELL_FP32 = 32.0   # 4 conserved values read + 4 written per cell-sweep
BYTES_PER_CELL_FP64 = 64.0


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def sample_clocks(stop, out):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    while not stop.is_set():
        try:
            r = subprocess.run(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits"],
                               capture_output=True, text=True, timeout=5)
            for line in r.stdout.strip().splitlines():
                out.append([x.strip() for x in line.split(",")])
        except Exception:
            pass
        stop.wait(0.2)


def summarize_clocks(samples, gpu_index):
    rows = [s for s in samples if s and s[0] == str(gpu_index)] or samples
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = set()
    for r in rows:
        for k, n in enumerate(names):
            if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                reasons.add(n)
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(rows)}


def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo)."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5)
        for line in r.stdout.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def combine_ranks(total_ms, cells, device):
    """Whole-job figures over all ranks: the slowest rank's timed region (max)
    and the cells all ranks updated per sweep (sum).  Works with any
    torch.distributed backend; single-process runs pass through."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), float(cells)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(cells)], dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t.item()), float(c.item())


def job_value(cells_all, steps, total_ms):
    """Cell-updates per second: every cell of every rank is updated twice per
    step (one x and one y sweep)."""
    return cells_all * 2 * steps / (total_ms * 1e-3)


def bulk_traffic(precision, wname):
    """DRAM bytes of the bulk update per sweep (mean over the x and y sweeps;
    each the concurrent pass plus the deferred-pair kernel) from the ncu
    capture summarised in profiles/bulk_traffic.json, or None when that
    capture is of another workload or precision or the kernel sources have
    changed since it was taken."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "bulk_traffic.json")
    try:
        d = json.load(open(prof))
        if d["workload"] != wname or d["precision"] != precision:
            return None
        for f, sha in d["sources_sha256"].items():
            with open(os.path.join(ROOT, "paper_1711_11361_gb300", "csrc", f), "rb") as fh:
                if hashlib.sha256(fh.read()).hexdigest() != sha:
                    return None
        v = list(d["per_sweep_bytes"].values())
        return float(sum(v) / len(v))
    except (OSError, KeyError, ValueError):
        return None


# FP32 lane operations per clock: 152 SMs x 128 FP32 lanes x 2.07 GHz
FP32_LANE_OPS_PEAK = 152 * 128 * 2.07e9


def bulk_alu(precision, wname):
    """FP32 lane operations per cell-sweep of the bulk update (mean over the
    x and y sweeps) from the ncu instruction counts summarised in
    profiles/bulk_alu.json, or None under the same conditions as
    bulk_traffic."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "bulk_alu.json")
    try:
        d = json.load(open(prof))
        if d["workload"] != wname or d["precision"] != precision:
            return None
        for f, sha in d["sources_sha256"].items():
            with open(os.path.join(ROOT, "paper_1711_11361_gb300", "csrc", f), "rb") as fh:
                if hashlib.sha256(fh.read()).hexdigest() != sha:
                    return None
        v = list(d["fp32_lane_ops_per_cell"].values())
        return float(sum(v) / len(v))
    except (OSError, KeyError, ValueError):
        return None


def fp64_pipe_per_cell(wname):
    """FP64-pipe lane operations per cell-sweep of the FP64 bulk kernels
    (every FP64 instruction -- add, multiply, FMA, compare, min/max,
    conversion -- holds the pipe alike), mean over the x and y sweeps, from
    the ncu capture summarised in profiles/fp64_ops.json; None when the
    kernel sources have changed since."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "fp64_ops.json")
    try:
        d = json.load(open(prof))
        for f, sha in d["sources_sha256"].items():
            with open(os.path.join(ROOT, "paper_1711_11361_gb300", "csrc", f), "rb") as fh:
                if hashlib.sha256(fh.read()).hexdigest() != sha:
                    return None
        v = list(d["fp64_pipe_lane_ops_per_cell"].values())
        return float(sum(v) / len(v))
    except (OSError, KeyError, ValueError):
        return None


def fp64_roofline_leg(mb, probs, wname, stream):
    """The plain FP64 path on the same batch: its bulk kernels' time per sweep
    (CUDA events around the bulk passes of 4 steps), cell-updates/s, and the
    FP64-pipe roofline against the GPU's measured FP64 FMA rate."""
    import torch
    sim = mb.Sim(probs, mb.FP64)
    sim.set_stream(stream.cuda_stream)
    sim.run(2, 0.0)
    sim.sync()
    sim.enable_timing(True)
    sim.run(4, 0.0)
    ms, n = sim.kernel_time()
    sim.enable_timing(False)
    sim.close()
    rate = mb.fp64_rate(stream.cuda_stream)
    cells = sum(p.nx * p.ny for p in probs)
    bulk_s = ms * 1e-3 / max(n, 1)
    out = {"bulk_ms_per_sweep": bulk_s * 1e3, "bulk_cell_updates_per_s": cells / bulk_s, "unit": UNIT,
           "peak_fp64_fma_per_s": rate, "peak_kind": "measured: mb_fp64_rate (independent FP64 FMA chains)"}
    ops = fp64_pipe_per_cell(wname)
    if ops is not None:
        achieved = ops * cells / bulk_s
        out["roofline"] = {"bound": "fp64", "achieved": achieved / 1e12, "peak": rate / 1e12,
                           "unit": "T FP64-pipe lane-ops/s", "frac": achieved / rate,
                           "fp64_pipe_lane_ops_per_cell": ops}
    return out


def accuracy_leg(mb, probs, steps=20):
    """FP32 batch against the FP64 GPU path (itself held to the oracle at
    1e-12 per step by the parity tests) on the same instances, the same
    initial states and a common fixed dt (the smallest CFL step of the
    instances): the relative L1 density error, alpha-weighted over fluid
    cells, and the drift of the conserved totals (rho, rho u, rho v, E)
    relative to the exactly conservative FP64 path, as maxima over
    instances."""
    s64 = mb.Sim(probs, mb.FP64)
    dts = s64.step(0.0, report=True)
    s64.close()
    dt = float(np.min(dts))
    s64 = mb.Sim(probs, mb.FP64)
    s32 = mb.Sim(probs, mb.FP32)
    for _ in range(steps):
        s64.step(dt)
        s32.step(dt)
    s64.sync()
    s32.sync()
    l1, drift = [], np.zeros(4)
    for k in range(len(probs)):
        a = s64.read_state(k, alpha=True)
        b = s32.read_state(k)
        al = a["alpha"]
        fl = al > 0
        r64, r32 = a["Q"][0][fl], b["Q"][0][fl]
        w = al[fl]
        l1.append(float(np.sum(w * np.abs(r32 - r64)) / np.sum(w * np.abs(r64))))
        # momentum components against the momentum magnitude (one of them
        # vanishes by symmetry in most instances)
        mom = np.sum(w * np.hypot(a["Q"][1][fl], a["Q"][2][fl]))
        for q in range(4):
            t64 = np.sum(w * a["Q"][q][fl])
            t32 = np.sum(w * b["Q"][q][fl])
            scale = mom if q in (1, 2) else np.sum(w * np.abs(a["Q"][q][fl]))
            drift[q] = max(drift[q], abs(t32 - t64) / scale if scale > 0 else 0.0)
    m32 = [s32.merge_count(k) for k in range(len(probs))]
    m64 = [s64.merge_count(k) for k in range(len(probs))]
    s64.close()
    s32.close()
    return {"l1_density_rel_max": max(l1), "l1_density_rel_mean": float(np.mean(l1)),
            "conservation_drift_rel_max": {"rho": drift[0], "rho_u": drift[1], "rho_v": drift[2], "E": drift[3]},
            "against": "FP64 GPU path, same instances and states", "steps": steps, "dt": dt,
            "safeguard_merged_cells": {
                "fp32": {"total": int(sum(m32)), "instances_merging": int(sum(1 for m in m32 if m)),
                         "max_instance": int(max(m32)), "per_step_mean": float(sum(m32)) / steps},
                "fp64": {"total": int(sum(m64)), "instances_merging": int(sum(1 for m in m64 if m)),
                         "max_instance": int(max(m64)), "per_step_mean": float(sum(m64)) / steps},
                "cells_per_step": len(probs) and sum(p.nx * p.ny for p in probs) * 2}}


def fp64_single_leg(mb, probs, steps=6):
    """The plain FP64 path one instance at a time (largest, median and
    smallest grid of the workload): cell-updates/s, for the speedup of the
    FP32 batched form."""
    import torch
    pick = sorted(probs, key=lambda q: q.nx * q.ny)
    pick = [pick[-1], pick[len(pick) // 2], pick[0]]
    cells, ms = 0, 0.0
    for p in pick:
        sim = mb.Sim([p], mb.FP64)
        st = torch.cuda.Stream()
        sim.set_stream(st.cuda_stream)
        sim.run(2, 0.0)
        sim.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        sim.run(steps, 0.0)
        e1.record(st)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        cells += p.nx * p.ny * 2 * steps
        sim.close()
    return {"value": cells / (ms * 1e-3), "unit": UNIT,
            "sample": "%d steps each of %s, one instance per sim, FP64 throughout" % (steps, ", ".join(p.name for p in pick))}


def run_served(args):
    """Served stream (continuous batching through mb_server_*): the seeded
    request stream (count, grid sizes and step counts set by the --c5-*
    options; the defaults are the full stream: 2000 requests, N log-uniform
    in 256..2048, 500..5000 steps), Poisson arrivals at an offered load of
    --c5-load times the batched throughput measured on the stream's own
    first 16 requests.  Requests are built when they arrive and their final
    states are not kept (host memory).  Reports aggregate cell-updates/s over
    the run, p50/p99 completion latency (submission to result on the host),
    and the serial plain-FP64 time of the same stream extrapolated from a
    seeded subsample (each sampled request timed over a few steps, scaled by
    its step count)."""
    import torch
    from paper_1711_11361_gb300 import inputs, mb
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    specs = inputs.c5_requests(n=args.c5_requests, nmin=args.c5_nmin, nmax=args.c5_nmax, smin=args.c5_smin,
                               smax=args.c5_smax)
    n = len(specs)
    work = np.array([sp["N"] ** 2 * 2.0 * sp["steps"] for sp in specs])
    # batched throughput of the stream's own instances sets the offered rate
    probe = [inputs.make_request(sp) for sp in specs[:16]]
    sim = mb.Sim(probe, mb.FP32)
    st = torch.cuda.Stream()
    sim.set_stream(st.cuda_stream)
    sim.run(3, 0.0)
    sim.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    sim.run(5, 0.0)
    e1.record(st)
    torch.cuda.synchronize()
    thr = sum(p.nx * p.ny for p in probe) * 2 * 5 / (e0.elapsed_time(e1) * 1e-3)
    sim.close()
    del probe
    mean_gap = float(np.mean(work)) / (args.c5_load * thr)
    arr = inputs.c5_arrivals(n, mean_gap)
    srv = mb.Server(mb.FP32, 0, budget_bytes=args.c5_budget_gib * 2 ** 30, max_active=args.c5_max_active)
    stop = threading.Event()
    samples = []
    th = threading.Thread(target=sample_clocks, args=(stop, samples), daemon=True)
    th.start()
    ids, k = [], 0
    t0 = time.perf_counter()
    peak = 0
    while True:
        now = time.perf_counter() - t0
        while k < n and arr[k] <= now:
            ids.append(srv.submit(inputs.make_request(specs[k]), specs[k]["steps"], keep_result=False))
            k += 1
        a, q, d = srv.tick()
        peak = max(peak, a)
        if d == n:
            break
        if a == 0 and q == 0 and k < n:
            time.sleep(max(0.0, min(arr[k] - (time.perf_counter() - t0), 0.01)))
    stop.set()
    th.join(timeout=2)
    info = [srv.query(i) for i in ids]
    failed = sum(1 for x in info if x["state"] != mb.Server.DONE)
    lat = np.array([x["t_done"] - x["t_submit"] for x in info])
    span = max(x["t_done"] for x in info) - min(x["t_submit"] for x in info)
    value = float(work.sum() / span)
    failures = [{"request": "c5_%04d_%s_N%d" % (specs[i]["k"], specs[i]["kind"], specs[i]["N"]),
                 "state": info[i]["state"], "error": info[i]["error"]}
                for i in range(n) if info[i]["state"] != mb.Server.DONE][:10]
    srv.close()
    # serial plain FP64: one request at a time, FP64 throughout, on a seeded
    # subsample; each sampled request's time = its per-step time x its steps
    rng = np.random.default_rng(inputs.BASE_SEED + 5)
    sample = sorted(rng.choice(n, size=min(args.c5_serial_sample, n), replace=False).tolist())
    t_sample, w_sample = 0.0, 0.0
    for i in sample:
        p = inputs.make_request(specs[i])
        s64 = mb.Sim(p, mb.FP64)
        s64.set_stream(st.cuda_stream)
        s64.run(1, 0.0)
        s64.sync()
        e0.record(st)
        s64.run(args.c5_serial_steps, 0.0)
        e1.record(st)
        torch.cuda.synchronize()
        t_sample += e0.elapsed_time(e1) * 1e-3 / args.c5_serial_steps * specs[i]["steps"]
        w_sample += work[i]
        s64.close()
    rate64 = w_sample / t_sample
    serial_s = float(work.sum() / rate64)
    if rank != 0:
        return
    line = {
        "metric": "cell-updates/s aggregate over a served request stream (continuous batching, FP32 bulk); "
                  "p50/p99 completion latency",
        "value": value, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "c5_served_%d_req_N%d-%d_steps%d-%d" % (n, args.c5_nmin, args.c5_nmax, args.c5_smin,
                                                                      args.c5_smax),
                   "arrivals": "Poisson, mean gap %.4g s = %.2f x batched throughput %.3g cell-updates/s"
                               % (mean_gap, args.c5_load, thr),
                   "budget_gib": args.c5_budget_gib, "max_active": args.c5_max_active},
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "mean": float(lat.mean())},
        "requests": n, "failed": failed, "peak_active": peak, "makespan_s": span, "total_cell_updates": float(work.sum()),
        "failures": failures,
        "clocks": summarize_clocks(samples, local),
        "serial_fp64": {"value": rate64, "unit": UNIT, "seconds_for_stream": serial_s,
                        "extrapolated": "from a seeded %d-request subsample: each timed over %d steps after one "
                                        "warm-up step, one instance at a time, scaled by its step count"
                                        % (len(sample), args.c5_serial_steps)},
        "speedup_vs_serial_fp64": serial_s / span,
    }
    print(json.dumps(line))


def run_period_accuracy(args):
    """The pitching NACA 0012 workload (1024^2) over one full pitch period,
    t = 2 pi / omega, in FP32 bulk arithmetic and in FP64, from the same
    initial state at a common fixed step (0.9 times the FP64 CFL step at
    t = 0): relative L1 density error (alpha-weighted over fluid cells) and
    the drift of the conserved totals, FP32 against FP64, at t = T."""
    import torch
    from paper_1711_11361_gb300 import inputs, mb
    torch.cuda.set_device(0)
    prob = inputs.c3_naca(1024)
    T = 2.0 * math.pi / prob.omega
    s64 = mb.Sim(prob, mb.FP64)
    dt0 = float(s64.step(0.0, report=True)[0])
    s64.close()
    nsteps = int(math.ceil(T / (0.9 * dt0)))
    dt = T / nsteps
    res = {}
    for name, prec in (("fp64", mb.FP64), ("fp32", mb.FP32)):
        sim = mb.Sim(prob, prec)
        st = torch.cuda.Stream()
        sim.set_stream(st.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        sim.run(nsteps, dt)
        e1.record(st)
        torch.cuda.synchronize()
        status = sim.sync()
        res[name] = (sim.read_state(0, alpha=True), e0.elapsed_time(e1) * 1e-3, int(status))
        sim.close()
    a64, t64, st64 = res["fp64"]
    a32, t32, st32 = res["fp32"]
    al = a64["alpha"]
    fl = al > 0
    w = al[fl]
    l1 = float(np.sum(w * np.abs(a32["Q"][0][fl] - a64["Q"][0][fl])) / np.sum(w * np.abs(a64["Q"][0][fl])))
    drift = {}
    for q, nm in enumerate(("rho", "rho_u", "rho_v", "E")):
        t_64 = np.sum(w * a64["Q"][q][fl])
        t_32 = np.sum(w * a32["Q"][q][fl])
        scale = np.sum(w * np.abs(a64["Q"][q][fl])) if q in (0, 3) else np.sum(
            w * np.hypot(a64["Q"][1][fl], a64["Q"][2][fl]))
        drift[nm] = float(abs(t_32 - t_64) / scale)
    cells = prob.nx * prob.ny * 2 * nsteps
    print(json.dumps({
        "metric": "FP32 bulk vs FP64 relative L1 density error after one pitch period (pitching NACA 0012)",
        "value": l1, "unit": "relative L1", "higher_is_better": False, "dtype": "f32 vs f64", "data": "synthetic",
        "config": {"workload": "c3_naca0012_1024_one_period", "T": T, "steps": nsteps, "dt": dt,
                   "dt_rule": "0.9 x FP64 CFL step at t = 0, common to both runs"},
        "t_end": {"fp64": a64["t"], "fp32": a32["t"]}, "status": {"fp64": st64, "fp32": st32},
        "conservation_drift_rel": drift,
        "throughput": {"fp64": cells / t64, "fp32": cells / t32, "unit": UNIT, "seconds": {"fp64": t64, "fp32": t32}},
    }))


def run_n1(args):
    """The paper's sloped-channel validation (Sec. III.A) as read in
    inputs.n1_channel, on the plain FP64 GPU path (held to the oracle per
    sweep by tests/test_gpu_configs.py): density error norms against the exact
    translated profile at t_end on the paper's five grids (160x32 ...
    2560x512) for the static channel, the moving channel with the paper's
    donor uncovering and with flux-GCL uncovering, and the paper's
    CFL-halving study (eq. CFLvarying) on the finest three grids.  Each run
    takes a fixed step: t_end split into equal steps no longer than the CFL
    step at t = 0.  Norms over fluid cells, weighted by volume fraction
    (L1, L2) or not (L_inf)."""
    import torch
    from paper_1711_11361_gb300 import inputs, mb
    torch.cuda.set_device(0)

    def run(level, moving, mode, cfl):
        p = inputs.n1_channel(level, moving, cfl=cfl)
        p.uncover_mode = mode
        s = mb.Sim(p, mb.FP64)
        dt0 = float(s.step(0.0, report=True)[0])
        s.close()
        n = int(math.ceil(p.t_end / dt0))
        s = mb.Sim(p, mb.FP64)
        s.run(n, p.t_end / n)
        status = int(s.sync())
        g = s.read_state(0, alpha=True)
        merged = s.merge_count(0)
        s.close()
        X, Y = p.cell_centres()
        a = g["alpha"]
        fl = a > 0
        e = np.abs(g["Q"][0][fl] - inputs.n1_exact_density(X, Y, g["t"], p.U[0])[fl])
        w = a[fl]
        return {"grid": f"{p.nx}x{p.ny}", "cfl": cfl, "steps": n, "status": status, "merged_cells": merged,
                "L1": float(np.sum(w * e) / np.sum(w)), "L2": float(math.sqrt(np.sum(w * e * e) / np.sum(w))),
                "Linf": float(e.max())}

    def orders(rows):
        for a, b in zip(rows, rows[1:]):
            b["orders"] = {k: math.log2(a[k] / b[k]) for k in ("L1", "L2", "Linf")}
        return rows

    out = {"metric": "density error norms of the sloped-channel validation (reading of Sec. III.A)",
           "dtype": "f64", "data": "synthetic", "config": {"workload": "n1_sloped_channel_5x1_160x32-2560x512"}}
    out["static"] = orders([run(l, False, inputs.UNCOVER_DONOR, 0.5) for l in range(5)])
    out["moving_donor"] = orders([run(l, True, inputs.UNCOVER_DONOR, 0.5) for l in range(5)])
    out["moving_flux_gcl"] = orders([run(l, True, inputs.UNCOVER_FLUX_GCL, 0.5) for l in range(5)])
    out["moving_donor_cfl_halving"] = orders([run(l, True, inputs.UNCOVER_DONOR, 0.5 / 2 ** (l - 2))
                                              for l in (2, 3, 4)])
    print(json.dumps(out))


def run_n2(args):
    """The paper's axisymmetric open-ended tube (Sec. III.E) as read in
    inputs.n2_open_tube, on the FP64 GPU path (held to the oracle per sweep by
    tests/test_gpu_configs.py), at 94, 189 and 378 cells per diameter (the
    paper's 1.6 mm and 0.8 mm single-level meshes and its finest AMR level,
    here as a single-level mesh).  Pressure on the axis is probed after every
    step at the exit plane and 1.5 D downstream; reported: the time the shock
    reaches the exit (converted to the paper's start, the piston face at
    5.5 D with no shock yet) and the peak overpressure at the probe with its
    time after that, beside the paper's values in the same units (tau =
    D / sqrt(p/rho) = 0.525 ms for its D = 0.151 m and air)."""
    import torch
    from paper_1711_11361_gb300 import inputs, mb
    torch.cuda.set_device(0)
    tau_ms = 0.1511 / math.sqrt(101325.0 / 1.225) * 1e3
    paper = {"exit_time_tau": 1.388 / tau_ms, "peak_overpressure": 98544.0 / 101325.0,
             "peak_t_ref_tau": 0.398 / tau_ms, "measured_peak_overpressure": 98341.0 / 101325.0,
             "measured_peak_t_ref_tau": 0.394 / tau_ms, "tau_ms": tau_ms}
    rows = []
    for k in args.n2_resolutions:
        p = inputs.n2_open_tube(k)
        info = p.n2
        r2, up, p2 = info["post_shock"]
        sim = mb.Sim(p, mb.FP64)
        cells = [info["exit_cell"], info["probe_cell"]]
        hist = []
        t = 0.0
        t0 = time.perf_counter()
        steps = 0
        while t < p.t_end:
            dt = float(sim.step(0.0, report=True)[0])
            t += dt
            steps += 1
            q = sim.probe(0, cells)
            pr = (p.gamma - 1.0) * (q[3] - 0.5 * (q[1] ** 2 + q[2] ** 2) / q[0])
            hist.append((t, pr[0], pr[1]))
        status = int(sim.sync())
        merged = sim.merge_count(0)
        sim.close()
        h = np.array(hist)
        half = 0.5 * (1.0 + p2)
        k_exit = int(np.argmax(h[:, 1] > half))
        ta, tb, pa, pb = h[k_exit - 1, 0], h[k_exit, 0], h[k_exit - 1, 1], h[k_exit, 1]
        t_exit = ta + (half - pa) * (tb - ta) / (pb - pa)
        # the start configuration has the shock (shock - face) ahead of a face
        # at 5.5 D from the exit; the paper's shock starts at the face
        d = 1.0 / k
        lead = 3.0 * d * info["shock_speed"] / (info["shock_speed"] - up) / info["shock_speed"]
        after = h[:, 0] >= t_exit
        j = int(np.argmax(np.where(after, h[:, 2], -np.inf)))
        rows.append({"cells_per_D": k, "grid": f"{p.nx}x{p.ny}", "steps": steps, "status": status,
                     "merged_cells": merged, "seconds": time.perf_counter() - t0,
                     "exit_time_tau": t_exit + lead, "peak_overpressure": float(h[j, 2] - 1.0),
                     "peak_t_ref_tau": float(h[j, 0] - t_exit)})
    print(json.dumps({"metric": "open-ended tube (reading of Sec. III.E): shock exit time and peak overpressure "
                                "1.5 D downstream on the axis", "dtype": "f64", "data": "synthetic",
                      "config": {"workload": "n2_axisymmetric_open_tube_10Dx4D"},
                      "units": "time in tau = D / sqrt(p/rho); overpressure in units of the ambient pressure",
                      "paper": paper, "runs": rows}))


def n3_flux_profile(precision):
    """(FP64-pipe lane operations, DRAM bytes) per face of the three-
    dimensional flux kernel k3_flux in the given precision ("fp64" or
    "fp32"), from the ncu captures summarised in profiles/n3_flux_ops.json;
    None when mb3.cu has changed since."""
    import hashlib
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "n3_flux_ops.json")))
        for f, sha in d["sources_sha256"].items():
            with open(os.path.join(ROOT, "paper_1711_11361_gb300", "csrc", f), "rb") as fh:
                if hashlib.sha256(fh.read()).hexdigest() != sha:
                    return None
        e = d[precision]
        return float(e["fp64_pipe_lane_ops_per_face"]), float(e["dram_bytes_per_face"])
    except (OSError, KeyError, ValueError):
        return None


N3_FLUX_F32_BYTES = 80   # per face: two cells' FP32 evolved states (2 x 20 B) read, the FP64 flux (40 B) written


def n3_flux_roofline(mb3, p, rate, precision="fp64"):
    """k3_flux, the three-dimensional path's dominant kernel: its device time
    per sweep (CUDA events around each launch on the simulation's stream,
    two steps' sweeps from the initial state) and faces per second.  FP64:
    FP64-pipe lane operations per second against the measured FP64 rate.
    FP32 flux option: algorithmic bytes per second against the measured HBM
    copy bandwidth.  `rate` is the FP64 FMA rate."""
    from paper_1711_11361_gb300 import inputs, mb
    sim = mb3.Sim3(p, precision=mb.FP32 if precision == "fp32" else mb.FP64)
    dt = sim.cfl_dt()
    n = p.nx * p.ny * p.nz
    nn = (p.nx, p.ny, p.nz)
    per = []
    for s in range(3):
        for d in ((0, 1, 2) if s % 2 == 0 else (2, 1, 0)):
            sim.sweep(d, dt)
            nfl = nn[d] + (0 if p.bc[2 * d] == inputs.PERIODIC else 1)
            if s > 0:   # the first step warms up
                per.append((nfl * (n // nn[d]), sim.flux_time_ms() * 1e-3))
    sim.close()
    faces = sum(f for f, _ in per)
    secs = sum(t for _, t in per)
    out = {"kernel": "k3_flux", "precision": precision, "ms_per_sweep": secs / len(per) * 1e3,
           "faces_per_s": faces / secs}
    prof = n3_flux_profile(precision)
    if precision == "fp32":
        hbm, kind = measured_peaks()
        achieved = N3_FLUX_F32_BYTES * faces / secs / 1e9
        out.update({"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                    "algorithmic_bytes_per_face": N3_FLUX_F32_BYTES, "peak_kind": f"{kind} (MEASURED_PEAKS hbm_gbs)",
                    "traffic": None if prof is None else prof[1] * faces / len(per)})
    elif prof is not None:
        ops, dram = prof
        achieved = ops * faces / secs
        out.update({"bound": "fp64", "achieved": achieved / 1e12, "peak": rate / 1e12,
                    "unit": "T FP64-pipe lane-ops/s", "frac": achieved / rate, "fp64_pipe_lane_ops_per_face": ops,
                    "traffic": dram * faces / len(per), "traffic_note": "DRAM bytes per launch, ncu bytes per "
                    "face at 20 cells per D scaled by the faces of one launch here",
                    "peak_kind": "measured: mb_fp64_rate (independent FP64 FMA chains)"})
    return out


def run_n3(args):
    """The paper's three-dimensional Schardin test (Sec. III.F) as read in
    inputs.n3_schardin_cone: a 60-degree cone moving with the gas into a
    stationary Mach-1.34 shock in the 10 D x 10 D x 5 D half domain, on the
    FP64 three-dimensional GPU path (held to the three-dimensional oracle by
    tests/test_gpu_3d.py), until 1.48 tau after contact (the paper's 102 us
    for its 20 mm cone), at each of --n3-resolutions cells per diameter.
    Reports cell-sweeps/s (cells x 3 sweeps per step), the steps, the cells
    merged by the safeguard and the status; the 3-D oracle on a bounded
    sample (the 10-per-D case's first steps, about 10 s) is the CPU baseline.  The FP32
    flux option (mb3_set_precision) runs the finest mesh too, with its
    alpha-weighted L1 density difference from the FP64 path over 40 steps
    at the FP64 path's dt on the 10-per-D mesh."""
    import torch
    from paper_1711_11361_gb300 import inputs, mb, mb3
    torch.cuda.set_device(0)

    def run(k, precision):
        p = inputs.n3_schardin_cone(k)
        sim = mb3.Sim3(p, precision=precision)
        sim.step()                       # untimed warm-up step (buffers, first launch)
        sim.write_state(p.Q0)
        t, steps, merged = 0.0, 0, 0
        t0 = time.perf_counter()
        while t < p.info["t_end"]:
            t += sim.step()
            steps += 1
            merged += sim.last_sweep()[1]
        el = time.perf_counter() - t0
        st = sim.read_state(check=False)
        sim.close()
        return {"cells_per_D": k, "grid": f"{p.nx}x{p.ny}x{p.nz}", "cells": p.info["cells"], "steps": steps,
                "seconds": el, "cell_sweeps_per_s": p.info["cells"] * 3 * steps / el,
                "ms_per_step": el / steps * 1e3, "status": int(st["status"]), "t_end": t,
                "merged_cells_last_sweeps": merged, "precision": "fp32" if precision == mb.FP32 else "fp64"}

    main = mb.FP32 if args.n3_precision == "fp32" else mb.FP64
    rows = [run(k, main) for k in args.n3_resolutions]
    fp32 = None
    if args.n3_precision != "fp64":
        fp32 = run(args.n3_resolutions[-1], mb.FP32) if args.n3_precision == "both" else rows[-1]
        p = inputs.n3_schardin_cone(args.n3_resolutions[0])
        s64, s32 = mb3.Sim3(p), mb3.Sim3(p, precision=mb.FP32)
        for _ in range(40):
            dt = s64.step()
            s32.step(dt)
        a, b = s64.read_state(alpha=True, check=False), s32.read_state(alpha=True, check=False)
        s64.close()
        s32.close()
        fl = a["alpha"] > 0
        w = a["alpha"][fl]
        fp32["l1_density_rel_vs_fp64"] = float(np.sum(w * np.abs(b["Q"][0][fl] - a["Q"][0][fl])) /
                                               np.sum(w * np.abs(a["Q"][0][fl])))
        fp32["accuracy_sample"] = f"{args.n3_resolutions[0]} cells per D, 40 steps at the FP64 path's dt"
        # the whole run (to 1.48 tau) at the FP64 path's dt, on the largest
        # mesh up to 20 cells per D
        kf = max([k for k in args.n3_resolutions if k <= 20] or [args.n3_resolutions[0]])
        p = inputs.n3_schardin_cone(kf)
        s64, s32 = mb3.Sim3(p), mb3.Sim3(p, precision=mb.FP32)
        t = 0.0
        while t < p.info["t_end"]:
            dt = s64.step()
            s32.step(dt)
            t += dt
        a, b = s64.read_state(alpha=True, check=False), s32.read_state(alpha=True, check=False)
        s64.close()
        s32.close()
        fl = a["alpha"] > 0
        w = a["alpha"][fl]
        fp32["l1_density_rel_vs_fp64_whole_run"] = float(np.sum(w * np.abs(b["Q"][0][fl] - a["Q"][0][fl])) /
                                                         np.sum(w * np.abs(a["Q"][0][fl])))
        fp32["whole_run_sample"] = f"{kf} cells per D, to {p.info['t_end']} tau at the FP64 path's dt"
        if args.n3_precision == "both":
            fp32["speedup_vs_fp64"] = fp32["cell_sweeps_per_s"] / rows[-1]["cell_sweeps_per_s"]
    f32 = main == mb.FP32
    line = {"metric": "cell-sweeps/s, three-dimensional " + ("path, FP32 flux option" if f32 else "FP64 path") +
                      " (x, y, z sweeps), Schardin cone",
            "value": rows[-1]["cell_sweeps_per_s"], "unit": "cell-sweeps/s", "dtype": "f32 flux, f64 state" if f32
            else "f64", "data": "synthetic",
            "config": {"workload": "n3_schardin_cone_10Dx10Dx5D", "mach": inputs.N3_MACH,
                       "t_after_contact_tau": inputs.N3_T_AFTER, "cone": "24-sided pyramid, apex angle 60 deg"},
            "runs": rows}
    if args.n3_precision != "fp64":
        line["fp32_flux_option"] = fp32
    rate = mb.fp64_rate(torch.cuda.current_stream().cuda_stream)
    finest = inputs.n3_schardin_cone(args.n3_resolutions[-1])
    line["roofline"] = n3_flux_roofline(mb3, finest, rate, "fp32" if f32 else "fp64")
    if args.n3_precision == "both":
        line["roofline_fp32_flux_option"] = n3_flux_roofline(mb3, finest, rate, "fp32")
    if not args.no_cpu_baseline:
        from oracle import o3
        p = inputs.n3_schardin_cone(10)
        o = o3.Oracle3(p)
        t0 = time.perf_counter()
        nst = 0
        while time.perf_counter() - t0 < 10.0:   # a bounded sample: whole steps for about 10 s
            o.step()
            nst += 1
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": p.info["cells"] * 3 * nst / el, "unit": "cell-sweeps/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"the first {nst} steps of the {p.nx}x{p.ny}x{p.nz} case from its initial "
                                          f"state, {el:.1f} s, single-threaded"}
    print(json.dumps(line))


def workload(rank, args):
    from paper_1711_11361_gb300 import inputs
    if args.workload == "c4":
        seed = None if rank == 0 else inputs.BASE_SEED + 1000 + rank
        return inputs.c4_batch(n=args.instances, seed=seed), "c4_batched_64_uneven_128-1024"
    if args.workload == "c2":
        return [inputs.c2_cylinder(400)], "c2_cylinder_400"
    if args.workload == "c3":
        return [inputs.c3_naca(1024)], "c3_naca0012_1024"
    if args.workload == "c5":
        specs = inputs.c5_requests(n=16, nmin=args.c5_nmin, nmax=args.c5_nmax, smin=args.c5_smin, smax=args.c5_smax)
        return [inputs.make_request(sp) for sp in specs], "c5_served_first16"
    raise SystemExit(f"unknown workload {args.workload}")


def e2e_leg(mb, probs, prec, steps, groups):
    """End to end through the C ABI: every step writes every instance's state
    from page-locked host memory in the batch's precision (mb_write_states_f32
    for the FP32 batch, mb_write_states for FP64), takes one step, and reads
    every state back the same way.  The instances are split into `groups`
    sub-batches of about equal cells, each with its own simulation, streams
    and host thread, so that one group's copies overlap another's step and the
    host link carries both directions at once.  Returns (cell-updates/s, bytes
    in per step, bytes out per step)."""
    import threading
    import torch
    f32 = prec == mb.FP32
    ndt, tdt = (np.float32, torch.float32) if f32 else (np.float64, torch.float64)
    order = sorted(range(len(probs)), key=lambda k: -probs[k].nx * probs[k].ny)
    gs, load = [[] for _ in range(max(1, groups))], [0] * max(1, groups)
    for k in order:   # largest instance onto the lightest group
        g = min(range(len(gs)), key=lambda q: load[q])
        gs[g].append(k)
        load[g] += probs[k].nx * probs[k].ny
    gs = [sorted(g) for g in gs if g]
    sims, ins, outs = [], [], []
    for g in gs:
        ps = [probs[k] for k in g]
        sims.append(mb.Sim(ps, prec))
        ins.append([torch.from_numpy(np.ascontiguousarray(p.Q0, dtype=ndt)).pin_memory() for p in ps])
        outs.append([torch.empty((p.nc, p.ny, p.nx), dtype=tdt).pin_memory() for p in ps])
    errors = []

    def run(q, n):
        try:
            s, a, b = sims[q], [t.data_ptr() for t in ins[q]], [t.data_ptr() for t in outs[q]]
            for _ in range(n):
                s.write_states(a, dtype=ndt)
                s.step(0.0)
                s.read_states(b, dtype=ndt)
        except Exception as ex:   # reported after the join
            errors.append(ex)

    def all_groups(n):
        ths = [threading.Thread(target=run, args=(q, n)) for q in range(len(sims))]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        if errors:
            raise RuntimeError(f"e2e state I/O failed: {errors[0]}")

    all_groups(1)   # untimed warm-up of the I/O path
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    all_groups(steps)
    el = time.perf_counter() - t0
    cells = sum(p.nx * p.ny for p in probs)
    nbytes = sum(t.numel() * t.element_size() for lst in ins for t in lst)
    for s in sims:
        s.close()
    return cells * 2 * steps / el, nbytes, nbytes, len(sims)


def cpu_baseline(probs, budget_s=12.0):
    """The oracle as it stands on this host's cores, on a bounded sample:
    full steps of the smallest instance of the workload until about
    budget_s of CPU time."""
    import oracle
    p = min(probs, key=lambda q: q.nx * q.ny)
    o = oracle.Oracle(p)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        o.step()
        steps += 1
    el = time.perf_counter() - t0
    value = p.nx * p.ny * 2 * steps / el
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{steps} full steps of instance {p.name} ({p.nx}x{p.ny}), {el:.1f} s, single-threaded"}


def _oracle_worker(args):
    """One host process: full oracle steps of one instance for about
    budget_s seconds; returns the cell-updates done and the seconds taken."""
    prob, budget_s = args
    import oracle
    o = oracle.Oracle(prob)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        o.step()
        steps += 1
    return prob.nx * prob.ny * 2 * steps, time.perf_counter() - t0


def cpu_baseline_all_cores(probs, budget_s=10.0):
    """The same oracle on every host core at once, one independent instance
    per process (the batch's smallest instances; spawned processes, so no
    CUDA state is inherited): aggregate cell-updates/s."""
    import multiprocessing as mp
    n = max(1, os.cpu_count() or 1)
    pick = sorted(probs, key=lambda q: q.nx * q.ny)
    pick = [pick[k % len(pick)] for k in range(n)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_worker, [(p, budget_s) for p in pick])
    wall = time.perf_counter() - t0
    cells = sum(r[0] for r in res)
    span = max(r[1] for r in res)
    return {"value": cells / span, "unit": UNIT, "cores": n, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{n} processes, one instance each (smallest of the batch, {pick[0].nx}^2 to "
                      f"{pick[-1].nx}^2), full steps for {budget_s:.0f} s; wall {wall:.1f} s with start-up"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    probs, wname = workload(0, args)
    import oracle
    p = min(probs, key=lambda q: q.nx * q.ny)
    o = oracle.Oracle(p)
    for _ in range(args.warmup):
        o.step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.step()
        times.append(time.perf_counter() - t0)
    cells = p.nx * p.ny * 2
    tot = sum(times)
    value = cells * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "sample": f"instance {p.name} ({p.nx}x{p.ny}) per step"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value, "unit": UNIT,
                             "sample": f"one full step of {p.name} per timed step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mb", choices=["mb", "reference"])
    ap.add_argument("--workload", default="c4")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-groups", type=int, default=8,
                    help="sub-batches (own simulation, streams and host thread each) of the end-to-end leg")
    ap.add_argument("--sweep-samples", type=int, default=100, help="steps sampled for the per-sweep p50/p99")
    ap.add_argument("--n2-resolutions", type=int, nargs="+", default=[94, 189, 378],
                    help="cells per tube diameter of the open-tube runs")
    ap.add_argument("--n3-resolutions", type=int, nargs="+", default=[10, 20],
                    help="cells per cone diameter of the three-dimensional Schardin runs")
    ap.add_argument("--n3-precision", choices=["both", "fp64", "fp32"], default="both",
                    help="three-dimensional runs: the FP64 path with the FP32 flux option beside it, or one of them")
    ap.add_argument("--c3-period", action="store_true",
                    help="FP32 vs FP64 accuracy of the pitching NACA 0012 workload after one full pitch period")
    ap.add_argument("--accuracy-steps", type=int, default=500,
                    help="steps of the FP32-vs-FP64 accuracy leg (the 64-instance workload runs 500)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="launch shapes of the bulk kernels from mb_autotune (it times the kernels alone, outside the "
                         "overlapped step; on the 64-instance batch its picks measured about 1.5% slower per step "
                         "than the default shapes)")
    ap.add_argument("--no-autotune", action="store_true", help="the default launch shapes (the default)")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the FP32-vs-FP64 and FP64 single-instance legs")
    ap.add_argument("--c5-requests", type=int, default=2000)
    ap.add_argument("--c5-nmin", type=int, default=256)
    ap.add_argument("--c5-nmax", type=int, default=2048)
    ap.add_argument("--c5-smin", type=int, default=500)
    ap.add_argument("--c5-smax", type=int, default=5000)
    ap.add_argument("--c5-serial-sample", type=int, default=50)
    ap.add_argument("--c5-serial-steps", type=int, default=4)
    ap.add_argument("--c5-load", type=float, default=0.9)
    ap.add_argument("--c5-budget-gib", type=float, default=32.0)
    ap.add_argument("--c5-max-active", type=int, default=64)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c5":
        return run_served(args)
    if args.c3_period:
        return run_period_accuracy(args)
    if args.workload == "n1":
        return run_n1(args)
    if args.workload == "n2":
        return run_n2(args)
    if args.workload == "n3":
        return run_n3(args)

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1711_11361_gb300 import mb

    probs, wname = workload(rank, args)
    prec = mb.FP32 if args.precision == "fp32" else mb.FP64
    sim = mb.Sim(probs, prec)
    stream = torch.cuda.Stream()
    sim.set_stream(stream.cuda_stream)
    tune = sim.autotune() if args.autotune and not args.no_autotune else {"x_cta": None, "y_cta": None,
                                                                           "y_rows": None}
    cells = sum(p.nx * p.ny for p in probs)
    with torch.cuda.stream(stream):
        sim.run(args.warmup, 0.0)
    sim.sync()
    # timed region: K graph replays, per-step events
    stop = threading.Event()
    samples = []
    th = threading.Thread(target=sample_clocks, args=(stop, samples), daemon=True)
    th.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        evs[0].record(stream)
        for k in range(args.steps):
            sim.run(1, 0.0)
            evs[k + 1].record(stream)
    torch.cuda.synchronize()
    stop.set()
    th.join(timeout=2)
    per = np.array([evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)])
    total_ms, cells_all = combine_ranks(float(per.sum()), cells, "cuda")
    status = sim.sync()
    value = job_value(cells_all, args.steps, total_ms)

    # the same steps with every bulk cell waiting for the band fluxes (no
    # overlap of the bulk pass with the geometry), for comparison
    serial_ms = None
    if prec == mb.FP32:
        sim.set_overlap(False)
        with torch.cuda.stream(stream):
            sim.run(2, 0.0)
            e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            sim.run(10, 0.0)
            e_b.record(stream)
        torch.cuda.synchronize()
        serial_ms = e_a.elapsed_time(e_b) / 10
        sim.set_overlap(True)

    # dominant kernel: bulk sweep, timed with CUDA events on its stream
    sim.enable_timing(True)
    sim.run(4, 0.0)
    bulk_ms, launches = sim.kernel_time()
    sim.enable_timing(False)
    avg_bulk_s = bulk_ms * 1e-3 / max(launches, 1)
    bpc = BYTES_PER_CELL_FP32 if prec == mb.FP32 else BYTES_PER_CELL_FP64
    achieved = cells * bpc / avg_bulk_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = bulk_traffic(args.precision, wname)
    ops_per_cell = bulk_alu(args.precision, wname)

    # per-sweep times of the real path (step graph replay): an event recorded
    # between a step's two sweeps, one step per sample
    ev_mid = torch.cuda.Event(enable_timing=True)
    ev_mid.record(stream)
    torch.cuda.synchronize()
    sim.set_sweep_event(ev_mid.cuda_event)
    e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sweeps = []
    with torch.cuda.stream(stream):
        sim.run(2, 0.0)
        for k in range(args.sweep_samples):
            e_a.record(stream)
            sim.run(1, 0.0)
            e_b.record(stream)
            e_b.synchronize()
            sweeps += [e_a.elapsed_time(ev_mid), ev_mid.elapsed_time(e_b)]
    torch.cuda.synchronize()
    sim.set_sweep_event(0)
    kernels_per_step = sim.graph_kernels()

    # end to end through the C ABI with pinned host buffers
    pinned_in = [torch.empty((p.nc, p.ny, p.nx), dtype=torch.float64).pin_memory() for p in probs]
    pinned_out = [torch.empty((p.nc, p.ny, p.nx), dtype=torch.float64).pin_memory() for p in probs]
    for k, p in enumerate(probs):
        pinned_in[k].copy_(torch.from_numpy(p.Q0))
    h2d = sum(t.numel() * 8 for t in pinned_in)
    e2e_steps = max(1, args.e2e_steps)
    p_in = sim._ptrs([t.data_ptr() for t in pinned_in])
    p_out = sim._ptrs([t.data_ptr() for t in pinned_out])
    mb.lib.mb_write_states(sim._h, p_in, None)   # untimed warm-up of the I/O path
    mb.lib.mb_read_states(sim._h, p_out, None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        # every instance's state in from pinned host memory, one step, every
        # state back out (mb_write_states / mb_step / mb_read_states)
        r_in = mb.lib.mb_write_states(sim._h, p_in, None)
        sim.step(0.0)
        r_out = mb.lib.mb_read_states(sim._h, p_out, None)
        if r_in != 0 or r_out != 0:
            raise RuntimeError(f"e2e state I/O failed: {r_in} {r_out}")
    e2e_s = time.perf_counter() - t0
    e2e_one_batch = cells * 2 * e2e_steps / e2e_s * (ws if ws > 1 else 1)
    e2e_value, e2e_in, e2e_out, e2e_groups = e2e_leg(mb, probs, prec, e2e_steps, args.e2e_groups)
    e2e_value *= ws if ws > 1 else 1

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == mb.FP32 else "f64", "data": "synthetic",
        "config": {"workload": wname, "instances": len(probs), "cells_per_sweep": cells,
                   "grid_sizes": [p.nx for p in probs], "bulk": args.precision,
                   "geometry_and_weights": "f64", "dt": "per-instance CFL on device",
                   "l2": "inputs larger than L2 (state per buffer %.2f GB)" % (cells * 16 / 1e9),
                   "parallelism": "instances" if ws == 1 else f"instances x{ws} ranks",
                   "autotuned": {k: tune.get(k) for k in ("x_cta", "y_cta", "y_rows", "x_min_ctas", "y_min_ctas",
                                                          "x_ring_chunks")}},
        "p50_ms_per_step": float(np.percentile(per, 50)), "p99_ms_per_step": float(np.percentile(per, 99)),
        "per_sweep_ms": {"p50": float(np.percentile(sweeps, 50)), "p99": float(np.percentile(sweeps, 99)),
                         "sweeps": len(sweeps),
                         "how": "CUDA events around single step-graph replays with an event between the sweeps"},
        "ms_per_step_without_overlap": serial_ms,
        "status": int(status),
        "roofline": {"kernel": "bulk sweep update (MUSCL-Hancock + HLLC), x and y: the pass concurrent with the "
                               "geometry plus the deferred cell pairs, per sweep", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": peak_kind, "bytes_per_cell": bpc, "avg_launch_ms": avg_bulk_s * 1e3,
                     "launches_timed": launches},
        # the same kernels against the FP32 lanes (context: they are issue-bound)
        "alu": None if ops_per_cell is None else {
            "fp32_lane_ops_per_cell": ops_per_cell, "achieved": ops_per_cell * cells / avg_bulk_s / 1e12,
            "peak": FP32_LANE_OPS_PEAK / 1e12, "unit": "T FP32 lane-ops/s",
            "frac": ops_per_cell * cells / avg_bulk_s / FP32_LANE_OPS_PEAK,
            "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz"},
        "clocks": summarize_clocks(samples, local),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": e2e_in, "d2h_bytes_per_step": e2e_out,
                "steps": e2e_steps, "host_dtype": "f32" if prec == mb.FP32 else "f64", "groups": e2e_groups,
                "how": "every step: every instance's state written from page-locked host memory in the batch's "
                       "precision (mb_write_states_f32 / mb_write_states), one step, every state read back; the "
                       "instances in sub-batches of about equal cells, one simulation, stream set and host thread "
                       "each, so that copies of one overlap the step of another",
                "one_batch_f64_host": {"value": e2e_one_batch, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
                                       "how": "the same with FP64 host states through one 64-instance batch"}},
        "gpu_launches": kernels_per_step * args.steps,
        "kernels_per_step": kernels_per_step,
    }
    if args.workload == "c4" and not args.no_accuracy:
        line["accuracy"] = accuracy_leg(mb, probs, steps=args.accuracy_steps)
        f64 = fp64_single_leg(mb, probs)
        line["fp64_single_instance"] = f64
        line["fp64_batch"] = fp64_roofline_leg(mb, probs, wname, stream)
        line["speedup_vs_fp64_single_instance"] = value / f64["value"]
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(probs)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(probs)
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
