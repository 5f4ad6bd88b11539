"""Throughput of the GB300 adaptive ray-tracing RT step.

One bench step = one complete simulation of the 16-source cosmological
workload: 128^3 lognormal density (sigma_ln = 1, P(k) ~ k^-2) in a 0.5 Mpc/h
box at z = 9, 16 sources in the densest cells (log-uniform 1e51..1e52 /s),
a 4-bin 1e5 K blackbody, temperature evolution, 100 RT steps of 0.1 Myr.
Every RT step runs emission, the fused march/deposit/split kernel and the
chemistry kernel.

value  : ray-cell segments per second with the density and sources already
         resident on the device (CUDA events on the simulation's stream).
e2e    : the same metric through the C-ABI from host buffers: create (H2D of
         the density), sources, 100 steps, fields back to the host (D2H).
roofline: the march kernel's algorithmic bytes per launch over its average
         CUDA-event duration, against the measured HBM copy bandwidth.
cpu_baseline / --impl reference: the FP64 C oracle on the host cores on a
         bounded sample of the same workload (its first RT steps).

Multi-GPU (torchrun): independent replicas, one simulation per rank per step
("replicas only": the simulations do not exchange data); value = segments of
all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ray-cell segments/s"
UNIT = "segments/s"
DEFAULT_PEAK_GBS = 6800.0
WORKLOAD_DESC = ("cosmo16: 128^3 lognormal (sigma_ln=1, P~k^-2) 0.5 Mpc/h z=9, 16 sources 1e51-1e52/s, "
                 "4-bin 1e5 K blackbody, T evolution, 100 RT steps x 0.1 Myr (one simulation per step)")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Dist:
    """Barrier and max-reduction across replicas (gloo on CPU, nccl on GPU)."""

    def __init__(self, backend=None):
        self.ws, self.rank, self.local = dist_env()
        self.pg = None
        if self.ws > 1:
            import torch.distributed as td
            td.init_process_group(backend=backend or "nccl")
            self.td = td

    def barrier(self):
        if self.ws > 1:
            self.td.barrier()

    def max(self, x: float) -> float:
        if self.ws == 1:
            return x
        import torch
        dev = "cuda" if self.td.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.td.all_reduce(t, op=self.td.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if self.ws == 1:
            return x
        import torch
        dev = "cuda" if self.td.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.td.all_reduce(t, op=self.td.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.ws > 1:
            self.td.destroy_process_group()


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return DEFAULT_PEAK_GBS, "fallback"


def kernel_sources_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in ("frt_march.cuh", "frt_kernels.cu", "frt_device.cuh", "frt_types.h"):
        with open(os.path.join(ROOT, "paper_2409_04521_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic():
    """DRAM bytes per march launch from the committed ncu summary, or None
    when the kernel sources have changed since those counters were taken."""
    p = os.path.join(ROOT, "profiles", "march_cosmo16_traffic.txt")
    try:
        vals = {}
        for line in open(p):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                vals[k.strip()] = v.strip().split()[0]
        if vals.get("kernel_sources_sha1") != kernel_sources_sha1():
            return None
        return float(vals["bytes_per_launch_scaled"])
    except Exception:
        return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
def problem(args):
    import dataclasses as dc
    import workloads as W
    if getattr(args, "problem", "cosmo16") == "cosmo20k":
        p = W.cosmo20k()
    else:
        p = W.cosmo16(n=args.grid, nsteps=args.rt_steps)
    if getattr(args, "gamma_iters", 1) > 1:
        p = dc.replace(p, options=dc.replace(p.options, gamma_iters=args.gamma_iters))
    if getattr(args, "gen_mode", False):
        p = dc.replace(p, options=dc.replace(p.options, gen_mode=True, gamma_iters=max(args.gamma_iters, 4)))
    return p


def workload_desc(args):
    if getattr(args, "problem", "cosmo16") == "cosmo20k":
        d = ("cosmo20k: 200^3 lognormal (sigma_ln=0.6) 200 Mpc/h z=7, 2e4 sources drawn by density, "
             "3 bins, sub-grid mfp law, isothermal, 200 RT steps x 1 Myr (one simulation per step)")
    else:
        d = WORKLOAD_DESC
    if getattr(args, "gen_mode", False):
        d += "; Generalized Opacity mode"
    return d


def run_oracle_sample(prob, budget_s, keep=False):
    """Oracle on the first RT steps of the workload until `budget_s` seconds
    of CPU work; returns (segments, seconds, steps[, fields, budget])."""
    import oracle
    t0 = time.perf_counter()
    o = oracle.OracleSim(prob)
    steps = 0
    while steps < prob.nsteps:
        o.step(prob.dt)
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    seg = o.counts()["segments_total"]
    extra = (o.fields(), o.budget()) if keep else ()
    o.close()
    return (seg, dt, steps) + extra


def oracle_parity(prob, steps, of, ob, capacity, variant):
    """The GPU path over the same first RT steps as the oracle sample: max
    and median error per field (Gamma_HI and n_HI relative on cells above
    1e-8 of their largest value, x_HII absolute, T relative) and the budget."""
    import paper_2409_04521_gb300 as F
    g = F.Simulation(prob, ray_capacity=capacity)
    if variant:
        g.set_launch(variant["agg"], variant["minb"], variant["blocks_per_sm"], variant["threads"], variant["slab"])
    for _ in range(steps):
        g.step(prob.dt)
    gf, gb = g.fields(), g.budget()
    g.close()

    def stats(a, b, rel, floor=1e-8):
        if rel:
            m = b >= floor * max(float(b.max()), 1e-300)
            e = np.abs(a - b)[m] / b[m] if m.any() else np.zeros(1)
        else:
            e = np.abs(a - b)
        return [float(e.max()), float(np.median(e))]
    return {"rt_steps": steps, "stat": "[max, median]",
            "gamma_HI_rel": stats(gf["gamma_HI"], of["gamma_HI"], True),
            "x_HII_abs": stats(gf["x_HII"], of["x_HII"], False),
            "T_rel": stats(gf["T"] / of["T"], np.ones_like(of["T"]), False),
            "n_HI_rel": stats(gf["n_HI"], of["n_HI"], True),
            "budget_rel_of_emitted": float(np.max(np.abs(gb - ob)) / ob[0])}


def impl_reference(args, dist):
    if dist.rank != 0:
        return
    prob = problem(args)
    for _ in range(args.warmup):
        run_oracle_sample(prob, args.ref_budget)
    segs, secs, steps = 0, 0.0, []
    for _ in range(args.steps):
        s, t, k = run_oracle_sample(prob, args.ref_budget)
        segs += s
        secs += t
        steps.append(k)
    v = segs / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_DESC},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {min(steps)}-{max(steps)} RT steps of the workload per step "
                                       f"(about {args.ref_budget:.0f} s of single-thread FP64 C each)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def impl_gpu(args, dist):
    import torch
    import paper_2409_04521_gb300 as F

    torch.cuda.set_device(dist.local)
    dev_index = torch.cuda.current_device()
    prob = problem(args)
    stream = torch.cuda.Stream()
    ncell = prob.ncell
    nb = prob.spectrum.nbins

    # device-resident runs
    sim = F.Simulation(prob, ray_capacity=args.capacity, stream=stream.cuda_stream)
    max_rays = 0
    tuned = None
    if args.variant:
        v = tuple(int(x) for x in args.variant.split(","))
        sim.set_launch(*v)
        v = v + (256, 512)[len(v) - 3:] if len(v) < 5 else v
        tuned = {"variant": {"agg": v[0], "minb": v[1], "blocks_per_sm": v[2], "threads": v[3], "slab": v[4]},
                 "candidates": 0}
    elif not args.no_tune:
        from paper_2409_04521_gb300 import autotune
        best, table = autotune.tune(sim, prob)
        tuned = {"variant": {"agg": best[0], "minb": best[1], "blocks_per_sm": best[2], "threads": best[3],
                             "slab": best[4]}, "candidates": len(table)}

    def one_sim():
        nonlocal max_rays
        sim.reset()
        for _ in range(prob.nsteps):
            sim.step(prob.dt)

    for _ in range(args.warmup):
        one_sim()
        sim.sync()
        max_rays = max(max_rays, sim.counts()["rays"])
    torch.cuda.synchronize()
    sim.profile(True)
    clocks = ClockSampler(dev_index)
    seg0 = 0
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    segs = 0
    ev0.record(stream)
    for _ in range(args.steps):
        one_sim()
        c = sim.counts()   # synchronises; reads this simulation's segment total
        segs += c["segments_total"] - seg0
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    kms, klaunch, krays = sim.kernel_times()
    sim.profile(False)
    # Generalized mode: photons the moving screens absorbed beyond their atoms
    # (ionising nothing) over those emitted, in the last timed simulation
    screen_excess = None
    if prob.options.gen_mode:
        screen_excess = sim.screen_excess() / max(sim.budget()[0], 1e-300)
    sim.close()

    t_max = dist.max(ms)
    segs_all = dist.sum(float(segs))
    value = segs_all / (t_max * 1e-3)

    # algorithmic bytes of the march kernel (per launch): rays read
    # (pixlev, emitter, birth, dir, photons) and photons written, plus the
    # compulsory cell traffic (kappa read, deposits read and written).
    ray_read = 24 + 4 * nb
    ray_write = 4 * nb
    b_cell = 8 + 24
    march_launches = max(int(klaunch["march"]), 1)
    alg_bytes = krays * (ray_read + ray_write) + march_launches * ncell * b_cell
    per_launch_bytes = alg_bytes / march_launches
    per_launch_s = kms["march"] * 1e-3 / march_launches
    achieved = per_launch_bytes / per_launch_s / 1e9
    peak, peak_src = measured_peak()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": committed_traffic(), "kernel": "k_march (fused march+deposit+split+compact)",
                "peak_source": peak_src, "algorithmic_bytes_per_launch": per_launch_bytes,
                "avg_launch_ms": per_launch_s * 1e3,
                "kernel_ms": {k: float(v) for k, v in kms.items()},
                "kernel_share": {k: float(v / max(sum(kms.values()), 1e-30)) for k, v in kms.items()}}

    # end to end through the C-ABI from host buffers
    e2e = None
    if not args.no_e2e:
        e2e_segs, e2e_t = 0, 0.0
        h2d = d2h = 0
        for _ in range(max(1, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = F.Simulation(prob, ray_capacity=args.capacity)
            if tuned:
                v = tuned["variant"]
                s2.set_launch(v["agg"], v["minb"], v["blocks_per_sm"], v["threads"], v["slab"])
            for _ in range(prob.nsteps):
                s2.step(prob.dt)
            f = s2.fields()
            t1 = time.perf_counter()
            e2e_segs += s2.counts()["segments_total"]
            e2e_t += t1 - t0
            s2.close()
            # host buffers the C ABI copies: the density, the sources and the
            # spectrum tables in; the per-cell state flexrt_get_fields reads
            # back (x f32, neutral fraction f64 and n_H f64 for n_HI, T f32,
            # Gamma f32)
            h2d = (np.asarray(prob.nH, np.float64).nbytes + np.asarray(prob.source_cells, np.int32).nbytes
                   + np.asarray(prob.source_ndot, np.float64).nbytes + 3 * nb * 8)
            d2h = ncell * (4 + 8 + 8 + 4 + 4)
            del f
        e2e = {"value": dist.sum(e2e_segs) / dist.max(e2e_t), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "note": "create+sources+100 RT steps+fields per step, host wall clock", "runs": max(1, args.steps)}

    # oracle baseline on the host cores (rank 0 only, N=1 only), and the
    # GPU's error against it over the same RT steps
    cpu = parity = None
    if dist.rank == 0 and dist.ws == 1 and not args.no_cpu:
        s, t, k, of, ob = run_oracle_sample(prob, args.ref_budget, keep=True)
        cpu = {"value": s / t, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {k} of {prob.nsteps} RT steps of the same workload, single-thread FP64 C "
                         f"({t:.1f} s)"}
        parity = oracle_parity(prob, k, of, ob, args.capacity, tuned["variant"] if tuned else None)

    # the batched and served forms against the plain path (N=1 only)
    batch = serve_line = None
    if dist.rank == 0 and dist.ws == 1 and not args.no_extra:
        batch = run_batch(args)
        serve_line = run_serve(args)

    launches_per_sim = 1 + prob.nsteps * (3 + (1 if len(prob.source_ndot) else 0)
                                          + 3 * (prob.options.gamma_iters - 1))
    if dist.rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": workload_desc(args), "grid": prob.grid[0], "rt_steps": prob.nsteps,
                           "gamma_iters": prob.options.gamma_iters,
                           "ray_capacity": args.capacity, "max_live_rays": max_rays,
                           "parallelism": f"replicas x{dist.ws}",
                           "l2": "working set larger than L2 (ray queues of several GB)",
                           "precision": "rays, deposits, segment lengths fp32; ionisation update in sums of "
                                        "positive terms with fp32 factors, neutral fraction combined and stored "
                                        "in fp64; temperature fp32; photon budget fp64 (error against the fp64 "
                                        "oracle: oracle_parity)",
                           "march_launch": tuned},
                "sims_per_hour": 3600.0 / (t_max * 1e-3 / args.steps) * dist.ws,
                "segments_per_sim": segs_all / args.steps / dist.ws,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches_per_sim * args.steps,
                "oracle_parity": parity, "batch": batch, "serve": serve_line}
        if screen_excess is not None:
            line["screen_excess_rel_of_emitted"] = screen_excess
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# batched and served configurations (extra lines; the default line above is
# the single-simulation workload)
# --------------------------------------------------------------------------
def _calibrate_capacity(prob):
    """Largest live-ray count of one simulation (untimed pre-pass)."""
    import paper_2409_04521_gb300 as F
    cap = max(1 << 20, 256 * prob.ncell)
    s = F.Simulation(prob, ray_capacity=cap)
    peak = 0
    for _ in range(prob.nsteps):
        s.step(prob.dt)
        peak = max(peak, s.counts()["rays"])
    s.close()
    return peak


def run_batch(args):
    """64 uneven simulations (32..96^3, 50 steps each): one batch with one
    launch per kernel per step for all members, against looping the
    single-simulation path over the same members; both from host inputs to
    fields on the host.  Returns a summary dict."""
    import torch
    import paper_2409_04521_gb300 as F
    import workloads as W
    probs = W.batch64(count=args.batch_count, nsteps=args.batch_steps)
    peaks = [_calibrate_capacity(p) for p in probs]
    caps = [int(1.25 * p) + 4096 for p in peaks]
    ncell = sum(p.ncell for p in probs)
    nem = sum(len(p.source_ndot) for p in probs)
    B = F.Batch(max_sims=len(probs), max_grid=max(p.grid[0] for p in probs), nbins=3,
                ray_capacity=sum(caps) + 64 * 1024, cell_capacity=ncell, emitter_capacity=nem + 64)

    def batched():
        slots = [B.add(p) for p in probs]
        for _ in range(args.batch_steps):
            B.step()
        B.sync()
        segs = 0
        for sl in slots:
            B.fields(sl)
            segs += B.counts(sl)["segments_total"]
        for sl in slots:
            B.retire(sl)
        B.step()          # lets the retired members' emitters be reused
        B.sync()
        return segs

    def plain():
        segs = 0
        for p, cap in zip(probs, caps):
            s = F.Simulation(p, ray_capacity=cap)
            s.set_launch(*best)
            for _ in range(args.batch_steps):
                s.step(p.dt)
            s.fields()
            segs += s.counts()["segments_total"]
            s.close()
        return segs

    # the autotuner's candidates, each timed on one whole batched run
    from paper_2409_04521_gb300 import autotune
    table = []

    def timed(vs):
        for v in vs:
            try:
                B.set_launch(*v)
            except F.FlexRTError:
                continue
            t0 = time.perf_counter()
            batched()
            table.append((time.perf_counter() - t0, v))
    timed(autotune.CANDIDATES)
    b3 = min(table)[1][:3]
    timed([b3 + sh for sh in autotune.SHAPES if sh != (256, 512)])
    best = min(table)[1]
    B.set_launch(*best)
    for _ in range(args.warmup):
        batched()
    tb, sb = [], 0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sb = batched()
        tb.append(time.perf_counter() - t0)
    plain()
    tp = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sp = plain()
        tp.append(time.perf_counter() - t0)
    B.close()
    t_b, t_p = statistics.median(tb), statistics.median(tp)
    return {"workload": f"batch{len(probs)}: uneven {sorted(set(p.grid[0] for p in probs))}^3, "
                        f"{args.batch_steps} RT steps each, 3 bins, mfp law, z=7; host inputs to host fields",
            "members": len(probs), "cells": ncell, "emitters": nem,
            "march_launch": {"agg": best[0], "minb": best[1], "blocks_per_sm": best[2], "threads": best[3],
                             "slab": best[4]},
            "batched": {"sims_per_hour": 3600 * len(probs) / t_b, "seconds": t_b, "segments_per_s": sb / t_b,
                        "runs": len(tb)},
            "plain_loop": {"sims_per_hour": 3600 * len(probs) / t_p, "seconds": t_p, "segments_per_s": sp / t_p,
                           "runs": len(tp)},
            "speedup_vs_plain": t_p / t_b}


def impl_batch(args, dist):
    import torch
    torch.cuda.set_device(dist.local)
    r = run_batch(args)
    line = {"metric": "sims/hour", "value": r["batched"]["sims_per_hour"], "unit": "sims/hour", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * r["batched"]["seconds"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": r["workload"]}, "batch": r,
            "e2e": {"value": r["batched"]["sims_per_hour"], "unit": "sims/hour",
                    "h2d_bytes_per_step": r["cells"] * 8, "d2h_bytes_per_step": r["cells"] * 28}}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Poisson request stream served by continuous batching under an HBM
    budget, against serving the same stream one simulation at a time; then
    the same requests offered faster than either path serves them."""
    from paper_2409_04521_gb300 import serve
    import workloads as W
    reqs = W.request_stream(count=args.requests, mean_gap_s=args.mean_gap)
    res_b, st_b = serve.serve(reqs, hbm_budget_bytes=args.hbm_budget)
    res_s, st_s = serve.serve_sequential(reqs)
    sat = [(t * args.saturate_gap / args.mean_gap, p) for t, p in reqs]
    _, sat_b = serve.serve(sat, hbm_budget_bytes=args.hbm_budget)
    _, sat_s = serve.serve_sequential(sat)
    return {"workload": f"serve: {args.requests} Poisson requests (mean gap {args.mean_gap} s), "
                        "grids {32,64,96,128,160}^3, 50-200 RT steps, 3 bins, mfp law",
            "hbm_budget_bytes": args.hbm_budget,
            "served": st_b, "sequential": st_s, "p50_s": st_b["p50_s"], "p99_s": st_b["p99_s"],
            "sequential_p50_s": st_s["p50_s"], "sequential_p99_s": st_s["p99_s"],
            "speedup_sims_per_hour": st_b["sims_per_hour"] / st_s["sims_per_hour"],
            "saturated": {"mean_gap_s": args.saturate_gap, "served": sat_b, "sequential": sat_s,
                          "speedup_sims_per_hour": sat_b["sims_per_hour"] / sat_s["sims_per_hour"]}}


def impl_serve(args, dist):
    import torch
    torch.cuda.set_device(dist.local)
    r = run_serve(args)
    st_b = r["served"]
    line = {"metric": "sims/hour", "value": st_b["sims_per_hour"], "unit": "sims/hour", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": 1e3 * st_b["wall_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": r["workload"], "hbm_budget_bytes": args.hbm_budget}, "serve": r}
    print(json.dumps(line), flush=True)


def impl_merge(args, dist):
    """Ray merging (Sec. 3.3) on the 16-source cosmological workload, as in
    Sec. 7.1 (Test 4 with 12 merge directions and N_ex = 16 and 4): time per
    simulation against the unmerged run, and the largest deviation of the
    global ionised fraction and Gamma from the unmerged run over the run."""
    import dataclasses as dc
    import torch
    import paper_2409_04521_gb300 as F
    from paper_2409_04521_gb300 import autotune

    torch.cuda.set_device(dist.local)
    dev_index = torch.cuda.current_device()
    base = problem(args)
    stream = torch.cuda.Stream()
    cases = [("plain", base)]
    for nex in args.merge_nex:
        cases.append((f"n_ex={nex:g},l_merge={args.l_merge}",
                      dc.replace(base, options=dc.replace(base.options, merge=True, n_ex=float(nex),
                                                          l_merge=args.l_merge))))
    results = {}
    traces = {}
    clocks = ClockSampler(dev_index)
    clk = None
    for name, prob in cases:
        sim = F.Simulation(prob, ray_capacity=args.capacity, stream=stream.cuda_stream)
        if not args.no_tune:
            autotune.tune(sim, prob)
        # untimed run sampling the global averages every `every` steps
        every = max(1, prob.nsteps // 20)
        tr = []
        sim.reset()
        for s in range(prob.nsteps):
            sim.step(prob.dt)
            if (s + 1) % every == 0:
                f = sim.fields(("x_HII", "gamma_HI"))
                tr.append((float(f["x_HII"].mean()), float((f["x_HII"] * prob.nH).sum() / prob.nH.sum()),
                           float(f["gamma_HI"].mean())))
        traces[name] = np.array(tr)
        max_rays = sim.counts()["rays"]
        for _ in range(args.warmup):
            sim.reset()
            for _ in range(prob.nsteps):
                sim.step(prob.dt)
            sim.sync()
        sim.profile(True)
        dist.barrier()
        torch.cuda.synchronize()
        if name == cases[-1][0]:
            clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        segs = 0
        ev0.record(stream)
        for _ in range(args.steps):
            sim.reset()
            for _ in range(prob.nsteps):
                sim.step(prob.dt)
            segs += sim.counts()["segments_total"]
        ev1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        if name == cases[-1][0]:
            clk = clocks.stop()
        kms, klaunch, _ = sim.kernel_times()
        sim.profile(False)
        sim.close()
        ms = dist.max(ev0.elapsed_time(ev1)) / args.steps
        results[name] = {"ms_per_sim": ms, "segments_per_sim": segs / args.steps,
                         "segments_per_s": segs / args.steps / (ms * 1e-3), "live_rays_at_end": max_rays,
                         "kernel_ms_per_sim": {k: float(v) / args.steps for k, v in kms.items()}}
    plain = results["plain"]
    for name, _ in cases[1:]:
        r = results[name]
        r["speedup_vs_plain"] = plain["ms_per_sim"] / r["ms_per_sim"]
        rel = np.abs(traces[name] / traces["plain"] - 1.0)[2:]    # from the third sample, when Gamma > 0
        r["max_dev"] = {"x_volume": float(rel[:, 0].max()), "x_mass": float(rel[:, 1].max()),
                        "gamma": float(rel[:, 2].max())}
    best = cases[-1][0]
    if dist.rank == 0:
        line = {"metric": "sims/hour", "value": 3600.0e3 / results[best]["ms_per_sim"] * dist.ws, "unit": "sims/hour",
                "n_gpus": dist.ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": results[best]["ms_per_sim"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "merge: " + WORKLOAD_DESC + "; ray merging as Sec. 7.1",
                           "cases": [c[0] for c in cases], "timed_case": best},
                "results": results, "clocks": clk,
                # per simulation: the cells' initialisation, then per RT step emission,
                # march, chemistry and the budget's commit plus the merge's eleven
                # launches (rotations, content histogram, two radix-select passes of
                # copy reduction and search, lower-bits histogram, group, weight,
                # placement scan, emit)
                "gpu_launches": args.steps * (1 + base.nsteps * (4 + 11))}
        print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="flexrt", choices=["flexrt", "reference"])
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--rt-steps", type=int, default=100)
    ap.add_argument("--capacity", type=int, default=200_000_000)
    ap.add_argument("--ref-budget", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and served measurements")
    ap.add_argument("--variant", default="", help="march launch agg,minb,blocks_per_sm (no autotuning)")
    ap.add_argument("--workload", default="cosmo16", choices=["cosmo16", "batch64", "serve", "merge"])
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=50)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--mean-gap", type=float, default=0.05)
    ap.add_argument("--hbm-budget", type=float, default=150e9)
    ap.add_argument("--saturate-gap", type=float, default=0.001)
    ap.add_argument("--merge-nex", type=float, nargs="+", default=[16.0, 4.0])
    ap.add_argument("--l-merge", type=int, default=0)
    ap.add_argument("--gamma-iters", type=int, default=1,
                    help="passes of the Gamma - <n_HI> iteration per RT step (1 = the plain step)")
    ap.add_argument("--problem", default="cosmo16", choices=["cosmo16", "cosmo20k"],
                    help="single-simulation workload of the default line")
    ap.add_argument("--gen-mode", action="store_true", help="Generalized Opacity mode (at least 4 passes)")
    args = ap.parse_args(argv)
    if args.workload == "merge" and args.impl != "reference":
        dist = Dist()
        impl_merge(args, dist)
        dist.close()
        return
    if args.workload == "batch64" and args.impl != "reference":
        dist = Dist()
        impl_batch(args, dist)
        dist.close()
        return
    if args.workload == "serve" and args.impl != "reference":
        dist = Dist()
        impl_serve(args, dist)
        dist.close()
        return
    if args.impl == "reference":
        dist = Dist(backend="gloo")
        impl_reference(args, dist)
    else:
        dist = Dist()
        impl_gpu(args, dist)
    dist.close()


if __name__ == "__main__":
    main()
