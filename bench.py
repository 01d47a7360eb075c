#!/usr/bin/env python3
"""Throughput of the full free-surface foaming step on GB300.

One step = the whole per-timestep sweep: interface mass exchange, fused
stream/collide/reconstruct/ADE, conversion with excess redistribution,
union-find bubble labelling, bubble table update (ideal gas), normals /
curvature / PLIC, disjoining pressure.

Workload: the 128^3 D3Q19 + D3Q7 case (FP32 storage, 8 bubbles, power-law
fluid, disjoining pressure on), seeded synthetic inputs.  Metric: MLUPS over
all lattice cells.  Populations (217 MB) exceed the 129 MB L2, so no flush
is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
The K steps are timed three times (each region exactly K steps, bracketed
by a barrier and a synchronise); the median is the reported value.
Under torchrun each rank runs an independent replica (the step has no
cross-GPU exchange); value = cells x steps of all ranks / max time.
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

METRIC = "MLUPS (D3Q19 FSLBM + D3Q7 ADE) and % HBM roofline; FP16+learned-κ vs FP32 plain"
WORKLOAD = "3D D3Q19 FSLBM + D3Q7 ADE, 128^3, FP32 storage, 8 bubbles (R 4-6), power-law n=0.6, disjoining on"
# label sync 1, exchange 1, sweep 2, conversion 4, labelling check, root scan and choice 3, union-find 4,
# relabel 1, label patch 1, bubble update 2, geometry 1, disjoining 1 (one of the two labelling branches
# returns at once)
KERNELS_PER_STEP = 21


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP16S + learned-curvature comparison")
    ap.add_argument("--config", default="default", choices=["default", "c1", "c3", "c5", "oracle"],
                    help="c1: 128^2 FP64 bubble, R(t) and Laplace jump; c3: 256^3 FP16S Carreau foam with the "
                         "learned curvature and its error; c5: 512x512x384 BF16S + learned curvature against FP32, "
                         "histograms; oracle: CPU oracle timings (single thread and all host cores)")
    args = ap.parse_args()
    args.steps_given = any(a == "--steps" or a.startswith("--steps=") for a in sys.argv[1:])
    return args


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region

def start_clocks(gpu: int):
    fd, path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except Exception:
        proc = None
    return proc, path


def stop_clocks(proc, path):
    if proc is not None:
        time.sleep(0.25)
        proc.terminate()
        try:
            proc.wait(timeout=5)
        except Exception:
            proc.kill()
    rows = []
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(path)
    except Exception:
        pass
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------

# DRAM bytes (read + write) per launch of the FP32 liquid sweep on this
# workload, mean of the two parities, from one ncu capture of
# k_stream_liquid<3,float> under this script's default run (dram__bytes_read.sum
# + dram__bytes_write.sum), valid while the sweep's sources are the ones that
# were profiled
SWEEP_TRAFFIC_BYTES = 264.1e6
SWEEP_SOURCES = ("paper_1908_04262_gb300/csrc/lbf_stream.cuh", "paper_1908_04262_gb300/csrc/lbf_common.cuh")
SWEEP_SOURCES_SHA256_16 = "a6b86d84b81863eb"


def sweep_traffic():
    import hashlib

    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return SWEEP_TRAFFIC_BYTES if h.hexdigest()[:16] == SWEEP_SOURCES_SHA256_16 else None


def algorithmic_bytes_sweep(counts, storage_bytes, Q=19, QA=7):
    """Bytes the liquid sweep must move in one launch: every liquid cell
    reads and writes its Q + QA populations once; every cell's flag byte is
    read."""
    gas, liq, ifc, wall = [float(x) for x in counts]
    N = gas + liq + ifc + wall
    return liq * 2 * (Q + QA) * storage_bytes + N * 1


def bubble_volume(b: dict) -> float:
    """Total volume of the bubbles (the atmosphere excluded)."""
    return float(sum(v for v, a in zip(b["volume"], b["atm"]) if not a))


REPEATS = 3  # timed regions of exactly K steps each; the median is reported


def timed_steps(sim, stream, steps: int, world: int = 1) -> list:
    """Device time (ms) of `steps` steps through lbf_step, REPEATS times:
    each region is bracketed by a barrier and a device synchronise on both
    sides and timed with CUDA events on the library's stream (max over
    ranks).  Every step graph shape was instantiated by the warm-up call."""
    import torch

    out = []
    for _ in range(REPEATS):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        out.append(reduce_max(e0.elapsed_time(e1), world))
    return out


def static_bubble_laplace(lbf, theta, storage: str, R: float = 5.0, steps: int = 1500, sigma: float = 0.01):
    """Relative error of the Laplace jump of a static bubble (48^3, periodic)
    against 2 sigma / R_eq after `steps` steps, mean of the last 4 samples."""
    import numpy as np

    from paper_1908_04262_gb300 import curvature

    n = 48
    sim = lbf.Sim(curvature.static_bubble_config(R, storage, sigma=sigma, n=n))
    c = [n / 2 + 0.31, n / 2 - 0.17, n / 2 + 0.23]
    sim.nucleate([c], [R])
    if theta is not None:
        sim.mlp_attach(theta)
    idx = np.arange(n ** 3)
    d = np.sqrt((idx % n - c[0]) ** 2 + ((idx // n) % n - c[1]) ** 2 + (idx // (n * n) - c[2]) ** 2)
    rel = []
    for _ in range(steps // 250):
        sim.step(250)
        b = sim.bubbles()
        f = sim.fields(["rho", "flags"])
        pl = f["rho"][((f["flags"] & 3) == 1) & (d > R + 4)].mean() / 3
        rel.append((b["pressure"][0] - pl) / (2 * sigma / np.cbrt(3 * b["volume"][0] / (4 * np.pi))) - 1)
    sim.close()
    return float(np.mean(rel[-4:]))


def crop_field_errors(lbf, steps: int = 20):
    """Per-field norm-relative errors of each storage form after `steps`
    steps of the 32^3 crop, against the FP64 CUDA form of the same crop
    (which the parity tests hold to the FP64 oracle within 1e-10): max |form
    - fp64| / max |fp64| over the cells liquid or interface in both."""
    import numpy as np

    from paper_1908_04262_gb300 import workloads as W

    names = ["rho", "u", "alpha", "mass", "conc"]
    got = {}
    for st in ("fp64", "fp32", "fp16s", "bf16s"):
        cfg, c, r = W.c2_crop_3d_32(storage=st)
        sim = lbf.Sim(cfg)
        sim.nucleate(c, r)
        sim.step(steps)
        got[st] = (sim.fields(names + ["flags"]), sim.bubbles()["volume"])
        sim.close()
    ref, vref = got["fp64"]
    out = {}
    for st in ("fp32", "fp16s", "bf16s"):
        g, v = got[st]
        both = ((g["flags"] == 1) | (g["flags"] == 2)) & ((ref["flags"] == 1) | (ref["flags"] == 2))
        e = {}
        for k in names:
            a, b = np.asarray(g[k], float)[both], np.asarray(ref[k], float)[both]
            e[k] = float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
        e["volume"] = float(np.max(np.abs(v - vref)) / np.max(np.abs(vref))) if len(v) == len(vref) else None
        e["flag_mismatches"] = int(np.sum(g["flags"] != ref["flags"]))
        out[st] = e
    return out


def forms_comparison(args, lbf, cfg, pts, rad, stream, fp32_line):
    """The same workload in shifted-FP16 storage with the learned curvature
    (and the two halves of that change alone) against FP32 with least
    squares; the network is trained first by the package's recipe."""
    import torch

    from paper_1908_04262_gb300 import curvature

    t0 = time.perf_counter()
    theta, info = curvature.train(seed=1, rounds=3, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    out = {"fp32_plain": fp32_line, "mlp_training_s": t_train, "mlp_training": info}
    N = cfg["nx"] * cfg["ny"] * cfg["nz"]
    for name, storage, use in (("fp16s_mlp", "fp16s", True), ("fp16s_plain", "fp16s", False),
                               ("fp32_mlp", "fp32", True)):
        sim = lbf.Sim(dict(cfg, storage=storage), stream=stream.cuda_stream)
        sim.nucleate(pts, rad)
        if use:
            sim.mlp_attach(theta)
        sim.step(args.warmup)
        reps = timed_steps(sim, stream, args.steps)
        ms = statistics.median(reps)
        V = bubble_volume(sim.bubbles())
        out[name] = {"mlups": N * args.steps / (ms / 1e3) / 1e6, "ms_per_step": ms / args.steps,
                     "repeats_ms_per_step": [r / args.steps for r in reps],
                     "bubble_volume_rel_diff_vs_fp32_plain": V / fp32_line["bubble_volume"] - 1}
        sim.close()
    # the collision variants of Sec. 2 on the same workload (FP32, least
    # squares): two relaxation times, and multiple relaxation times at the
    # rates d'Humieres et al. suggest for D3Q19 (energy 1.19, energy square
    # and fourth order 1.4, third order 1.98; the energy flux at the TRT rate)
    out["collisions"] = {}
    for name, coll, rates in (("fp32_trt", 1, (0.0, 0.0, 0.0, 0.0)), ("fp32_mrt", 2, (1.19, 1.4, 1.4, 1.98))):
        sim = lbf.Sim(dict(cfg, collision=coll, trt_magic=3.0 / 16.0, mrt_rates=rates), stream=stream.cuda_stream)
        sim.nucleate(pts, rad)
        sim.step(args.warmup)
        reps = timed_steps(sim, stream, args.steps)
        ms = statistics.median(reps)
        out["collisions"][name] = {"mlups": N * args.steps / (ms / 1e3) / 1e6, "ms_per_step": ms / args.steps,
                                   "mrt_rates": list(rates) if coll == 2 else None}
        sim.close()
    out["laplace_rel_err_static_bubble_R5"] = {
        "fp32_plain": static_bubble_laplace(lbf, None, "fp32"),
        "fp16s_mlp": static_bubble_laplace(lbf, theta, "fp16s")}
    out["field_errors_vs_fp64_32cube_20steps"] = crop_field_errors(lbf)
    out["note"] = ("same workload, steps and warm-up as the headline; bubble volume = total over the "
                   "bubbles after warm-up + timed steps; Laplace error of a static R=5 bubble, 48^3; "
                   "field errors: 32^3 crop after 20 steps against the FP64 CUDA form")
    return out


def algorithmic_bytes_step(counts, storage_bytes, Q=19, QA=7):
    """Bytes one whole step must move by the per-step model: every liquid or
    interface cell reads and writes its populations once and its flag byte
    (base = 2 (Q + QA) s + 2); an interface cell adds its mass, velocity,
    curvature, disjoining pressure, normal and its own outgoing populations
    for the exchange (~120 B in the FP32 form); a gas cell adds its flag and
    label (9 B) for the labelling."""
    gas, liq, ifc, wall = [float(x) for x in counts]
    return (liq + ifc) * (2 * (Q + QA) * storage_bytes + 2) + ifc * 120.0 + gas * 9.0


def reduce_max(x: float, world: int) -> float:
    """The largest x over the ranks (the slowest rank's time); the tensor
    lives where the process group's backend reduces (NCCL: the GPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def host_cpu():
    """Core count and model string of the host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        import platform

        model = platform.processor() or platform.machine()
    return os.cpu_count() or 1, model


def _oracle_worker(cfg, pts, rad, steps, barrier, queue):
    """One oracle instance in its own process: build and nucleate, wait for
    every worker, then time `steps` steps (wall clock)."""
    sys.path.insert(0, ROOT)
    import oracle

    ora = oracle.OracleSim(cfg)
    ora.nucleate(pts, rad)
    barrier.wait()
    t0 = time.time()
    ora.step(steps)
    queue.put((t0, time.time()))


def cpu_baseline_oracle(cfg, pts, rad, steps=1, parallel=True):
    """The FP64 CPU oracle, as it stands (one thread per instance), on the
    same workload: single thread, then one instance per host core at once
    (processes started with spawn), each timing `steps` steps after its
    construction and nucleation."""
    import multiprocessing as mp

    import oracle

    N = cfg["nx"] * cfg["ny"] * cfg["nz"]
    ora = oracle.OracleSim(cfg)
    ora.nucleate(pts, rad)
    t0 = time.perf_counter()
    ora.step(steps)
    dt = time.perf_counter() - t0
    del ora
    ncores, model = host_cpu()
    single = N * steps / dt / 1e6
    out = {"value": single, "unit": "MLUPS", "cores": 1, "kind": "oracle", "nproc": ncores, "cpu_model": model,
           "sample": "%d full step(s) of the workload (%.1f s, one thread)" % (steps, dt)}
    if parallel and ncores > 1:
        workers = min(ncores, 16)
        ctx = mp.get_context("spawn")
        barrier, queue = ctx.Barrier(workers), ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker, args=(cfg, pts, rad, steps, barrier, queue)) for _ in range(workers)]
        for pr in procs:
            pr.start()
        spans = [queue.get() for _ in procs]
        for pr in procs:
            pr.join()
        wall = max(b for _, b in spans) - min(a for a, _ in spans)
        out["all_cores"] = {"value": workers * N * steps / wall / 1e6, "unit": "MLUPS", "cores": workers,
                            "sample": "%d concurrent single-thread instances, %d step(s) each, %.1f s wall"
                                      % (workers, steps, wall)}
    return out


def reference_sample_cfg():
    """Bounded sample of the workload for the oracle: the same physics on a
    48^3 lattice with one bubble (same seed); about 0.15 s per step on one
    core, so that a default run stays near a minute."""
    from paper_1908_04262_gb300 import workloads as W

    cfg, c, r = W.c2_crop_3d_32()
    n = 48
    cfg.update(nx=n, ny=n, nz=n, fill_height=0.75 * n)
    return cfg, [[24.0 + c[0][0] - 16.0, 24.0 + c[0][1] - 16.0, 18.0 + c[0][2] - 12.0]], list(r)


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle

    cfg, c, r = reference_sample_cfg()
    ora = oracle.OracleSim(cfg)
    ora.nucleate(c, r)
    ora.step(args.warmup)
    t0 = time.perf_counter()
    ora.step(args.steps)
    dt = time.perf_counter() - t0
    N = cfg["nx"] * cfg["ny"] * cfg["nz"]
    v = N * args.steps / dt / 1e6
    sample = "each step: one oracle step of the workload's physics on a 48^3 lattice with one bubble"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    from paper_1908_04262_gb300 import build as B

    if rank == 0:
        B.build()
    barrier(world)
    from paper_1908_04262_gb300 import lbf
    from paper_1908_04262_gb300 import workloads as W

    cfg, pts, rad = W.c2_3d_128_fp32()
    N = cfg["nx"] * cfg["ny"] * cfg["nz"]
    stream = torch.cuda.Stream()
    sim = lbf.Sim(cfg, stream=stream.cuda_stream)
    sim.nucleate(pts, rad)
    sim.step(args.warmup)
    counts0 = sim.cell_counts()

    # --- timed regions: device-resident state, CUDA-graph steps ----------
    clk = start_clocks(local_rank)
    reps = timed_steps(sim, stream, args.steps, world)
    clocks = stop_clocks(*clk)
    ms = statistics.median(reps)
    counts1 = sim.cell_counts()
    fp32_volume = bubble_volume(sim.bubbles())
    value = N * args.steps * world / (ms / 1e3) / 1e6

    # --- kernel timing (CUDA events around every kernel group) -----------
    kp = max(50, min(args.steps, 400))
    sim.timing_enable(True)
    ca = sim.cell_counts()
    sim.step(kp)
    groups = sim.timing_read()
    cb = sim.cell_counts()
    sim.timing_enable(False)
    sweep_ms, sweep_n = groups["stream_liquid"]
    avg_counts = (np.asarray(ca, float) + np.asarray(cb, float)) / 2
    bytes_sweep = algorithmic_bytes_sweep(avg_counts, 4)
    achieved = bytes_sweep / (sweep_ms / sweep_n / 1e3) / 1e9
    peak, peak_kind = peaks()
    total_ms = sum(v[0] for v in groups.values())
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": sweep_traffic(),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of "
                                  "k_stream_liquid<3,float> under python bench.py",
                "kernel": "k_stream_liquid<3,float> (liquid cells of the sweep)",
                "bytes_per_launch": bytes_sweep, "launch_ms": sweep_ms / sweep_n,
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                "sweep_share_of_step": sweep_ms / total_ms if total_ms > 0 else None}
    kernel_ms = {k: v[0] / max(v[1], 1) for k, v in groups.items()}
    step_bytes = algorithmic_bytes_step(np.asarray(counts1, float), 4)
    step_achieved = step_bytes / (ms / args.steps / 1e3) / 1e9 * world
    step_roofline = {"bound": "hbm", "achieved": step_achieved, "peak": peak, "unit": "GB/s",
                     "frac": step_achieved / (peak * world), "bytes_per_step": step_bytes,
                     "note": "whole step (all %d kernels) against the per-step byte model; "
                             "the step is latency- and instruction-bound outside the sweep" % KERNELS_PER_STEP}

    # --- end to end through the public API with host buffers -------------
    f = sim.fields(["flags", "rho", "u", "alpha", "conc"])
    pinned = {}
    for k, v in f.items():
        t = torch.empty(v.size, dtype=torch.uint8 if k == "flags" else torch.float64, pin_memory=True)
        t.numpy()[:] = v.reshape(-1).astype(np.uint8 if k == "flags" else np.float64)
        pinned[k] = t.numpy()
    h2d = N * (1 + 8 + 24 + 8 + 8)
    # page-locked result buffers, made before the timed region like the inputs
    res = {k: torch.empty(N, dtype=torch.int32 if k == "flags" else torch.float64, pin_memory=True).numpy()
           for k in ("rho", "alpha", "flags")}
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    sim.set_cells(pinned["flags"], pinned["rho"], pinned["u"], pinned["alpha"], pinned["conc"])
    nb_rows = 0
    for _ in range(args.steps):
        sim.step(1)
        nb_rows = len(sim.bubbles()["id"])
    out = sim.fields(["rho", "alpha", "flags"], out=res)
    torch.cuda.synchronize()
    t_e2e = reduce_max(time.perf_counter() - t0, world)
    e2e = {"value": N * args.steps * world / t_e2e / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / args.steps,
           "d2h_bytes_per_step": 16 + 40 * max(64, nb_rows) + N * (8 + 8 + 4) / args.steps,
           "note": "lbf_set_cells from pinned host arrays, then per step lbf_step(1) + lbf_bubbles "
                   "(one packed copy of the header and the first 64 rows; %d live rows), then lbf_fields(rho, alpha, flags) "
                   "into page-locked host arrays"
                   % nb_rows}
    del out

    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "repeats_ms_per_step": [r / args.steps for r in reps],
            "repeat_spread": (max(reps) - min(reps)) / ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": N, "seed": W.DEFAULT_SEED,
                       "l2": "inputs larger than L2: 217 MB of populations per replica",
                       "parallelism": "replicas x%d" % world,
                       "cells_gas_liquid_interface_wall": [int(x) for x in counts1]},
            "roofline": roofline, "kernel_ms": kernel_ms,
            "step_roofline": step_roofline,
            "fluid_mlups": (counts0[1] + counts0[2]) * args.steps * world / (ms / 1e3) / 1e6,
            "gpu_launches": KERNELS_PER_STEP * args.steps, "clocks": clocks, "e2e": e2e}
    if world == 1 and not args.no_forms:
        line["forms"] = forms_comparison(args, lbf, cfg, pts, rad, stream,
                                         {"mlups": value, "ms_per_step": ms / args.steps,
                                          "bubble_volume": fp32_volume})
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle(cfg, pts, rad)
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the paper-derived configurations (--config), one JSON line each


def _timed(sim, stream, steps):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def config_c1(args, lbf, W, stream):
    """128^2 D2Q9 FP64, free surface at y = 112, one bubble R = 8: the bubble
    radius against time and the Laplace jump p_g - p_l against sigma / R
    (2D), every 100 steps."""
    import numpy as np

    steps = args.steps if args.steps_given else 2000
    cfg, c, r = W.c1_2d_128_fp64()
    sim = lbf.Sim(cfg, stream=stream.cuda_stream)
    sim.nucleate(c, r)
    nx, ny = cfg["nx"], cfg["ny"]
    idx = np.arange(nx * ny)
    x, y = idx % nx, idx // nx
    rows, ms = [], 0.0
    for t in range(100, steps + 1, 100):
        ms += _timed(sim, stream, 100)
        b = sim.bubbles()
        k = int(np.flatnonzero(b["atm"] == 0)[0])
        R = float(np.sqrt(b["volume"][k] / np.pi))
        f = sim.fields(["rho", "flags"])
        far = (f["flags"] == 1) & (np.hypot(x - c[0][0], y - c[0][1]) > R + 6) & (y < 100)
        pl = float(f["rho"][far].mean() / 3.0)
        jump = float(b["pressure"][k] - pl)
        rows.append([t, R, jump, cfg["sigma"] / R, jump / (cfg["sigma"] / R)])
    sim.close()
    return {"config": "c1", "workload": "2D D2Q9 FSLBM + D2Q5 ADE, 128^2, FP64, one bubble R = 8, free surface y = 112",
            "metric": "MLUPS", "value": nx * ny * steps / (ms / 1e3) / 1e6, "unit": "MLUPS", "steps": steps,
            "note": "16,384 cells: launch-bound, no roofline claim",
            "R_t_and_laplace": {"columns": ["step", "R = sqrt(V/pi)", "p_g - p_l", "sigma / R", "ratio"], "rows": rows}}


def _kappa_errors(lbf, cfg, fields, vols, labels, theta):
    """Curvature of every interface cell of a state, by the least squares and
    by the learned network (the state set into fresh sims), against 1/R_eq of
    the cell's bubble (R_eq = (3V/4pi)^(1/3)); relative RMS over the cells of
    bubbles with R_eq in [2, 40]."""
    import numpy as np

    out = {}
    types = fields["flags"].astype(np.uint8)
    for name, th in (("least_squares", None), ("learned", theta)):
        s2 = lbf.Sim(cfg)
        if th is not None:
            s2.mlp_attach(th)
        s2.set_cells(types, fields["rho"], fields["u"].reshape(-1), fields["alpha"], fields["conc"])
        kap = s2.fields(["kappa"])["kappa"]
        s2.close()
        ifc = np.flatnonzero((types == 2) & (labels >= 0))
        R = np.cbrt(3.0 * vols[labels[ifc]] / (4.0 * np.pi))
        keep = (R >= 2.0) & (R <= 40.0)
        kt = 1.0 / R[keep]
        e = (kap[ifc][keep] - kt) / kt
        out[name] = {"rel_rms": float(np.sqrt(np.mean(e * e))), "cells": int(keep.sum())}
    return out


def config_c3(args, lbf, W, stream):
    """256^3 D3Q19 shifted FP16, Carreau, 200 nuclei appearing over the first
    5000 steps, with the learned curvature in the loop: MLUPS, the step
    roofline, and the curvature error of the final state against the bubbles'
    equivalent spheres, learned against least squares."""
    import numpy as np

    from paper_1908_04262_gb300 import curvature

    steps = args.steps if args.steps_given else 20000
    cfg, pts, rad, times = W.c3_3d_256_fp16s()
    theta, _ = curvature.train(seed=1, rounds=3, stream=stream.cuda_stream)
    sim = lbf.Sim(cfg, stream=stream.cuda_stream)
    sim.nucleate(pts, rad, times)
    sim.mlp_attach(theta)
    ms = _timed(sim, stream, steps)
    N = cfg["nx"] * cfg["ny"] * cfg["nz"]
    counts = np.asarray(sim.cell_counts(), float)
    f = sim.fields(["flags", "rho", "u", "alpha", "conc", "label"])
    b = sim.bubbles()
    peak, kind = peaks()
    step_bytes = algorithmic_bytes_step(counts, 2)
    out = {"config": "c3", "workload": "3D D3Q19 + D3Q7, 256^3, shifted FP16, Carreau n=0.5 lambda=50, "
                                       "200 nuclei (times U[0,5000]), learned curvature in the loop",
           "metric": "MLUPS", "value": N * steps / (ms / 1e3) / 1e6, "unit": "MLUPS", "steps": steps,
           "ms_per_step": ms / steps, "bubbles": int(np.sum(b["atm"] == 0)),
           "step_roofline": {"achieved": step_bytes / (ms / steps / 1e3) / 1e9, "peak": peak,
                             "frac": step_bytes / (ms / steps / 1e3) / 1e9 / peak, "unit": "GB/s",
                             "peak_source": kind + " hbm_gbs", "bytes_per_step": step_bytes}}
    vols = np.asarray(b["volume"])
    out["kappa_error_final_state"] = _kappa_errors(lbf, cfg, f, vols, np.asarray(f["label"]), theta)
    sim.close()
    return out


def _histograms(b):
    import numpy as np

    v = np.asarray(b["volume"])[np.asarray(b["atm"]) == 0]
    edges = [0, 10, 20, 40, 80, 160, 320, 640, 1280, 1e12]
    h, _ = np.histogram(v, bins=edges)
    return {"count": int(v.size), "volume_bin_edges": edges[:-1] + ["inf"], "volume_histogram": h.tolist(),
            "total_volume": float(v.sum())}


def config_c5(args, lbf, W, stream):
    """512x512x384 D3Q19 shifted BF16 with the learned curvature (least-squares
    fallback) against the plain FP32 form, same nuclei and steps: MLUPS, the
    step roofline, bubble count and volume histograms."""
    import numpy as np

    from paper_1908_04262_gb300 import curvature

    steps = args.steps if args.steps_given else 2000
    cfg, pts, rad = W.c5_3d_512x512x384_bf16s()
    theta, _ = curvature.train(seed=1, rounds=3, stream=stream.cuda_stream)
    N = cfg["nx"] * cfg["ny"] * cfg["nz"]
    peak, kind = peaks()
    out = {"config": "c5", "workload": "3D D3Q19 + D3Q7, 512x512x384, power law n=0.7, 2000 nuclei",
           "metric": "MLUPS", "unit": "MLUPS", "steps": steps, "forms": {}}
    for name, storage, use in (("bf16s_mlp", "bf16s", True), ("fp32_plain", "fp32", False)):
        sim = lbf.Sim(dict(cfg, storage=storage), stream=stream.cuda_stream)
        sim.nucleate(pts, rad)
        if use:
            sim.mlp_attach(theta)
        sim.step(5)
        ms = _timed(sim, stream, steps)
        counts = np.asarray(sim.cell_counts(), float)
        sb = 2 if storage == "bf16s" else 4
        step_bytes = algorithmic_bytes_step(counts, sb)
        ach = step_bytes / (ms / steps / 1e3) / 1e9
        out["forms"][name] = {"mlups": N * steps / (ms / 1e3) / 1e6, "ms_per_step": ms / steps,
                              "step_roofline": {"achieved": ach, "peak": peak, "frac": ach / peak, "unit": "GB/s",
                                                "peak_source": kind + " hbm_gbs"},
                              "bubbles": _histograms(sim.bubbles())}
        sim.close()
    out["value"] = out["forms"]["bf16s_mlp"]["mlups"]
    a, b = out["forms"]["bf16s_mlp"]["bubbles"], out["forms"]["fp32_plain"]["bubbles"]
    out["bf16s_mlp_vs_fp32_plain"] = {"count_diff": a["count"] - b["count"],
                                      "total_volume_rel_diff": a["total_volume"] / b["total_volume"] - 1}
    return out


def config_oracle(args):
    """The CPU oracle on the paper-derived cases (timings only): the 128^2
    case for 2000 steps (one thread), the 32^3 crop for 20 steps and a 128^3
    window of steps, each on one thread and on all host cores."""
    import oracle

    from paper_1908_04262_gb300 import workloads as W

    out = {"config": "oracle", "metric": "MLUPS", "unit": "MLUPS"}
    ncores, model = host_cpu()
    out["nproc"], out["cpu_model"] = ncores, model
    cfg, c, r = W.c1_2d_128_fp64()
    ora = oracle.OracleSim(cfg)
    ora.nucleate(c, r)
    t0 = time.perf_counter()
    ora.step(2000)
    dt = time.perf_counter() - t0
    out["c1_128sq_2000_steps"] = {"value": 128 * 128 * 2000 / dt / 1e6, "seconds": dt, "cores": 1}
    cfg, c, r = W.c2_crop_3d_32(storage="fp64")
    out["c2_crop_32cube_20_steps"] = cpu_baseline_oracle(cfg, c, r, steps=20)
    cfg, c, r = W.c2_3d_128_fp32()
    cfg = dict(cfg, storage="fp64")
    window = args.steps if args.steps_given else 5
    out["c2_128cube_window"] = cpu_baseline_oracle(cfg, c, r, steps=window)
    out["value"] = out["c2_128cube_window"]["value"]
    return out


def run_config(args):
    import torch

    torch.cuda.set_device(0)
    from paper_1908_04262_gb300 import build as B

    B.build()
    from paper_1908_04262_gb300 import lbf
    from paper_1908_04262_gb300 import workloads as W

    stream = torch.cuda.Stream()
    fn = {"c1": config_c1, "c3": config_c3, "c5": config_c5}[args.config]
    print(json.dumps(fn(args, lbf, W, stream)), flush=True)


def main():
    args = parse()
    if args.config == "oracle":
        print(json.dumps(config_oracle(args)), flush=True)
        return
    if args.config != "default":
        run_config(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
