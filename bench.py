#!/usr/bin/env python3
"""Benchmark of the OReg D2Q9 stream-collide path on GB300.

Default workload: one 8192 x 8192 periodic rotated shear wave (angle from
seed 0, theta = 1/3, tau = 0.6, u0 = 0.05), guided equilibrium, OReg
collision, FP32 storage and compute, A-B layout.  One "step" is one lattice
time step (gather, moments, equilibrium, OReg projection, relaxation, store);
the FP64 diagnostics reduction (mass, momentum, non-finite count) runs every
100 steps and after the last step, inside the timed region.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (bounded sample of the same workload).

Multi-GPU (torchrun, one rank per GPU): every rank advances its own
independent lattice (weak scaling, no data-path collective); the timing is
the max over ranks.  The CPU baseline and the extended sections (precision,
batched, serving, Mach sweep) run at N = 1 only.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
DIAG_EVERY = 100


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--side", type=int, default=8192)
    ap.add_argument("--theta", type=float, default=1.0 / 3.0)
    ap.add_argument("--storage", default="f32", choices=["f64", "f32", "f16", "bf16"])
    ap.add_argument("--layout", default="ab", choices=["ab", "aa"])
    ap.add_argument("--comp", type=int, default=None,
                    help="OLB_OPT_COMPENSATED for f32: exact conserved sums (library default: 1)")
    ap.add_argument("--warps", type=int, default=4, help="OLB_OPT_WARPS_PER_BLOCK")
    ap.add_argument("--sr", type=int, default=None,
                    help="OLB_OPT_STOCHASTIC_ROUNDING for f16/bf16 (library default: 1)")
    ap.add_argument("--f64-collision", type=int, default=0,
                    help="OLB_OPT_F64_COLLISION (FP32 storage, collision in FP64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extended", action="store_true",
                    help="skip the batched, serving and precision sections")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched section and print its JSON (profiling)")
    ap.add_argument("--batch-config", default=None,
                    help="layout,warps_per_block,blocks_per_sm,item_passes,steps_per_launch "
                         "instead of the autotuner (e.g. ab,2,0,2,100)")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--decay-samples", type=int, default=1000,
                    help="shear lattices of the batched mix whose decay-rate error is measured")
    ap.add_argument("--serve-count", type=int, default=300)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-side", type=int, default=1024)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


STEP_KERNEL_SOURCES = ("oreg_device.cuh", "oreg_kernels.cuh")


def kernel_source_hash() -> str:
    """Hash of the sources that define the stream-collide kernels."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2501_16000_gb300", "csrc")
    for name in STEP_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_key: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel_key]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return float(e["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(value: float, device="cpu") -> float:
    """Maximum of a per-rank value over all ranks (identity without a process
    group); the only collective the benchmark uses (timing, not data)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_mlups(world: int, nodes_per_rank: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: every rank advances its own lattice of
    nodes_per_rank nodes `steps` times; the slowest rank sets the time."""
    return world * nodes_per_rank * steps / (max_ms / 1e3) / 1e6


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(args):
    from paper_2501_16000_gb300 import workloads as W
    return W.large_shear(theta=args.theta, seed=0, side=args.side, steps=args.steps)


def cpu_baseline(args, case, seconds: float):
    """The FP64 oracle, as it stands, on the host cores: the same lattice
    parameters on a side x side periodic sample, stepped for ~seconds."""
    from oracle import oracle as O
    from paper_2501_16000_gb300 import workloads as W
    side = args.cpu_sample_side
    m, n, _ = W.wave_vector_from_angle(side, side, math.atan2(case.n / case.ny, case.m / case.nx))
    p = O.params(side, side, case.tau, case.theta, O.GUIDED, O.OREG)
    f = O.init_equilibrium(p, *W.shear_wave_fields(side, side, 1.0, case.u0, m, n))
    threads = O.get_threads()
    f = O.run(f, p, 1)  # warm-up
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        f = O.run(f, p, 2)
        steps += 2
    dt = time.perf_counter() - t0
    mlups = side * side * steps / dt / 1e6
    # the same oracle on one core, on a quarter-side sample for ~seconds / 3
    side1 = max(64, side // 4)
    m1, n1, _ = W.wave_vector_from_angle(side1, side1, math.atan2(case.n / case.ny, case.m / case.nx))
    p1 = O.params(side1, side1, case.tau, case.theta, O.GUIDED, O.OREG)
    f1 = O.init_equilibrium(p1, *W.shear_wave_fields(side1, side1, 1.0, case.u0, m1, n1))
    O.set_threads(1)
    try:
        f1 = O.run(f1, p1, 1)
        steps1, t1 = 0, time.perf_counter()
        while time.perf_counter() - t1 < seconds / 3:
            f1 = O.run(f1, p1, 2)
            steps1 += 2
        dt1 = time.perf_counter() - t1
    finally:
        O.set_threads(threads)
    return {"value": round(mlups, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"{side}x{side} periodic shear wave, same tau/theta/u0, {steps} FP64 "
                      f"steps in {dt:.1f} s, OpenMP over rows ({threads} threads)",
            "single_thread": {"value": round(side1 * side1 * steps1 / dt1 / 1e6, 3),
                              "unit": "MLUPS", "cores": 1,
                              "sample": f"{side1}x{side1}, {steps1} FP64 steps in {dt1:.1f} s"}}


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, rank 0 only."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2501_16000_gb300 import workloads as W
    case = workload(args)
    side = args.cpu_sample_side
    m, n, _ = W.wave_vector_from_angle(side, side, math.atan2(case.n / case.ny, case.m / case.nx))
    p = O.params(side, side, case.tau, case.theta, O.GUIDED, O.OREG)
    f = O.init_equilibrium(p, *W.shear_wave_fields(side, side, 1.0, case.u0, m, n))
    threads = O.get_threads()
    # each benchmark step = one oracle lattice step on the sample; the sample
    # shrinks if needed so that warm-up + steps stay within a few minutes
    f = O.run(f, p, 1)
    t0 = time.perf_counter()
    f = O.run(f, p, 2)
    per_step = (time.perf_counter() - t0) / 2
    budget = 150.0
    total = args.warmup + args.steps
    while per_step * total > budget and side > 64:
        side //= 2
        per_step /= 4
        m, n, _ = W.wave_vector_from_angle(side, side, math.atan2(case.n / case.ny, case.m / case.nx))
        p = O.params(side, side, case.tau, case.theta, O.GUIDED, O.OREG)
        f = O.init_equilibrium(p, *W.shear_wave_fields(side, side, 1.0, case.u0, m, n))
    f = O.run(f, p, args.warmup)
    t0 = time.perf_counter()
    f = O.run(f, p, args.steps)
    dt = time.perf_counter() - t0
    mlups = side * side * args.steps / dt / 1e6
    sample = (f"{side}x{side} periodic sample of the {case.nx}x{case.ny} shear wave "
              f"(same tau/theta/u0), FP64 oracle, {threads} OpenMP threads")
    line = {
        "impl": "reference", "metric": "MLUPS", "value": round(mlups, 3), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"shear{case.nx}x{case.ny}-oreg-guided-{args.layout}",
                   "nodes": case.nodes, "theta": case.theta, "tau": case.tau, "u0": case.u0,
                   "wave": [case.m, case.n], "sample": sample},
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_native(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2501_16000_gb300 import build
    build.build()
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.engine import Lattice, bytes_per_node_step

    case = workload(args)
    N = case.nodes
    stream = torch.cuda.Stream()
    lat = Lattice(case.nx, case.ny, case.tau, case.theta, "guided", "oreg", args.storage,
                  args.layout, stream=stream)
    if args.comp is not None:
        lat.set_option(B.OLB_OPT_COMPENSATED, args.comp)
    lat.set_option(B.OLB_OPT_WARPS_PER_BLOCK, args.warps)
    if args.sr is not None:
        lat.set_option(B.OLB_OPT_STOCHASTIC_ROUNDING, args.sr)
    if args.f64_collision:
        lat.set_option(B.OLB_OPT_F64_COLLISION, args.f64_collision)
    lat.init_case(case)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    # warm-up
    with torch.cuda.stream(stream):
        lat.step(args.warmup)
        lat.diagnostics()
    barrier()

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for s in range(K):
            ev[s][0].record(stream)
            lat.step(1)
            ev[s][1].record(stream)
            launches += 1
            if (s + 1) % DIAG_EVERY == 0 or s + 1 == K:
                d = lat.diagnostics()          # FP64 mass/momentum/non-finite check
                launches += 2
                if d["nonfinite"]:
                    raise RuntimeError("non-finite populations")
        t_end.record(stream)
    barrier()
    clocks = sampler.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    kern_ms = sum(a.elapsed_time(b) for a, b in ev) / K
    elapsed_ms = max_over_ranks(elapsed_ms, "cuda")
    mlups = weak_scaling_mlups(world, N, K, elapsed_ms)

    bpn = bytes_per_node_step(args.storage)
    peak, peak_kind = measured_peaks()
    achieved = bpn * N / (kern_ms / 1e3) / 1e9
    kernel_key = (f"step_{args.layout}_{args.storage}{'_c64' if args.f64_collision else ''}"
                  f"_guided_oreg_{case.nx}x{case.ny}")
    traffic = profiled_traffic(kernel_key)

    # end to end through the public API: host fields (pinned) in, moments out
    e2e, e2e_500 = None, None
    if not args.no_e2e:
        h = [torch.empty((case.ny, case.nx), dtype=torch.float64, pin_memory=True)
             for _ in range(6)]
        rho, ux, uy = case.fields()
        h[0].numpy()[:] = rho
        h[1].numpy()[:] = ux
        h[2].numpy()[:] = uy
        outs = [a.numpy().ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in h[3:6]]
        # untimed warm-up solve: the library's staging scratch is allocated on
        # first use
        lat.init_fields(h[0].numpy(), h[1].numpy(), h[2].numpy())
        lat.step(2)
        B.call("olb_moments", lat.handle, *outs, None)
        barrier()

        def solve(k):
            barrier()
            t0 = time.perf_counter()
            lat.init_fields(h[0].numpy(), h[1].numpy(), h[2].numpy())   # waits for its copies
            t1 = time.perf_counter()
            lat.step(k)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            B.call("olb_moments", lat.handle, *outs, None)
            barrier()
            t3 = time.perf_counter()
            secs = max_over_ranks(t3 - t0, "cuda")
            return {"value": round(world * N * k / secs / 1e6, 1), "unit": "MLUPS",
                    "h2d_bytes_per_step": int(3 * N * 8 / k),
                    "d2h_bytes_per_step": int(3 * N * 8 / k), "steps": k,
                    "note": f"one solve of {k} steps: olb_init_fields from pinned host "
                            f"fields ({3 * N * 8 / 1e9:.2f} GB), olb_step, olb_moments to "
                            f"pinned host arrays ({3 * N * 8 / 1e9:.2f} GB)",
                    "phases_ms": {"init_fields": round((t1 - t0) * 1e3, 1),
                                  "steps": round((t2 - t1) * 1e3, 1),
                                  "moments": round((t3 - t2) * 1e3, 1)}}
        e2e = solve(K)
        if K != 500:
            e2e_500 = solve(500)
    lat.close()
    extra = {}
    # the extended sections and the CPU baseline are single-GPU measurements:
    # at N > 1 they are left out, so that the other GPUs are not held meanwhile
    if rank == 0 and world == 1 and not args.no_extended:
        extra["precision_vs_fp64"] = precision_section(args)
        extra["batched"] = batched_section(args)
        extra["serving"] = serving_section(args, extra["batched"])
        extra["mach_sweep"] = mach_sweep_section()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, case, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": "MLUPS", "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": round(elapsed_ms / K, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.storage, "data": "synthetic",
            "config": {"workload": f"shear{case.nx}x{case.ny}-oreg-guided-{args.layout}",
                       "nodes": N, "theta": case.theta, "tau": case.tau, "u0": case.u0,
                       "wave": [case.m, case.n], "storage": args.storage,
                       "layout": args.layout,
                       "diagnostics": f"FP64 mass/momentum/non-finite check every {DIAG_EVERY} "
                                      f"steps and after the last, inside the timed region",
                       "exact_conserved_sums": (args.comp if args.comp is not None else
                                                int(args.storage == "f32")),
                       "warps_per_block": args.warps,
                       "collision": "f64" if args.f64_collision else
                                    ("f64" if args.storage == "f64" else "f32"),
                       "stochastic_rounding": (args.sr if args.sr is not None else
                                               int(args.storage in ("f16", "bf16"))),
                       "l2": f"inputs larger than L2 ({lat_bytes(args.storage, N) / 1e9:.1f} GB "
                             f"state vs 126 MB L2)"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": traffic, "peak_kind": peak_kind,
                         "bytes_per_node": bpn, "kernel_ms": round(kern_ms, 4)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "e2e_at_500_steps": e2e_500 if e2e_500 is not None else e2e,
            "clocks": clocks,
            "gpu_launches": launches,
            **extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _timed_batch_solve(groups, tuned, steps):
    """Wall seconds of one solve of `steps` steps of every lattice, the cases
    of each storage format in its own BatchEngine (own stream), the engines'
    rounds enqueued side by side; a warm-up solve (graph capture) first, and
    states created and initialised outside the timed region."""
    import torch
    from paper_2501_16000_gb300.batch import BatchEngine, work_items
    K, R = tuned["steps_per_launch"], tuned["item_passes"]
    engines = []
    for storage, cases in groups.items():
        if cases:
            items = sum(work_items(c.nx, c.ny, storage, R) for c in cases)
            engines.append((BatchEngine(storage, tuned["layout"], max_lattices=len(cases),
                                        max_items=items, steps_per_launch=K,
                                        warps_per_block=tuned["warps_per_block"],
                                        blocks_per_sm=tuned["blocks_per_sm"],
                                        item_passes=R), cases))
    try:
        for rep in range(2):
            lats = []
            for eng, cases in engines:
                for c in cases:
                    lat = eng.new_lattice(c)
                    eng.add(lat, steps)
                    lats.append(lat)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range((steps + K - 1) // K):
                for eng, _ in engines:
                    eng.run(1)
            for eng, _ in engines:
                eng.wait()
            dt = time.perf_counter() - t0
            for lat in lats:
                lat.close()
    finally:
        for eng, _ in engines:
            eng.close()
    return dt


def batched_section(args):
    """Batched workload: 512 independent uneven lattices (shear waves and shock
    tubes), FP16 storage (stochastic rounding) / FP32 compute, autotuned batch
    (layout, block shape, grid, warp passes per work item, steps per CUDA-graph
    replay).  Timed twice: every lattice in FP16, and with precision routing
    (shear waves whose decay rate FP16 cannot resolve to 1e-4 run in an FP32
    batch beside the FP16 one); against serial plain FP32 single-lattice
    solves of the same set.  Decay-rate error against FP64 for every shear
    lattice of the mix, in FP16 and in the routed format."""
    import numpy as np
    import torch
    from paper_2501_16000_gb300 import workloads as W
    from paper_2501_16000_gb300.analysis import measure_decay
    from paper_2501_16000_gb300.batch import autotune, kernel_classes, route_storage
    from paper_2501_16000_gb300.engine import Lattice
    steps = args.batch_steps
    cases = W.batch_mix(count=args.batch_count, seed=1, steps=steps)
    nodes = sum(c.nodes for c in cases)
    t_tune = time.perf_counter()
    if args.batch_config:
        lay, w, b, r, k = args.batch_config.split(",")
        tuned = {"layout": lay, "warps_per_block": int(w), "blocks_per_sm": int(b),
                 "item_passes": int(r), "steps_per_launch": int(k), "given": True}
    else:
        tuned = autotune(cases, "f16", use_cache=False)
    t_tune = time.perf_counter() - t_tune
    K = tuned["steps_per_launch"]
    dt = _timed_batch_solve({"f16": cases}, tuned, steps)
    # the same lattices over six kernel / constant classes (slots), tuned anew
    classes = W.batch_mix_classes(count=args.batch_count, seed=1, steps=steps)
    tuned_cls = tuned if args.batch_config else autotune(classes, "f16", use_cache=False)
    dt_cls = _timed_batch_solve({"f16": classes}, tuned_cls, steps)
    route = [route_storage(c, "f16") for c in cases]
    routed = {"f16": [c for c, r in zip(cases, route) if r == "f16"],
              "f32": [c for c, r in zip(cases, route) if r == "f32"]}
    dt_routed = _timed_batch_solve(routed, tuned, steps)
    # serial plain FP32: the same lattices one after another (states created
    # and initialised outside the timed region, as for the batch)
    ser = [Lattice(c.nx, c.ny, c.tau, c.theta, c.eq, c.coll, "f32", "ab") for c in cases]
    for lat, c in zip(ser, cases):
        lat.init_case(c)
    ser[0].step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for lat in ser:
        lat.step(steps)
    torch.cuda.synchronize()
    dt_ser = time.perf_counter() - t0
    for lat in ser:
        lat.close()
    # decay-rate error against FP64 of the shear lattices of the mix (single-
    # lattice runs: batched results are bitwise those of the lattice alone)
    shear = [c for c in cases if c.case == "shear"][: args.decay_samples]
    err16, err_routed = [], []
    for c in shear:
        g = {}
        for st in ("f64", "f16", "f32") if route_storage(c, "f16") == "f32" else ("f64", "f16"):
            with Lattice(c.nx, c.ny, c.tau, c.theta, storage=st, layout="ab") as lat:
                lat.init_case(c)
                g[st] = measure_decay(lat, c, steps, every=20)[0]
        err16.append(abs(g["f16"] / g["f64"] - 1))
        err_routed.append(abs(g[route_storage(c, "f16")] / g["f64"] - 1))

    def stats(e):
        e = np.array(e)
        if not len(e):
            return None
        return {"cases": len(e), "max": float(f"{e.max():.3e}"),
                "median": float(f"{np.median(e):.3e}"), "le_1e-4": int((e <= 1e-4).sum())}

    r32 = routed["f32"]
    peak, peak_kind = measured_peaks()
    gbs = nodes * steps * 36 / dt / 1e9                      # FP16: 9 reads + 9 writes x 2 B
    return {
        "workload": f"{len(cases)} lattices, sides log-uniform [32,1024] (seed 1), tau U[0.51,1], "
                    f"u0 U[0.01,0.1], shear/shock 50/50, {steps} steps each, FP16 storage "
                    f"(stochastic rounding) / FP32 compute, graph replay per {K} steps",
        "nodes": nodes, "solves_per_s": round(len(cases) / dt, 2), "seconds": round(dt, 4),
        "mlups": round(nodes * steps / dt / 1e6, 1), "tuned": tuned,
        "roofline": {"bound": "hbm", "bytes_per_node": 36, "achieved": round(gbs, 1),
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(gbs / peak, 4),
                     "note": "whole solve (wall clock, graph replays included) x 36 B per node-step"},
        "tune_seconds": round(t_tune, 1),
        "six_classes": {"workload": "the same lattices, BGK for odd j, polynomial equilibrium for odd "
                                    "j // 2, else guided at theta 0.36 / 0.30 (workloads.batch_mix_classes)",
                        "slots": kernel_classes(classes),
                        "solves_per_s": round(len(classes) / dt_cls, 2),
                        "mlups": round(nodes * steps / dt_cls / 1e6, 1), "tuned": tuned_cls},
        "routed": {"rule": "shear waves with 1/(u0 sqrt(N) gamma T) > 0.12 in FP32 storage",
                   "fp32_lattices": len(r32),
                   "fp32_node_fraction": round(sum(c.nodes for c in r32) / nodes, 4),
                   "solves_per_s": round(len(cases) / dt_routed, 2),
                   "seconds": round(dt_routed, 4),
                   "mlups": round(nodes * steps / dt_routed / 1e6, 1),
                   "speedup_vs_fp32_serial": round(dt_ser / dt_routed, 2),
                   "decay_rate_error_vs_fp64": stats(err_routed)},
        "baseline_fp32_serial": {"solves_per_s": round(len(cases) / dt_ser, 2),
                                 "seconds": round(dt_ser, 4),
                                 "mlups": round(nodes * steps / dt_ser / 1e6, 1)},
        "speedup_vs_fp32_serial": round(dt_ser / dt, 2),
        "decay_rate_error_vs_fp64": stats(err16),
    }


def serving_section(args, batched):
    """Serving workload: Poisson arrivals at ~80% of the measured batched capacity,
    sides 64..2048, steps 100..10000, continuous batching (FP16, stochastic
    rounding, the tuned batch configuration), three runs of the same trace:
    a 120 GB admission budget (not binding), a budget of half that run's peak
    (binding: requests wait for memory), and every request arriving at once
    (saturation: the server's own throughput against the batched MLUPS); vs
    serial FP32 solves of the trace."""
    import numpy as np
    from paper_2501_16000_gb300 import workloads as W
    from paper_2501_16000_gb300.serve import Server, serve_serial, summarize
    unit = W.arrival_trace(args.serve_count, rate_per_s=1.0, seed=2)
    mean_work = float(np.mean([r.lattice.nodes * r.lattice.steps for r in unit]))
    capacity = batched["mlups"] * 1e6 / mean_work            # requests per second
    rate = 0.8 * capacity
    tuned = batched["tuned"]

    def serve(budget, time_scale, label):
        srv = Server("f16", tuned["layout"], budget_bytes=budget,
                     steps_per_launch=tuned["steps_per_launch"],
                     warps_per_block=tuned["warps_per_block"],
                     blocks_per_sm=tuned["blocks_per_sm"],
                     item_passes=tuned["item_passes"])
        res, wall = srv.run(unit, time_scale=time_scale)
        stats = summarize(res, wall, label)
        stats.update({"budget_gb": round(budget / 1e9, 3), "rounds": srv.rounds,
                      "peak_inflight": srv.peak_inflight,
                      "peak_gb": round(srv.peak_bytes / 1e9, 3)})
        srv.close()
        return stats

    free = serve(120e9, 1.0 / rate, "continuous batching, FP16, 120 GB budget")
    binding = serve(0.5 * free["peak_gb"] * 1e9, 1.0 / rate,
                    "continuous batching, FP16, budget = half the unconstrained peak")
    saturated = serve(120e9, 0.0, "continuous batching, FP16, all requests at t = 0")
    saturated["vs_batched_mlups"] = round(saturated["mlups"] / batched["mlups"], 3)
    sres, swall = serve_serial(unit, "f32", "ab", time_scale=1.0 / rate)
    return {"requests": len(unit), "rate_per_s": round(rate, 2),
            "capacity_estimate_per_s": round(capacity, 2),
            "served": free, "served_binding_budget": binding, "served_saturated": saturated,
            "baseline_fp32_serial": summarize(sres, swall, "serial FP32")}


def precision_section(args):
    """Error of each reduced-precision storage against the FP64 GPU run
    (itself matched to the FP64 oracle by the parity tests) on a periodic
    shear wave, max |f - f64| / max |f64| over all populations."""
    import numpy as np
    from paper_2501_16000_gb300 import workloads as W
    from paper_2501_16000_gb300.engine import Lattice
    side, steps = 1024, 500
    c = W.large_shear(theta=1.0 / 3.0, seed=0, side=side, steps=steps)
    f = {}
    for st in ("f64", "f32", "f16", "bf16"):
        with Lattice(c.nx, c.ny, c.tau, c.theta, storage=st, layout="ab") as lat:
            lat.init_case(c)
            lat.step(steps)
            f[st] = lat.populations()
    den = np.abs(f["f64"]).max()
    return {"workload": f"{side}x{side} shear wave, tau={c.tau}, {steps} steps",
            **{st: float(f"{np.abs(f[st] - f['f64']).max() / den:.3e}") for st in ("f32", "f16", "bf16")}}


def mach_sweep_section():
    """nu~/nu of the decaying shear wave on a mean flow u_y = Ma sqrt(theta)
    (Sec. IV, Fig. 2): wavelength 200, nu = 0.01 (tau = 0.53), amplitude 1e-3,
    FP64 storage, first-order start (Eq. 5), 20000 steps per lattice."""
    from paper_2501_16000_gb300 import analysis
    t0 = time.perf_counter()
    rows = analysis.mach_sweep(machs=(0.0, 0.1, 0.2, 0.3, 0.4), length=200, steps=20000,
                               every=200)
    out = {"workload": "axis: 4x200, k along y; diagonal: 283x283, k along (-1, 1); "
                       "mean flow (0, Ma sqrt(1/3)); nu = 0.01; f64; 20000 steps",
           "wall_s": round(time.perf_counter() - t0, 2)}
    for r in rows:
        g, ma = r["geometry"], f"{r['mach']:.1f}"
        unstable = r.get("unstable", False)
        out.setdefault(g + "_nu_ratio", {}).setdefault(ma, {})[r["coll"]] = (
            "unstable" if unstable else round(r["nu_ratio"], 5))
        if r["mach"] > 0 and not unstable:
            out.setdefault(g + "_phase_rate_over_Uk", {}).setdefault(ma, {})[r["coll"]] = round(
                r["omega"] / r["omega_advect"], 5)
    return out


def lat_bytes(storage, N):
    from paper_2501_16000_gb300.engine import ELEM_BYTES
    return 2 * 9 * N * ELEM_BYTES[storage]


def main():
    args = parse_args()
    if args.batched_only:
        from paper_2501_16000_gb300 import build
        build.build()
        print(json.dumps(batched_section(args)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
