"""Batched path: many independent lattices in one launch per step (and slot),
steps_per_launch steps per CUDA-graph replay (C ABI ``olb_batch_*``).

``BatchEngine`` owns the batch and a torch stream; its lattices are created on
that stream with torch-allocated population memory.  ``autotune`` picks the
layout, warps per block, grid size, warp passes per work item and
steps per graph replay for a workload by timing graph replays, and caches the
choice per (ABI, storage, size class).
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import statistics
import time

from . import binding as B
from .engine import LAYOUT, STORAGE, Lattice

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


ITEM_PASSES = 4   # the library's default warp passes per work item


def warp_passes(nx: int, ny: int, v: int) -> int:
    """Warp passes over a lattice, as the library makes them: 32 consecutive
    vectors of v nodes each of the row-major planes, whose rows hold nx
    rounded up to v nodes, back to back."""
    return math.ceil(math.ceil(nx / v) * ny / 32)


def work_items(nx: int, ny: int, storage: str, passes: int = ITEM_PASSES) -> int:
    """Warp work items of one lattice: up to `passes` consecutive warp passes
    (``warp_passes``) each."""
    v = 16 // {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[storage]
    return math.ceil(warp_passes(nx, ny, v) / passes)


class BatchEngine:
    def __init__(self, storage="f16", layout="ab", max_lattices=1024, max_items=1 << 22,
                 steps_per_launch=100, warps_per_block=4, blocks_per_sm=0, stream=None,
                 item_passes=ITEM_PASSES):
        import torch
        self.storage, self.layout = storage, layout
        self.steps_per_launch = int(steps_per_launch)
        self.item_passes = int(item_passes)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.params = B.olb_batch_params(STORAGE[storage], LAYOUT[layout], int(max_lattices),
                                         int(max_items), int(steps_per_launch),
                                         int(warps_per_block), int(blocks_per_sm),
                                         self.stream.cuda_stream, int(item_passes))
        h = ctypes.c_void_p()
        B.check(B.load().olb_batch_create(ctypes.byref(self.params), ctypes.byref(h)),
                "olb_batch_create")
        self._h = h
        self.members: list[Lattice] = []

    # -- membership ---------------------------------------------------------
    def new_lattice(self, case, **kw) -> Lattice:
        """A lattice of a ``workloads.LatticeCase`` on this batch's stream,
        initialised (not yet added)."""
        lat = Lattice(case.nx, case.ny, case.tau, case.theta, case.eq, case.coll, self.storage,
                      self.layout, torch_memory=True, stream=self.stream,
                      boundary=case.boundary, theta_mode=case.theta_mode, **kw)
        lat.init_case(case)
        return lat

    def add(self, lat: Lattice, nsteps: int) -> None:
        B.call("olb_batch_add", self._h, lat.handle, int(nsteps))
        self.members.append(lat)

    def remove(self, lat: Lattice) -> None:
        B.call("olb_batch_remove", self._h, lat.handle)
        self.members.remove(lat)

    def remaining(self, lat: Lattice) -> int:
        r = ctypes.c_int64()
        B.call("olb_batch_remaining", self._h, lat.handle, ctypes.byref(r))
        return r.value

    @property
    def size(self) -> int:
        return int(B.load().olb_batch_size(self._h))

    @property
    def items(self) -> int:
        return int(B.load().olb_batch_work_items(self._h))

    # -- execution ----------------------------------------------------------
    def run(self, nrounds: int = 1) -> None:
        """Enqueues nrounds graph replays (asynchronous)."""
        B.call("olb_batch_run", self._h, int(nrounds))

    def record_event(self):
        """A torch CUDA event recorded on the batch's stream after the work
        enqueued so far (its ``synchronize()`` waits for it)."""
        import torch
        ev = torch.cuda.Event()
        ev.record(self.stream)
        return ev

    def side_stream(self):
        """A new torch stream for work beside the batch's (read-backs)."""
        import torch
        return torch.cuda.Stream()

    def read_back(self, lat: Lattice, after, stream, keep_fields: bool = True):
        """Reads a lattice that left the batch back on `stream` once the
        batch's work up to the event `after` has run (see
        ``Lattice.read_back_on``); blocks the calling thread only."""
        stream.wait_event(after)
        return lat.read_back_on(stream, keep_fields)

    def wait(self, timeout: float | None = None) -> bool:
        """Waits for the enqueued rounds: without a timeout until they have
        finished; with one at most `timeout` seconds, returning False if they
        are still running then (nothing is cancelled)."""
        if timeout is None:
            B.call("olb_batch_wait", self._h)
            return True
        st = B.load().olb_batch_wait_for(self._h, float(timeout))
        if st == B.OLB_ERR_TIMEOUT:
            return False
        B.check(st, "olb_batch_wait_for")
        return True

    def close(self) -> None:
        if self._h is not None:
            st = B.load().olb_batch_destroy(self._h)
            self._h = None
            B.check(st, "olb_batch_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# Precision routing.  A half-precision batch rounds the stored populations
# stochastically: unbiased, but each step adds noise of ~2^-11 of the shifted
# populations.  The decay rate of a shear wave is fitted from the mode
# amplitude, an average over the N nodes of the wave's velocity, so the noise
# reaching the fit scales as 1 / (u0 sqrt(N)) against a signal, the decay over
# the fitted steps T, of gamma T (gamma = theta (tau - 1/2) |k|^2, Eq. 14a).
# The measured FP16 decay-rate error of the batched workload's shear lattices
# grows as ~1.1e-4 x ratio^0.77 with ratio = 1 / (u0 sqrt(N) gamma T); at
# ratio <= 0.12 none of the 262 exceeded 1e-4 (the largest 9.7e-5), above it
# a fifth did.  Such lattices run in FP32 storage instead (exact conserved
# sums, within 1e-4 of FP64 on 261 of the 262).
FP16_NOISE_LIMIT = 0.12


def half_noise_ratio(case, steps=None) -> float:
    """1 / (u0 sqrt(N) gamma T) of a shear-wave case (0 for other cases):
    the half formats' rounding noise against the decay the rate fit sees, T
    the steps after the start-up transient the fit skips."""
    if case.case != "shear":
        return 0.0
    steps = case.steps if steps is None else steps
    k2 = (2 * math.pi * case.m / case.nx) ** 2 + (2 * math.pi * case.n / case.ny) ** 2
    gamma = case.theta * (case.tau - 0.5) * k2
    t_fit = max(1.0, steps - max(20.0, 20.0 * case.tau))
    return 1.0 / (abs(case.u0) * math.sqrt(case.nx * case.ny) * gamma * t_fit)


def route_storage(case, storage="f16", limit=FP16_NOISE_LIMIT, steps=None) -> str:
    """Storage a case runs in: `storage` (a half format) unless its shear-wave
    decay rate would be resolved worse than the limit allows, then FP32."""
    if storage in ("f16", "bf16") and half_noise_ratio(case, steps) > limit:
        return "f32"
    return storage


def kernel_classes(cases) -> int:
    """Distinct (boundary, equilibrium, collision, temperature mode, theta,
    rho0) combinations: the slots a batch of these lattices launches (one
    kernel each per step)."""
    return len({(c.boundary, c.eq, c.coll, c.theta_mode, c.theta, c.rho0) for c in cases})


def size_class(cases) -> str:
    nodes = sum(c.nx * c.ny for c in cases)
    return f"n{len(cases)}-2^{int(math.log2(max(nodes, 1)))}-s{kernel_classes(cases)}"


# Search space of the tuner.  The stages run in this order, each over one
# group of parameters with the best values found so far for the others:
# (layout, warps per block, blocks per SM), then warp passes per work item,
# then steps per graph replay.  Blocks per SM above the resident count (0)
# oversubscribe the grid: its warps still stride over the work items, but
# blocks start as earlier ones finish, so the block scheduler evens out a mix
# of uneven items (on the 512-lattice FP16 mix: 136 GLUPS with every block
# resident, 142 with 64 blocks per SM, 4 warp passes per item).
TUNE_STAGES = (
    {"layout": ("ab", "aa"), "warps_per_block": (1, 2, 4), "blocks_per_sm": (0, 2, 32, 64, 128)},
    {"item_passes": (1, 2, 4, 8)},
    {"steps_per_launch": (25, 50, 100, 200)},
)
TUNE_START = {"layout": "ab", "warps_per_block": 4, "blocks_per_sm": 0,
              "item_passes": ITEM_PASSES, "steps_per_launch": 50}


def _grid(stage: dict):
    keys = list(stage)
    out = [{}]
    for k in keys:
        out = [dict(o, **{k: v}) for o in out for v in stage[k]]
    return out


def measure_replays(cases, storage: str, cfg: dict, repeats: int, lattices=None) -> list:
    """ms per step of `repeats` timed graph replays (after one untimed replay,
    which captures the graph) of the whole workload in the configuration
    `cfg`.  `lattices` maps a layout to lattices to reuse (created on first
    use on a shared stream, so that they can move between batches)."""
    import torch
    lattices = {} if lattices is None else lattices
    K = int(cfg["steps_per_launch"])
    stream = lattices.setdefault("_stream", torch.cuda.Stream())
    items = sum(work_items(c.nx, c.ny, storage, cfg["item_passes"]) for c in cases)
    with BatchEngine(storage, cfg["layout"], max_lattices=len(cases), max_items=items,
                     steps_per_launch=K, warps_per_block=cfg["warps_per_block"],
                     blocks_per_sm=cfg["blocks_per_sm"], item_passes=cfg["item_passes"],
                     stream=stream) as eng:
        if cfg["layout"] not in lattices:
            lattices[cfg["layout"]] = [eng.new_lattice(c) for c in cases]
        lats = lattices[cfg["layout"]]
        for lat in lats:
            eng.add(lat, (repeats + 1) * K)
        eng.run(1)
        eng.wait()
        out = []
        for _ in range(repeats):
            t0 = time.perf_counter()
            eng.run(1)
            eng.wait()
            out.append((time.perf_counter() - t0) * 1e3 / K)
        for lat in lats:
            eng.remove(lat)
    return out


def autotune(cases, storage="f16", stages=TUNE_STAGES, start=None, repeats=3, use_cache=True,
             cache_path=None, measure=None, verbose=False):
    """Chooses the batch configuration for a workload: layout, warps per block,
    blocks per SM, warp passes per work item and steps per graph replay.

    Each candidate is timed as the median ms per step of `repeats` graph
    replays (``measure_replays``, or `measure(cfg) -> [ms, ...]`); the stages
    of `stages` run in order, each keeping the others at the best values so
    far.  The result (a dict of the five parameters plus ``ms_per_step`` and
    ``candidates``, the number timed) is cached per (ABI version, storage,
    size class) in `cache_path` (default: the build folder)."""
    cache_path = _CACHE if cache_path is None else cache_path
    key = f"abi{B.ABI_VERSION}:{storage}:{size_class(cases)}"
    cache = {}
    if use_cache and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except ValueError:
            cache = {}
        if key in cache:
            return cache[key]
    pool = {}
    if measure is None:
        def measure(cfg):
            return measure_replays(cases, storage, cfg, repeats, pool)
    best = dict(TUNE_START if start is None else start)
    best_ms, seen = None, {}
    try:
        for stage in stages:
            for delta in _grid(stage):
                cfg = dict(best, **delta)
                ident = tuple(sorted(cfg.items()))
                if ident not in seen:
                    samples = list(measure(cfg))
                    seen[ident] = statistics.median(samples)
                    if verbose:
                        print(cfg, [round(x, 4) for x in samples], flush=True)
                if best_ms is None or seen[ident] < best_ms:
                    best, best_ms = cfg, seen[ident]
    finally:
        for name, lats in pool.items():
            if name != "_stream":
                for lat in lats:
                    lat.close()
    result = dict(best, ms_per_step=best_ms, candidates=len(seen), repeats=repeats)
    if use_cache:
        cache[key] = result
        os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return result
