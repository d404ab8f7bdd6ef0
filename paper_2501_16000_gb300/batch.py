"""Batched path: many independent lattices in one persistent launch per step,
steps_per_launch steps per CUDA-graph replay (C ABI ``olb_batch_*``).

``BatchEngine`` owns the batch and a torch stream; its lattices are created on
that stream with torch-allocated population memory.  ``autotune`` picks the
layout, warps per block and persistent-grid size for a workload by timing
short runs, and caches the choice per (storage, size class).
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import time

from . import binding as B
from .engine import LAYOUT, STORAGE, Lattice

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


ITEM_ROW_GROUPS = 4


def segment_lanes(nx: int, ny: int, v: int) -> int:
    """Lanes W per row segment, as the library chooses them: a warp pass covers
    32/W rows of one W-lane segment of W*v nodes, and W (a power of two <= 32)
    needs the fewest passes; among equal counts the widest."""
    best, best_passes = 32, None
    for w in (32, 16, 8, 4, 2, 1):
        passes = math.ceil(nx / (w * v)) * math.ceil(ny / (32 // w))
        if best_passes is None or passes < best_passes:
            best, best_passes = w, passes
    return best


def work_items(nx: int, ny: int, storage: str) -> int:
    """Warp work items of one lattice: a warp pass covers a row group of 32/W
    rows of one W-lane row segment (``segment_lanes``); an item is up to
    ITEM_ROW_GROUPS row groups of one segment."""
    v = 16 // {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[storage]
    w = segment_lanes(nx, ny, v)
    return math.ceil(math.ceil(ny / (32 // w)) / ITEM_ROW_GROUPS) * math.ceil(nx / (w * v))


class BatchEngine:
    def __init__(self, storage="f16", layout="ab", max_lattices=1024, max_items=1 << 22,
                 steps_per_launch=100, warps_per_block=4, blocks_per_sm=0, stream=None):
        import torch
        self.storage, self.layout = storage, layout
        self.steps_per_launch = int(steps_per_launch)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.params = B.olb_batch_params(STORAGE[storage], LAYOUT[layout], int(max_lattices),
                                         int(max_items), int(steps_per_launch),
                                         int(warps_per_block), int(blocks_per_sm),
                                         self.stream.cuda_stream)
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
        B.call("olb_batch_run", self._h, int(nrounds))

    def wait(self) -> None:
        B.call("olb_batch_wait", self._h)

    def close(self) -> None:
        if self._h is not None:
            st = B.load().olb_batch_destroy(self._h)
            self._h = None
            B.check(st, "olb_batch_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def size_class(cases) -> str:
    nodes = sum(c.nx * c.ny for c in cases)
    return f"n{len(cases)}-2^{int(math.log2(max(nodes, 1)))}"


def autotune(cases, storage="f16", steps=20, candidates=None, use_cache=True, verbose=False):
    """Times `steps` steps of the whole workload for each candidate
    (layout, warps_per_block, blocks_per_sm) and returns the fastest as a dict
    with its measured ms per step.  Results are cached per (storage, size class)."""
    import torch
    # the key carries the library's ABI version: kernels and limits change with it
    key = f"abi{B.ABI_VERSION}:{storage}:{size_class(cases)}"
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            cache = json.load(open(_CACHE))
        except ValueError:
            cache = {}
        if key in cache:
            return cache[key]
    if candidates is None:
        candidates = [(lay, w, b) for lay in ("ab", "aa") for w in (1, 2, 4) for b in (0, 1, 2)]
    items = sum(work_items(c.nx, c.ny, storage) for c in cases)
    best = None
    for lay, w, b in candidates:
        with BatchEngine(storage, lay, max_lattices=len(cases), max_items=items,
                         steps_per_launch=steps, warps_per_block=w, blocks_per_sm=b) as eng:
            lats = [eng.new_lattice(c) for c in cases]
            for lat in lats:
                eng.add(lat, 2 * steps)
            eng.run(1)            # capture + warm-up round
            eng.wait()
            t0 = time.perf_counter()
            eng.run(1)
            eng.wait()
            ms = (time.perf_counter() - t0) * 1e3 / steps
            for lat in lats:
                lat.close()
        r = {"layout": lay, "warps_per_block": w, "blocks_per_sm": b, "ms_per_step": ms}
        if verbose:
            print(r, flush=True)
        if best is None or ms < best["ms_per_step"]:
            best = r
    torch.cuda.synchronize()
    if use_cache:
        cache[key] = best
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        json.dump(cache, open(_CACHE, "w"), indent=1)
    return best
