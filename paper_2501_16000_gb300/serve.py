"""Continuous-batching request server for shear-wave and shock-tube solves.

Requests (``workloads.Request``: arrival time, lattice, step count) arrive
over wall-clock time.  Arrived requests wait in a FIFO queue and are admitted
as soon as their device memory (``Server.request_bytes``: populations plus the
FP64 fields they are read back into) fits the HBM budget next to everything
in flight; admitted requests join the running ``BatchEngine`` and advance
together with all other in-flight requests, one CUDA-graph round of K steps
at a time, their states resident in HBM.  A request whose steps are done
leaves the batch and is read back on a side stream by a worker thread (FP64
diagnostics: a solve that turned non-finite is reported with status
"nonfinite" and no fields; moments to host), after which its memory is freed,
which may admit the next ones.  A request can be cancelled while it waits or
while it runs (status "cancelled"; an in-flight one leaves the batch at the
next round boundary and frees its memory).  Latency is arrival -> result in
host memory.

The loop keeps the GPU fed: joining and leaving the batch enqueue their table
changes on the batch's stream without waiting, round r + 1 is enqueued before
the host waits for round r, and the read-back of requests that finished in a
round runs on its own stream, overlapping the next round, while the host
admits new requests.  The library allocates no device memory on this path.

``serve_serial`` replays the same trace with one plain FP32 single-lattice
solve at a time (the baseline).
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import time

import numpy as np

from .batch import ITEM_PASSES, BatchEngine, work_items
from .engine import Lattice, required_bytes


@dataclasses.dataclass
class Result:
    rid: int
    arrival_s: float
    admitted_s: float
    done_s: float
    nodes: int
    steps: int
    case: str
    fields: tuple | None = None
    status: str = "ok"          # "ok", "nonfinite" or "cancelled"

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


def summarize(results, wall_s, label):
    """Throughput and latency of the completed ("ok") solves; failed and
    cancelled requests are counted separately."""
    failed = sum(r.status == "nonfinite" for r in results)
    cancelled = sum(r.status == "cancelled" for r in results)
    results = [r for r in results if r.status == "ok"]
    lat = np.array([r.latency_s for r in results])
    work = sum(r.nodes * r.steps for r in results)
    return {
        "label": label,
        "solves": len(results),
        "nonfinite": failed,
        "cancelled": cancelled,
        "wall_s": round(wall_s, 3),
        "solves_per_s": round(len(results) / wall_s, 2) if wall_s > 0 else None,
        "mlups": round(work / wall_s / 1e6, 1) if wall_s > 0 else None,
        "p50_latency_s": round(float(np.percentile(lat, 50)), 4) if len(lat) else None,
        "p99_latency_s": round(float(np.percentile(lat, 99)), 4) if len(lat) else None,
        "max_latency_s": round(float(lat.max()), 4) if len(lat) else None,
    }


def _bytes(lat_case, storage, layout):
    return required_bytes(nx=lat_case.nx, ny=lat_case.ny, tau=lat_case.tau,
                          theta=lat_case.theta, eq=lat_case.eq, coll=lat_case.coll,
                          storage=storage, layout=layout)


class Server:
    def __init__(self, storage="f16", layout="ab", budget_bytes=120e9, steps_per_launch=100,
                 max_lattices=8192, max_items=1 << 24, warps_per_block=4, blocks_per_sm=0,
                 keep_fields=True, engine=None, item_passes=ITEM_PASSES, round_timeout_s=None):
        """``engine`` replaces the BatchEngine (anything with its new_lattice,
        add, remove, remaining, run, record_event, read_back and close
        methods).  ``round_timeout_s``: if set, the host waits at most this
        long for each enqueued round (polling its event) and ``run`` raises
        TimeoutError when a round has not finished by then, instead of
        blocking on a stalled device."""
        self.storage, self.layout = storage, layout
        self.budget = float(budget_bytes)
        self.keep_fields = keep_fields
        self.engine = engine if engine is not None else BatchEngine(
            storage, layout, max_lattices=max_lattices, max_items=max_items,
            steps_per_launch=steps_per_launch, warps_per_block=warps_per_block,
            blocks_per_sm=blocks_per_sm, item_passes=item_passes)
        self.item_passes = int(item_passes)
        self.max_items = max_items
        self.round_timeout_s = round_timeout_s
        self.rounds = 0
        self.peak_bytes = 0
        self.peak_inflight = 0

    def close(self):
        self.engine.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _wait_round(self, ev) -> None:
        if self.round_timeout_s is None:
            ev.synchronize()
            return
        until = time.perf_counter() + self.round_timeout_s
        while not ev.query():
            if time.perf_counter() >= until:
                raise TimeoutError(f"a batch round did not finish within {self.round_timeout_s} s")
            time.sleep(5e-5)

    def request_bytes(self, case) -> int:
        """Device memory a request holds while admitted: its populations and,
        when fields are kept, the FP64 rho, u_x, u_y it is read back into."""
        fields = 24 * case.nodes + 64 if self.keep_fields else 64
        return _bytes(case, self.storage, self.layout) + fields

    def run(self, trace, time_scale: float = 1.0, cancel_at=None, prepare=None):
        """Serves the trace in real time (arrival times scaled by time_scale);
        returns (results, wall seconds).

        cancel_at: {rid: trace time} at which a request is cancelled (a
        waiting one is dropped, an in-flight one removed from the batch).
        prepare(request, lattice): called once a request's lattice is created
        and initialised, before it joins the batch."""
        eng = self.engine
        pending = collections.deque(sorted(trace, key=lambda r: r.arrival_s))
        queue = collections.deque()
        inflight = {}           # rid -> (request, lattice, bytes, items, admitted_s)
        finishing = {}          # rid -> future of (Result, bytes, items)
        rounds = collections.deque()   # events of enqueued rounds not yet waited for
        in_bytes = 0
        in_items = 0
        results = []
        cancels = dict(cancel_at or {})
        side = eng.side_stream() if hasattr(eng, "side_stream") else None
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0

        def cancelled(req, admitted_s):
            return Result(req.rid, req.arrival_s * time_scale, admitted_s, now(),
                          req.lattice.nodes, req.lattice.steps, req.lattice.case, None,
                          "cancelled")

        def finish(req, lat, after, need, items, adm):
            # worker thread: waits for the round, reads back, frees the lattice
            _, nonfinite, fields = eng.read_back(lat, after, side, self.keep_fields)
            lat.close()
            ok = nonfinite == 0
            res = Result(req.rid, req.arrival_s * time_scale, adm, now(), req.lattice.nodes,
                         req.lattice.steps, req.lattice.case, fields if ok else None,
                         "ok" if ok else "nonfinite")
            return res, need, items

        worker = concurrent.futures.ThreadPoolExecutor(max_workers=1)
        try:
            while pending or queue or inflight or finishing:
                # read-backs that completed free their memory for admission
                for rid in [r for r, fut in finishing.items() if fut.done()]:
                    res, need, items = finishing.pop(rid).result()
                    results.append(res)
                    in_bytes -= need
                    in_items -= items
                t = now()
                while pending and pending[0].arrival_s * time_scale <= t:
                    queue.append(pending.popleft())
                # cancellations that are due: drop waiting requests, evict running ones
                for rid in [r for r, ct in cancels.items() if ct * time_scale <= t]:
                    del cancels[rid]
                    for dq in (pending, queue):
                        hit = [q for q in dq if q.rid == rid]
                        for q in hit:
                            dq.remove(q)
                            results.append(cancelled(q, now()))
                    if rid in inflight:
                        req, lat, need, items, adm = inflight.pop(rid)
                        eng.remove(lat)
                        lat.close()     # waits for the rounds already enqueued
                        in_bytes -= need
                        in_items -= items
                        results.append(cancelled(req, adm))
                # FIFO admission against the memory budget (and the item table)
                while queue:
                    req = queue[0]
                    need = self.request_bytes(req.lattice)
                    items = work_items(req.lattice.nx, req.lattice.ny, self.storage,
                                       self.item_passes)
                    if need > self.budget:
                        raise ValueError(f"request {req.rid} needs {need} B > budget")
                    if in_bytes + need > self.budget or in_items + items > self.max_items:
                        break
                    queue.popleft()
                    lat = eng.new_lattice(req.lattice)
                    if prepare is not None:
                        prepare(req, lat)
                    eng.add(lat, req.lattice.steps)
                    inflight[req.rid] = (req, lat, need, items, now())
                    in_bytes += need
                    in_items += items
                self.peak_bytes = max(self.peak_bytes, in_bytes)
                self.peak_inflight = max(self.peak_inflight, len(inflight) + len(finishing))
                if inflight:
                    eng.run(1)
                    self.rounds += 1
                    ev = eng.record_event()
                    for rid in [r for r, v in inflight.items() if eng.remaining(v[1]) == 0]:
                        req, lat, need, items, adm = inflight.pop(rid)
                        eng.remove(lat)
                        finishing[rid] = worker.submit(finish, req, lat, ev, need, items, adm)
                    # round r + 1 is enqueued before the host waits for round r
                    rounds.append(ev)
                    if len(rounds) > 1:
                        self._wait_round(rounds.popleft())
                    continue
                while rounds:
                    self._wait_round(rounds.popleft())
                # idle: wait for the next arrival or a read-back
                wait = 0.01
                if pending:
                    wait = min(wait, pending[0].arrival_s * time_scale - now())
                if finishing:
                    wait = min(wait, 0.0005)
                if wait > 0:
                    time.sleep(wait)
        finally:
            worker.shutdown(wait=True)
        return results, now()


def serve_serial(trace, storage="f32", layout="ab", time_scale: float = 1.0, keep_fields=True):
    """Baseline: FIFO, one plain single-lattice solve at a time."""
    pending = collections.deque(sorted(trace, key=lambda r: r.arrival_s))
    results = []
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    while pending:
        req = pending.popleft()
        wait = req.arrival_s * time_scale - now()
        if wait > 0:
            time.sleep(wait)
        c = req.lattice
        start = now()
        with Lattice(c.nx, c.ny, c.tau, c.theta, c.eq, c.coll, storage, layout,
                     boundary=c.boundary, theta_mode=c.theta_mode) as lat:
            lat.init_case(c)
            lat.step(c.steps)
            fields = lat.moments() if keep_fields else None
            if not keep_fields:
                lat.diagnostics()
        results.append(Result(req.rid, req.arrival_s * time_scale, start, now(), c.nodes,
                              c.steps, c.case, fields))
    return results, now()
