"""Host-side logic on CPU: seeded input generators, the decay-rate fit, the
work-item count and the serving loop's admission against a memory budget
(with a stand-in for the GPU batch engine)."""
import math
import time

import numpy as np
import pytest

from paper_2501_16000_gb300 import workloads as W
from paper_2501_16000_gb300.analysis import fit_decay
from paper_2501_16000_gb300.batch import warp_passes, work_items
from paper_2501_16000_gb300.engine import required_bytes


def test_generators_are_seeded_and_in_range():
    a, b = W.batch_mix(64, seed=1), W.batch_mix(64, seed=1)
    assert a == b
    assert a != W.batch_mix(64, seed=2)
    for c in a:
        assert 32 <= c.nx <= 1024 and 32 <= c.ny <= 1024
        assert 0.51 <= c.tau <= 1.0
        if c.case == "shear":
            assert (c.m, c.n) != (0, 0) and 0.01 <= c.u0 <= 0.1
        else:
            assert c.x_split == c.nx // 2
    t = W.arrival_trace(100, rate_per_s=10.0, seed=2)
    arr = [r.arrival_s for r in t]
    assert arr == sorted(arr) and all(64 <= r.lattice.nx <= 2048 for r in t)
    assert all(100 <= r.lattice.steps <= 10000 for r in t)
    # mean inter-arrival of a Poisson process
    assert 0.05 < np.mean(np.diff([0.0] + arr)) < 0.2


def test_shear_wave_fields_and_window_agree():
    rho, ux, uy = W.shear_wave_fields(40, 30, 1.0, 0.05, 3, 2)
    ex, ey = W.shear_wave_direction(40, 30, 3, 2)
    assert np.allclose(ux * ey - uy * ex, 0.0)                 # velocity along e_perp
    assert abs(np.sum(ux)) < 1e-12 and np.isclose(np.abs(ux * ex + uy * ey).max(), 0.05, atol=2e-3)
    wr, wx, wy = W.shear_wave_window(40, 30, 1.0, 0.05, 3, 2, 35, 25, 10, 10)   # wraps
    xs, ys = (35 + np.arange(10)) % 40, (25 + np.arange(10)) % 30
    assert np.array_equal(wx, ux[np.ix_(ys, xs)]) and np.array_equal(wy, uy[np.ix_(ys, xs)])
    m, n, ang = W.wave_vector_from_angle(8192, 8192, math.pi / 6)
    assert (m, n) == (111, 64) and abs(ang - math.pi / 6) < 1e-2


def test_fit_decay_recovers_an_exponential():
    ts = np.arange(0, 2001, 20, dtype=float)
    amps = 0.05 * np.exp(-3e-3 * ts)
    assert abs(fit_decay(ts, amps, tau=0.8) / 3e-3 - 1) < 1e-12
    noisy = amps * (1 + 1e-6 * np.random.default_rng(0).standard_normal(ts.size))
    noisy[ts > 1000] = 1e-9                                    # noise floor: excluded
    assert abs(fit_decay(ts, noisy, tau=0.8) / 3e-3 - 1) < 1e-3
    with pytest.raises(ValueError):
        fit_decay([0, 10], [1.0, 0.9], tau=0.8)


@pytest.mark.parametrize("storage,v", [("f64", 2), ("f32", 4), ("f16", 8)])
def test_warp_passes_cover_every_node_once(storage, v):
    """The stream-collide kernels' lane mapping, restated: warp pass p, lane l
    holds vector 32 p + l of the row-major planes (rows of ceil(nx / v)
    vectors), i.e. row y = vector // vpr and nodes xb .. xb + v - 1 with
    xb = v (vector % vpr); lanes past the last vector idle.  Every node is
    held by exactly one lane, and only the last pass has idle lanes."""
    for nx in (1, 5, 33, 37, 100, 256, 257, 300, 1024, 3000):
        for ny in (1, 3, 4, 32, 33, 500):
            vpr = math.ceil(nx / v)
            passes = warp_passes(nx, ny, v)
            vec = np.arange(passes * 32)
            y, xb = vec // vpr, (vec % vpr) * v
            live = y < ny
            assert (~live).sum() < 32 and live[: (passes - 1) * 32].all()
            held = np.zeros((ny, nx), dtype=int)
            for j in range(v):
                ok = live & (xb + j < nx)
                np.add.at(held, (y[ok], xb[ok] + j), 1)
            assert (held == 1).all()
            for r in (1, 2, 4, 8):
                assert work_items(nx, ny, storage, r) == math.ceil(passes / r)
    assert warp_passes(8192, 8192, 8) == 8192 * 8192 // 256


class _FakeLattice:
    def __init__(self, case):
        self.case, self.closed, self.poisoned = case, False, False

    def moments(self):
        return (np.ones((self.case.ny, self.case.nx)),) * 3

    def diagnostics(self, raise_nonfinite=True):
        return {"mass": 1.0, "mom_x": 0.0, "mom_y": 0.0, "nonfinite": 7 if self.poisoned else 0}

    def close(self):
        self.closed = True


class _FakeEngine:
    """Advances every member K steps per round; no GPU."""

    def __init__(self, K, round_s=0.0):
        self.K, self.left, self.order, self.rounds = K, {}, [], 0
        self.round_s, self.evicted = round_s, []

    def new_lattice(self, case):
        return _FakeLattice(case)

    def add(self, lat, n):
        self.left[id(lat)] = n
        self.order.append(lat.case)

    def remove(self, lat):
        if self.left[id(lat)] > 0:
            self.evicted.append(lat.case)
        del self.left[id(lat)]

    def remaining(self, lat):
        return self.left[id(lat)]

    def run(self, n=1):
        self.rounds += n
        if self.round_s:
            time.sleep(self.round_s * n)
        for k in self.left:
            self.left[k] = max(0, self.left[k] - n * self.K)

    def wait(self):
        pass

    def record_event(self):
        return _Done()

    def read_back(self, lat, after, stream, keep_fields=True):
        after.synchronize()
        d = lat.diagnostics(raise_nonfinite=False)
        return d["mass"], d["nonfinite"], (lat.moments() if keep_fields else None)

    def close(self):
        pass


class _Done:
    def synchronize(self):
        pass

    def query(self):
        return True


class _Stalled:
    """An event of a round that never finishes (a stalled device)."""

    def synchronize(self):
        raise AssertionError("an unbounded wait on a stalled round")

    def query(self):
        return False


def test_server_reports_a_stalled_round_within_its_timeout():
    """With round_timeout_s the server polls each round's event and raises
    TimeoutError once the limit has passed, instead of blocking on a round
    that never finishes (a fake event stands in for a stalled GPU)."""
    from paper_2501_16000_gb300 import build
    build.build()                                   # request_bytes is a host-only library call
    from paper_2501_16000_gb300.serve import Server
    eng = _FakeEngine(K=10)
    eng.record_event = lambda: _Stalled()
    trace = [W.Request(0, 0.0, W.LatticeCase(nx=8, ny=8, tau=0.8, steps=100))]
    srv = Server(engine=eng, budget_bytes=1e9, round_timeout_s=0.05)
    t0 = time.perf_counter()
    with pytest.raises(TimeoutError):
        srv.run(trace)
    assert time.perf_counter() - t0 < 5.0
    assert eng.rounds >= 2            # round r + 1 was enqueued before waiting for round r


def test_serving_admission_fifo_and_budget():
    from paper_2501_16000_gb300 import build
    build.build()                                   # required_bytes is a host-only library call
    from paper_2501_16000_gb300.serve import Server
    trace = W.arrival_trace(30, rate_per_s=2000.0, seed=5, lo=16, hi=256, steps_lo=10,
                            steps_hi=500)
    probe = Server("f16", "ab", engine=_FakeEngine(K=1))
    sizes = [probe.request_bytes(r.lattice) for r in trace]
    assert all(sz > required_bytes(nx=r.lattice.nx, ny=r.lattice.ny, tau=r.lattice.tau,
                                   storage="f16", layout="ab") for sz, r in zip(sizes, trace))
    budget = 3 * max(sizes)
    eng = _FakeEngine(K=50)
    srv = Server("f16", "ab", budget_bytes=budget, engine=eng)
    results, wall = srv.run(trace)
    assert len(results) == len(trace)
    assert srv.peak_bytes <= budget and srv.peak_inflight >= 2
    # admission is first come, first served
    assert [c for c in eng.order] == [r.lattice for r in sorted(trace, key=lambda r: r.arrival_s)]
    for r in results:
        assert r.done_s >= r.admitted_s >= r.arrival_s - 1e-9 and r.latency_s >= 0
        assert r.fields[0].shape == (next(q.lattice.ny for q in trace if q.rid == r.rid),
                                     next(q.lattice.nx for q in trace if q.rid == r.rid))


def test_paper_workloads_use_the_printed_parameters():
    """The Sec. IV workloads are built from the values the paper prints
    (tests/golden/paper_values.json): the walled shock tube's grid, steps,
    temperatures and viscosities, and the shear wave's amplitude, length,
    temperature and viscosity.  The axis-aligned wave runs 4 columns wide
    instead of the printed 1 (the wave does not vary in x, so the columns
    are identical)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.json")
    g = json.load(open(path))
    s = g["walled_shock_tube"]
    for gc in s["cases"]:
        c = W.shock_tube_walls(theta=gc["theta"], nu=gc["nu"])
        assert [c.nx, c.ny] == s["grid"] and c.steps == s["steps"]
        assert c.boundary == "walls_x" and c.eq == "guided"
        assert abs(c.theta * (c.tau - 0.5) - gc["nu"]) <= 1e-15
    d = g["decaying_shear_wave"]
    theta = d["theta"][0] / d["theta"][1]
    for ma in (0.0, 0.2, 0.4):
        c = W.mach_wave("axis", ma)
        assert c.ny == d["grid"][1] and (c.m, c.n) == (0, 1)
        assert abs(c.u0) == d["A0"] and abs(c.theta - theta) <= 1e-15
        assert abs(c.theta * (c.tau - 0.5) - d["nu"]) <= 1e-15
        assert abs(c.uy_mean - ma * math.sqrt(theta)) <= 1e-15
        x, y = np.meshgrid(np.arange(c.nx), np.arange(c.ny))
        rho, ux, uy = c.fields()
        assert np.allclose(rho, d["rho0"])
        assert np.allclose(ux, d["A0"] * np.sin(2 * np.pi * y / d["grid"][1]), rtol=0, atol=1e-15)
        assert np.allclose(uy, c.uy_mean, rtol=0, atol=1e-15)
    # the pi/4 wave: u = (A0, A0 + Ma sqrt(theta)) with sin(2 pi (-x + y) / (L sqrt 2))
    c = W.mach_wave("diagonal", 0.2)
    x, y = np.meshgrid(np.arange(c.nx), np.arange(c.ny))
    rho, ux, uy = c.fields()
    s = d["A0"] * np.sin(2 * np.pi * (-x + y) / c.nx)
    assert c.nx == round(d["grid"][1] * math.sqrt(2))
    assert np.allclose(ux, s, rtol=0, atol=1e-15)
    assert np.allclose(uy, c.uy_mean + s, rtol=0, atol=1e-15)


def test_serving_reports_nonfinite_and_cancelled_requests():
    """A request whose solve turns non-finite is reported as such, without
    fields; cancelled requests are dropped while waiting or evicted while
    running, their memory freed; every other request completes."""
    from paper_2501_16000_gb300 import build
    build.build()
    from paper_2501_16000_gb300.serve import Server, summarize
    trace = W.arrival_trace(24, rate_per_s=500.0, seed=9, lo=16, hi=128, steps_lo=100,
                            steps_hi=2000)
    by_arrival = sorted(trace, key=lambda r: r.arrival_s)
    long_run = max(trace, key=lambda r: r.lattice.steps)      # cancelled while running
    early = next(r.rid for r in reversed(by_arrival) if r.rid != long_run.rid)  # before arrival
    poison = next(r.rid for r in by_arrival if r.rid not in (long_run.rid, early))
    sizes = [Server("f16", "ab", engine=_FakeEngine(K=1)).request_bytes(r.lattice)
             for r in trace]
    eng = _FakeEngine(K=50, round_s=0.002)
    srv = Server("f16", "ab", budget_bytes=sum(sizes), engine=eng)
    cancel_at = {early: -1.0, long_run.rid: long_run.arrival_s + 0.006}
    results, wall = srv.run(trace, cancel_at=cancel_at,
                            prepare=lambda req, lat: setattr(lat, "poisoned", req.rid == poison))
    status = {r.rid: r.status for r in results}
    assert sorted(status) == sorted(r.rid for r in trace)       # every request answered once
    assert status[poison] == "nonfinite"
    assert next(r for r in results if r.rid == poison).fields is None
    assert status[early] == "cancelled" and early not in [c for c in eng.order]
    assert status[long_run.rid] == "cancelled"
    assert long_run.lattice in eng.evicted                    # it was running
    for r in results:
        if r.rid not in cancel_at and r.rid != poison:
            assert r.status == "ok" and r.fields is not None
    s = summarize(results, wall, "fake")
    assert s["nonfinite"] == 1 and s["cancelled"] == len(cancel_at)
    assert s["solves"] == len(trace) - 1 - len(cancel_at)
    assert not eng.left                                        # nothing left in the batch


def test_autotune_picks_the_fastest_candidate_and_honours_the_cache(tmp_path):
    """The tuner with a stand-in measurement (no GPU): a known cost surface,
    noisy samples whose median is the true cost; it must return the cheapest
    configuration of its staged search, time each candidate once, take the
    median of the samples, and answer a second call from the cache."""
    from paper_2501_16000_gb300 import batch as BT
    cases = W.batch_mix(8, seed=1)
    calls = []

    def cost(cfg):
        c = 1.0
        c += {"ab": 0.0, "aa": 0.3}[cfg["layout"]]
        c += {1: 0.2, 2: 0.05, 4: 0.0}[cfg["warps_per_block"]]
        c += {0: 0.0, 2: 0.1, 32: 0.03, 64: 0.2, 128: 0.4}[cfg["blocks_per_sm"]]
        c += {1: 0.08, 2: 0.0, 4: 0.02, 8: 0.05}[cfg["item_passes"]]
        c += {25: 0.04, 50: 0.02, 100: 0.0, 200: 0.01}[cfg["steps_per_launch"]]
        return c

    def measure(cfg):
        calls.append(dict(cfg))
        c = cost(cfg)
        return [c + 5.0, c, c - 0.001]        # one outlier: the median is c

    path = str(tmp_path / "tune.json")
    r = BT.autotune(cases, "f16", repeats=3, cache_path=path, measure=measure)
    assert (r["layout"], r["warps_per_block"], r["blocks_per_sm"]) == ("ab", 4, 0)
    assert (r["item_passes"], r["steps_per_launch"]) == (2, 100)
    assert abs(r["ms_per_step"] - 1.0) < 1e-12
    idents = [tuple(sorted(c.items())) for c in calls]
    assert len(idents) == len(set(idents)) == r["candidates"]
    assert {c["steps_per_launch"] for c in calls} == {25, 50, 100, 200}
    n = len(calls)
    r2 = BT.autotune(cases, "f16", repeats=3, cache_path=path, measure=measure)
    assert r2 == r and len(calls) == n                      # answered from the cache
    r3 = BT.autotune(BT_cases := W.batch_mix(16, seed=1), "f16", cache_path=path, measure=measure)
    assert len(calls) > n and BT.size_class(BT_cases) != BT.size_class(cases)
    # the same lattices over more kernel classes (slots) are tuned anew
    mix, classes = W.batch_mix(16, seed=1), W.batch_mix_classes(16, seed=1)
    assert BT.kernel_classes(mix) == 1 and BT.kernel_classes(classes) == 6
    assert [(c.nx, c.ny, c.tau) for c in mix] == [(c.nx, c.ny, c.tau) for c in classes]
    n3 = len(calls)
    BT.autotune(classes, "f16", cache_path=path, measure=measure)
    assert len(calls) > n3


def test_precision_router_rule():
    """The half-noise ratio 1 / (u0 sqrt(N) gamma T) (gamma = theta (tau -
    1/2) |k|^2, T the steps after the fit's start-up window): shock tubes and
    FP32/FP64 batches are never rerouted; a shear wave moves to FP32 exactly
    when the ratio exceeds the limit, and the ratio falls with amplitude,
    size, viscosity and step count as that formula says."""
    from paper_2501_16000_gb300.batch import FP16_NOISE_LIMIT, half_noise_ratio, route_storage
    shock = W.shock_2048x4()
    assert half_noise_ratio(shock) == 0.0 and route_storage(shock, "f16") == "f16"
    c = W.LatticeCase(nx=64, ny=64, tau=0.6, case="shear", u0=0.05, m=1, n=0, steps=1000)
    k2 = (2 * math.pi / 64) ** 2
    want = 1.0 / (0.05 * 64 * (1 / 3) * 0.1 * k2 * (1000 - max(20, 20 * 0.6)))
    assert abs(half_noise_ratio(c) / want - 1) < 1e-12
    import dataclasses
    assert half_noise_ratio(dataclasses.replace(c, u0=0.1)) == pytest.approx(want / 2)
    assert half_noise_ratio(dataclasses.replace(c, ny=256)) == pytest.approx(want / 2)  # k along x
    for st in ("f32", "f64"):
        assert route_storage(dataclasses.replace(c, u0=1e-6), st) == st
    for u0 in (1e-4, 1e-3, 1e-2, 0.1):
        r = half_noise_ratio(dataclasses.replace(c, u0=u0))
        assert route_storage(dataclasses.replace(c, u0=u0), "f16") == (
            "f32" if r > FP16_NOISE_LIMIT else "f16")
