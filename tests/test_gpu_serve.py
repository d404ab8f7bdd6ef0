"""Serving on the GPU: requests served with continuous batching (joining and
leaving while others run, admission against a memory budget) give the same
result, bitwise, as the same request solved alone."""
import numpy as np
import pytest

from paper_2501_16000_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16000_gb300 import build
    build.build()


def small_trace(n=14, seed=11):
    return W.arrival_trace(n, rate_per_s=400.0, seed=seed, lo=8, hi=96, steps_lo=10,
                           steps_hi=300)


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_served_results_equal_alone(layout):
    from paper_2501_16000_gb300.engine import Lattice
    from paper_2501_16000_gb300.serve import Server
    trace = small_trace()
    srv = Server("f16", layout, budget_bytes=1e9, steps_per_launch=16)
    results, wall = srv.run(trace)
    srv.close()
    assert len(results) == len(trace)
    assert srv.peak_inflight > 1                     # work actually overlapped
    by_id = {r.rid: r for r in results}
    for req in trace:
        c = req.lattice
        with Lattice(c.nx, c.ny, c.tau, c.theta, c.eq, c.coll, "f16", layout) as lat:
            lat.init_case(c)
            lat.step(c.steps)
            alone = lat.moments()
        for a, b in zip(alone, by_id[req.rid].fields):
            assert np.array_equal(a, b), req.rid
        assert by_id[req.rid].latency_s >= 0


def test_served_requests_of_many_kernel_classes_equal_alone():
    """Requests of six kernel / constant classes (OReg and BGK, guided at two
    temperatures and polynomial) arriving while others run: new classes join
    mid-run (the batch graph is captured again, each class on its own capture
    stream), and every result is still bitwise that of the request alone."""
    import dataclasses

    from paper_2501_16000_gb300.engine import Lattice
    from paper_2501_16000_gb300.serve import Server
    trace = small_trace(n=12, seed=17)
    classes = []
    for j, req in enumerate(sorted(trace, key=lambda r: r.arrival_s)):
        poly = (j // 2) % 2 == 1
        lat = dataclasses.replace(req.lattice, coll="bgk" if j % 2 else "oreg",
                                  eq="poly2" if poly else "guided",
                                  theta=1.0 / 3.0 if poly else (0.30 if (j // 4) % 2 else 0.36))
        classes.append(dataclasses.replace(req, lattice=lat))
    srv = Server("f16", "ab", budget_bytes=1e9, steps_per_launch=16)
    results, _ = srv.run(classes)
    srv.close()
    assert len(results) == len(classes) and srv.peak_inflight > 1
    by_id = {r.rid: r for r in results}
    for req in classes:
        c = req.lattice
        with Lattice(c.nx, c.ny, c.tau, c.theta, c.eq, c.coll, "f16", "ab") as lat:
            lat.init_case(c)
            lat.step(c.steps)
            alone = lat.moments()
        for a, b in zip(alone, by_id[req.rid].fields):
            assert np.array_equal(a, b), (req.rid, c.coll, c.eq, c.theta)


def test_admission_respects_the_budget():
    from paper_2501_16000_gb300.serve import Server
    trace = small_trace(n=10, seed=3)
    srv = Server("f16", "ab", budget_bytes=1.0, steps_per_launch=16)
    sizes = [srv.request_bytes(r.lattice) for r in trace]
    srv.budget = budget = 2 * max(sizes)
    results, _ = srv.run(trace)
    srv.close()
    assert len(results) == len(trace)
    assert srv.peak_bytes <= budget
    assert srv.peak_bytes > max(sizes)       # requests did overlap within the budget


def test_nonfinite_request_is_reported_and_the_others_are_unaffected():
    """A NaN planted on the host in one request's populations (before it joins
    the batch) makes that request come back with status "nonfinite" and no
    fields; a request cancelled before it arrives is never admitted; every
    other result stays bitwise equal to the same request solved alone."""
    from paper_2501_16000_gb300.engine import Lattice
    from paper_2501_16000_gb300.serve import Server
    trace = small_trace(n=10, seed=5)
    by_arrival = sorted(trace, key=lambda r: r.arrival_s)
    poison, early = by_arrival[1].rid, by_arrival[-1].rid

    def prepare(req, lat):
        if req.rid == poison:
            f = lat.populations()
            f[2, lat.ny // 2, lat.nx // 2] = np.nan
            lat.set_populations(f, 0)

    srv = Server("f16", "ab", budget_bytes=1e9, steps_per_launch=16)
    results, _ = srv.run(trace, cancel_at={early: -1.0}, prepare=prepare)
    srv.close()
    by_id = {r.rid: r for r in results}
    assert sorted(by_id) == sorted(r.rid for r in trace)
    assert by_id[poison].status == "nonfinite" and by_id[poison].fields is None
    assert by_id[early].status == "cancelled"
    for req in trace:
        if req.rid in (poison, early):
            continue
        c = req.lattice
        with Lattice(c.nx, c.ny, c.tau, c.theta, c.eq, c.coll, "f16", "ab") as lat:
            lat.init_case(c)
            lat.step(c.steps)
            alone = lat.moments()
        assert by_id[req.rid].status == "ok"
        for a, b in zip(alone, by_id[req.rid].fields):
            assert np.array_equal(a, b), req.rid
