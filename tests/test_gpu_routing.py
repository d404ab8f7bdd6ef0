"""Precision routing of the batched workload on the GPU: the hardest shear
lattices of the 512-lattice mix (seed 1) meet the 1e-4 decay-rate target
against their FP64 runs in the storage the router gives them.

The three with the largest half-precision noise ratio (routed to FP32) and
the three largest the router keeps in FP16 run in batches of their format,
the mode amplitude read between graph rounds of 20 steps; their FP64
references run alone."""
import numpy as np
import pytest

from paper_2501_16000_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TARGET = 1e-4
STEPS, EVERY = 1000, 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16000_gb300 import build
    build.build()


def _hardest():
    from paper_2501_16000_gb300.batch import half_noise_ratio, route_storage
    shear = [c for c in W.batch_mix(512, seed=1, steps=STEPS) if c.case == "shear"]
    shear.sort(key=half_noise_ratio, reverse=True)
    to32 = [c for c in shear if route_storage(c, "f16") == "f32"][:3]
    kept = [c for c in shear if route_storage(c, "f16") == "f16"][:3]
    return to32, kept


def _batched_rates(cases, storage):
    from paper_2501_16000_gb300.analysis import fit_decay
    from paper_2501_16000_gb300.batch import BatchEngine, work_items
    items = sum(work_items(c.nx, c.ny, storage) for c in cases)
    with BatchEngine(storage, "ab", max_lattices=len(cases), max_items=items,
                     steps_per_launch=EVERY) as eng:
        lats = [eng.new_lattice(c) for c in cases]
        for lat in lats:
            eng.add(lat, STEPS)
        amps = [[lat.wave_amplitude(c.m, c.n)] for lat, c in zip(lats, cases)]
        for _ in range(STEPS // EVERY):
            eng.run(1)
            eng.wait()
            for a, lat, c in zip(amps, lats, cases):
                a.append(lat.wave_amplitude(c.m, c.n))
        ts = np.arange(0, STEPS + 1, EVERY)
        rates = [fit_decay(ts, a, c.tau) for a, c in zip(amps, cases)]
        for lat in lats:
            lat.close()
    return rates


def _fp64_rate(c):
    from paper_2501_16000_gb300.analysis import measure_decay
    from paper_2501_16000_gb300.engine import Lattice
    with Lattice(c.nx, c.ny, c.tau, c.theta, storage="f64", layout="ab") as lat:
        lat.init_case(c)
        return measure_decay(lat, c, STEPS, every=EVERY)[0]


@pytest.mark.parametrize("group", ["routed_to_f32", "kept_in_f16"])
def test_hardest_lattices_meet_the_decay_target_in_their_routed_format(group):
    to32, kept = _hardest()
    cases, storage = (to32, "f32") if group == "routed_to_f32" else (kept, "f16")
    assert len(cases) == 3
    for c, g in zip(cases, _batched_rates(cases, storage)):
        err = abs(g / _fp64_rate(c) - 1)
        print(f"{storage} {c.nx}x{c.ny} tau {c.tau:.3f} u0 {c.u0:.3f}: decay-rate error {err:.2e}")
        assert err <= TARGET, (c, err)
