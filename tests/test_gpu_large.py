"""The 8192 x 8192 rotated shear wave (benchmark lattice) on the GPU.

FP64 GPU and the benchmark's FP32 A-B configuration vs the FP64 oracle
through a domain-of-dependence crop after the benchmark's 500 steps: a node then depends only on initial nodes within
Chebyshev distance T = 500, so the oracle runs a (W + 2T)^2 = 1256^2 window
initialised from the same global field (periodic on the window: the wrap
contaminates only the outer T nodes) and its central W x W block must equal
the GPU crop.  The FP32, FP16 and BF16 runs are compared with the FP64 GPU
run over the whole lattice (olb_compare, a max-abs reduction on the GPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_16000_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16000_gb300 import build
    build.build()


@pytest.mark.parametrize("theta", [1.0 / 3.0, 0.3])
def test_8192_fp64_crop_matches_oracle(theta):
    from paper_2501_16000_gb300.engine import Lattice
    case = W.large_shear(theta=theta, seed=0, side=8192, steps=500)
    T, Wd = case.steps, 256
    crops = [(8192 - 128, 8192 - 100)]       # across the periodic wrap in x and y
    x0, y0 = crops[0]

    def crop(lat):
        # a crop straddling the periodic boundary is read in pieces
        big = np.empty((9, Wd, Wd))
        for (xs, wx, gx) in ((x0, 8192 - x0, 0), (0, Wd - (8192 - x0), 8192 - x0)):
            for (ys, wy, gy) in ((y0, 8192 - y0, 0), (0, Wd - (8192 - y0), 8192 - y0)):
                big[:, gy:gy + wy, gx:gx + wx] = lat.region(xs, ys, wx, wy)
        return big

    got = {}
    # FP64 (in-place layout), and the benchmark's own configuration: FP32
    # storage and collision, A-B layout, 4 warps per block
    for storage, layout in (("f64", "aa"), ("f32", "ab")):
        with Lattice(case.nx, case.ny, case.tau, theta, storage=storage, layout=layout) as lat:
            lat.init_case(case)
            lat.step(T)
            got[storage] = crop(lat)
    p = O.params(Wd + 2 * T, Wd + 2 * T, case.tau, theta, O.GUIDED, O.OREG)
    fields = W.shear_wave_window(case.nx, case.ny, 1.0, case.u0, case.m, case.n,
                                 x0 - T, y0 - T, Wd + 2 * T, Wd + 2 * T)
    ref = O.run(O.init_equilibrium(p, *fields), p, T)[:, T:T + Wd, T:T + Wd]
    for storage, tol in (("f64", 1e-12), ("f32", 1e-5)):
        err = np.abs(got[storage] - ref).max() / np.abs(ref).max()
        print(f"8192^2 {storage} crop at ({x0}, {y0}) after {T} steps, theta {theta:.3f}: "
              f"rel Linf vs oracle {err:.3e}")
        assert err <= tol, (storage, err)


def test_8192_reduced_precision_vs_fp64_over_the_whole_lattice():
    from paper_2501_16000_gb300.engine import Lattice
    case = W.large_shear(theta=1.0 / 3.0, seed=0, side=8192, steps=500)
    err = {}
    with Lattice(case.nx, case.ny, case.tau, storage="f64", layout="aa") as ref:
        ref.init_case(case)
        ref.step(case.steps)
        d64 = ref.diagnostics()
        for st in ("f32", "f16", "bf16"):
            with Lattice(case.nx, case.ny, case.tau, storage=st, layout="ab") as lat:
                lat.init_case(case)
                lat.step(case.steps)
                d = lat.diagnostics()
                drift = abs(d["mass"] / d64["mass"] - 1)
                print(st, "relative mass difference to FP64 after 500 steps:", drift)
                # FP32 arithmetic drifts ~1e-11 per step; stochastic half-format
                # rounding adds unbiased noise of ~1e-3 ulp-relative per node
                assert drift < {"f32": 1e-7, "f16": 1e-5, "bf16": 1e-4}[st]
                diff, scale = lat.compare(ref)
                err[st] = diff / scale
    print("8192^2, 500 steps, rel Linf over all 604M populations vs FP64 GPU:", err)
    assert err["f32"] <= 1e-5
    assert err["f16"] <= 1e-3
    assert err["bf16"] <= 1e-2


def test_compare_finds_a_planted_difference():
    """olb_compare against a host reduction on a small lattice, including a
    planted difference and a non-finite population (read as infinity)."""
    import math

    from paper_2501_16000_gb300.engine import Lattice
    case = W.shear_64("oreg")
    with Lattice(64, 64, case.tau, storage="f64", layout="aa") as ref, \
            Lattice(64, 64, case.tau, storage="f16", layout="ab") as lat:
        for x in (ref, lat):
            x.init_case(case)
            x.step(7)
        fr, fl = ref.populations(), lat.populations()
        d, r = lat.compare(ref)
        assert d == np.abs(fl - fr).max() and r == np.abs(fr).max()
        fl[4, 10, 20] += 0.25
        lat.set_populations(fl, lat.time)
        fl = lat.populations()
        d, _ = lat.compare(ref)
        assert d == np.abs(fl - fr).max() and d > 0.2
        fl[2, 3, 4] = np.nan
        lat.set_populations(fl, lat.time)
        d, _ = lat.compare(ref)
        assert math.isinf(d)


def test_512_lattice_mix_in_the_benchmarked_batch_configuration():
    """The benchmark's batched workload (all 512 lattices of the mix, FP16)
    in the configuration the tuner picks for it on this machine (A-B, an
    oversubscribed grid, 4 warp passes per item, 200 steps per replay): a
    sample of the lattices, small and large, shear and shock, ends bitwise
    equal to the same lattice advanced alone."""
    from paper_2501_16000_gb300.batch import BatchEngine, work_items
    from paper_2501_16000_gb300.engine import Lattice
    steps = 230                                  # one full replay and part of a second
    cases = W.batch_mix(512, seed=1, steps=steps)
    R, K = 4, 200
    items = sum(work_items(c.nx, c.ny, "f16", R) for c in cases)
    by_size = sorted(range(len(cases)), key=lambda j: cases[j].nodes)
    sample = sorted(set(by_size[:3] + by_size[-3:] + by_size[250:252] +
                        [j for j in range(len(cases)) if cases[j].case == "shock"][:2]))
    with BatchEngine("f16", "ab", max_lattices=len(cases), max_items=items, steps_per_launch=K,
                     warps_per_block=2, blocks_per_sm=128, item_passes=R) as eng:
        lats = [eng.new_lattice(c) for c in cases]
        for lat in lats:
            eng.add(lat, steps)
        eng.run(2)
        eng.wait()
        got = {j: lats[j].populations() for j in sample}
        assert all(lat.time == steps for lat in lats)
        for lat in lats:
            lat.close()
    for j in sample:
        c = cases[j]
        with Lattice(c.nx, c.ny, c.tau, c.theta, c.eq, c.coll, "f16", "ab") as ref:
            ref.init_case(c)
            ref.step(steps)
            assert np.array_equal(ref.populations(), got[j]), (j, c.nx, c.ny, c.case)
