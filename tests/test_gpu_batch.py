"""Batched path on the GPU: every lattice advanced in a mixed batch (uneven
sizes, own tau/theta/equilibrium/collision, joining at different rounds,
finishing at different steps) ends bitwise equal to the same lattice advanced
alone with olb_step; and the FP64 batch matches the FP64 oracle."""
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


def mixed_cases():
    cases = W.batch_mix(count=12, seed=7, lo=5, hi=300, steps=0)
    extra = [W.LatticeCase(nx=37, ny=3, tau=0.7, theta=0.35, coll="bgk", case="shear", u0=0.03,
                           m=1, n=1),
             W.LatticeCase(nx=130, ny=9, tau=0.55, eq="poly2", case="shock", x_split=40),
             W.LatticeCase(nx=1, ny=7, tau=0.9, case="shear", m=0, n=1, u0=0.02)]
    return cases + extra


@pytest.mark.parametrize("blocks", [0, 256])           # every block resident / oversubscribed
@pytest.mark.parametrize("storage", ["f16", "f32", "bf16"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_batch_equals_alone_bitwise(storage, layout, blocks):
    from paper_2501_16000_gb300.batch import BatchEngine
    from paper_2501_16000_gb300.engine import Lattice
    cases = mixed_cases()
    K = 7
    steps = [5 + 3 * j for j in range(len(cases))]        # odd and even totals, mid-round ends
    with BatchEngine(storage, layout, max_lattices=64, max_items=1 << 16, steps_per_launch=K,
                     warps_per_block=4, blocks_per_sm=blocks) as eng:
        lats = []
        for j, c in enumerate(cases):
            lat = eng.new_lattice(c)
            lats.append(lat)
            if j % 3 != 2:
                eng.add(lat, steps[j])
        eng.run(1)                                       # some join one round late
        for j, lat in enumerate(lats):
            if j % 3 == 2:
                eng.add(lat, steps[j])
        rounds = max(steps) // K + 2
        eng.run(rounds)
        eng.wait()
        for j, lat in enumerate(lats):
            assert lat.time == steps[j]
            assert eng.remaining(lat) == 0
        got = [lat.populations() for lat in lats]
        for lat in lats:
            lat.close()
    for j, c in enumerate(cases):
        with Lattice(c.nx, c.ny, c.tau, c.theta, c.eq, c.coll, storage, layout) as ref:
            ref.init_case(c)
            ref.step(steps[j])
            assert np.array_equal(ref.populations(), got[j]), (j, c)


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_many_slots_overlap_and_stay_bitwise(layout):
    """Ten constant classes (theta 0.30 .. 0.39, alternating OReg and BGK), more
    slots than the graph's side streams: the slots' launches run on streams
    forked from the batch stream, two slots share a stream, and every lattice
    still ends bitwise equal to its run alone."""
    from paper_2501_16000_gb300.batch import BatchEngine
    from paper_2501_16000_gb300.engine import Lattice
    cases = [W.LatticeCase(nx=40 + 13 * j, ny=9 + 5 * j, tau=0.55 + 0.03 * j, theta=0.30 + 0.01 * j,
                           coll="bgk" if j % 2 else "oreg", case="shear", u0=0.04, m=1, n=1)
             for j in range(10)]
    steps = 2 * 6 + 3
    with BatchEngine("f16", layout, max_lattices=16, max_items=1 << 14, steps_per_launch=6,
                     warps_per_block=4, blocks_per_sm=32) as eng:
        lats = [eng.new_lattice(c) for c in cases]
        for lat in lats:
            eng.add(lat, steps)
        eng.run(3)
        eng.wait()
        got = [lat.populations() for lat in lats]
        for lat in lats:
            assert lat.time == steps
            lat.close()
    for c, g in zip(cases, got):
        with Lattice(c.nx, c.ny, c.tau, c.theta, c.eq, c.coll, "f16", layout) as ref:
            ref.init_case(c)
            ref.step(steps)
            assert np.array_equal(ref.populations(), g), c


def test_bounded_wait_reports_running_rounds():
    """olb_batch_wait_for returns OLB_ERR_TIMEOUT (False here) while enqueued
    rounds are still running, without cancelling them; a later wait finishes
    and the lattice has advanced every enqueued step, as without the timeout."""
    from paper_2501_16000_gb300.batch import BatchEngine
    from paper_2501_16000_gb300.engine import Lattice
    case = W.LatticeCase(nx=4096, ny=4096, tau=0.8, case="shear", u0=0.05, m=1, n=1)
    with BatchEngine("f32", "ab", max_lattices=2, max_items=1 << 16, steps_per_launch=50) as eng:
        lat = eng.new_lattice(case)
        eng.add(lat, 1000)
        eng.run(20)                      # 1000 steps of 16.8 M nodes, ~0.2 s of work
        assert eng.wait(timeout=0.0) is False
        assert eng.wait(timeout=60.0) is True
        assert lat.time == 1000 and eng.remaining(lat) == 0
        got = lat.diagnostics()
        lat.close()
    with Lattice(case.nx, case.ny, case.tau, storage="f32", layout="ab") as ref:
        ref.init_case(case)
        ref.step(1000)
        want = ref.diagnostics()
    assert got == want


def test_batch_fp64_matches_oracle():
    from paper_2501_16000_gb300.batch import BatchEngine
    cases = mixed_cases()[:6]
    with BatchEngine("f64", "aa", max_lattices=16, max_items=1 << 14, steps_per_launch=10) as eng:
        lats = [eng.new_lattice(c) for c in cases]
        for lat in lats:
            eng.add(lat, 23)
        eng.run(3)
        eng.wait()
        for lat, c in zip(lats, cases):
            p = O.params(c.nx, c.ny, c.tau, c.theta, O.GUIDED if c.eq == "guided" else O.POLY2,
                         O.OREG if c.coll == "oreg" else O.BGK)
            ref = O.run(O.init_equilibrium(p, *c.fields()), p, 23)
            err = np.abs(lat.populations() - ref).max() / np.abs(ref).max()
            assert err <= 1e-12, (c, err)
            lat.close()


def test_batch_membership_rules():
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.batch import BatchEngine
    from paper_2501_16000_gb300.engine import Lattice
    with BatchEngine("f16", "ab", max_lattices=2, max_items=64, steps_per_launch=4) as eng:
        c = W.LatticeCase(nx=64, ny=8, tau=0.8, case="shear", m=1, n=1)
        a = eng.new_lattice(c)
        eng.add(a, 8)
        with pytest.raises(B.OregError) as e:      # members advance only with the batch
            a.step(1)
        assert e.value.status == B.OLB_ERR_STATE
        with pytest.raises(B.OregError) as e:      # same storage/layout required
            other = Lattice(64, 8, 0.8, storage="f32", layout="ab", stream=eng.stream)
            eng.add(other, 1)
        other.close()
        # 256 x 400 f16: 400 warp passes, 100 items of 4 passes > 64
        big = eng.new_lattice(W.LatticeCase(nx=256, ny=400, tau=0.8, case="shock", x_split=10))
        with pytest.raises(B.OregError) as e:      # work-item capacity
            eng.add(big, 1)
        assert e.value.status == B.OLB_ERR_NOMEM
        big.close()
        eng.run(3)
        eng.wait()
        assert a.time == 8
        eng.remove(a)
        a.step(1)                                  # free again after removal
        assert a.time == 9
        a.close()


def test_nonfinite_member_stays_isolated():
    """A NaN planted in one member's populations spreads only through that
    lattice: the other members of the batch end bitwise equal to their runs
    alone, and the poisoned one reports its non-finite nodes."""
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.batch import BatchEngine
    from paper_2501_16000_gb300.engine import Lattice
    cases = [W.LatticeCase(nx=61, ny=40, tau=0.7, m=1, n=2, steps=60),
             W.LatticeCase(nx=96, ny=33, tau=0.8, m=2, n=1, steps=60),
             W.LatticeCase(nx=45, ny=70, tau=0.6, case="shock", x_split=20, steps=60)]
    alone = {}
    for j in (0, 2):
        c = cases[j]
        with Lattice(c.nx, c.ny, c.tau, c.theta, storage="f16", layout="aa") as lat:
            lat.init_case(c)
            lat.step(c.steps)
            alone[j] = lat.populations()
    with BatchEngine("f16", "aa", max_lattices=4, max_items=1 << 12, steps_per_launch=20) as eng:
        lats = [eng.new_lattice(c) for c in cases]
        f = lats[1].populations()
        f[4, 10, 30] = np.nan
        lats[1].set_populations(f)
        for lat, c in zip(lats, cases):
            eng.add(lat, c.steps)
        eng.run(3)
        eng.wait()
        for j in (0, 2):
            assert np.array_equal(lats[j].populations(), alone[j])
            assert lats[j].diagnostics()["nonfinite"] == 0
        with pytest.raises(B.OregError) as e:
            lats[1].diagnostics()
        assert e.value.status == B.OLB_ERR_NONFINITE
        assert lats[1].diagnostics(raise_nonfinite=False)["nonfinite"] > 100
        for lat in lats:
            lat.close()


def test_batch_rejects_a_grid_beyond_256_blocks_per_sm():
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.batch import BatchEngine
    with pytest.raises(B.OregError) as e:
        BatchEngine("f16", "ab", max_lattices=4, max_items=1 << 12, blocks_per_sm=257)
    assert e.value.status == B.OLB_ERR_INVALID


def test_batch_rejects_a_lattice_with_the_fp64_collision():
    """OLB_OPT_F64_COLLISION is a single-lattice mode: olb_batch_add refuses
    such a lattice, and accepts it once the option is off again."""
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.batch import BatchEngine
    with BatchEngine("f32", "ab", max_lattices=4, max_items=1 << 12, steps_per_launch=4,
                     warps_per_block=4) as eng:
        lat = eng.new_lattice(W.shear_64("oreg"))
        lat.set_option(B.OLB_OPT_F64_COLLISION, 1)
        with pytest.raises(B.OregError) as e:
            eng.add(lat, 8)
        assert e.value.status == B.OLB_ERR_INVALID
        lat.set_option(B.OLB_OPT_F64_COLLISION, 0)
        eng.add(lat, 8)
        eng.run(3)
        eng.wait()
        assert lat.time == 8 and eng.remaining(lat) == 0
        lat.close()
