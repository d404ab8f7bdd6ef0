"""GPU parity of the full-way bounce-back wall columns (x = 0 and x = nx - 1,
the Sec. IV shock tube) against the FP64 CPU oracle, in every layout and
storage format, alone and inside a batch.

Tolerances: FP64 1e-12 and FP32 1e-5 relative L_inf over all 9 canonical
populations, as for the periodic lattice; half formats as in
test_gpu_parity.py."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_16000_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16000_gb300 import build
    build.build()


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _eq(e):
    return O.GUIDED if e == "guided" else O.POLY2


def _coll(c):
    return O.OREG if c == "oreg" else O.BGK


def random_state(nx, ny, eq, theta, seed):
    """Equilibrium of random smooth-ish fields plus a random non-equilibrium
    part of 1% (stress and ghost modes present at every node)."""
    rng = np.random.default_rng(seed)
    p = O.params(nx, ny, 0.7, theta, _eq(eq), O.OREG, walls=True)
    f = O.init_equilibrium(p, rng.uniform(0.9, 1.1, (ny, nx)), rng.uniform(-0.05, 0.05, (ny, nx)),
                           rng.uniform(-0.05, 0.05, (ny, nx)))
    return f * (1 + 0.01 * rng.standard_normal(f.shape))


# nx - 1 at every position inside a vector of 2, 4 and 8 elements, and the
# smallest lattice with a fluid column
SIZES = [(3, 5), (8, 3), (9, 4), (37, 13), (70, 9), (133, 6)]


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("eq,coll", [("guided", "oreg"), ("guided", "bgk"), ("poly2", "oreg")])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_random_states_with_walls(nx, ny, eq, coll, layout, storage):
    from paper_2501_16000_gb300.engine import Lattice
    theta = 0.3 if eq == "guided" else 1 / 3
    f0 = random_state(nx, ny, eq, theta, seed=nx * 100 + ny)
    p = O.params(nx, ny, 0.6, theta, _eq(eq), _coll(coll), walls=True)
    steps = 41
    want = O.run(f0, p, steps)
    with Lattice(nx, ny, 0.6, theta, eq, coll, storage, layout, boundary="walls_x") as lat:
        lat.set_populations(f0)
        lat.step(steps)
        err = rel_linf(lat.populations(), want)
    assert err <= TOL[storage], err


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("theta,nu", [(0.35, 1e-5), (0.4, 1e-9)])
def test_shock_tube_between_walls_fp64(theta, nu, layout):
    """The Sec. IV shock tube (800 x 1, 500 steps) at the paper's two
    temperatures and viscosities."""
    from paper_2501_16000_gb300.engine import Lattice
    case = W.shock_tube_walls(theta=theta, nu=nu)
    p = O.params(case.nx, case.ny, case.tau, theta, O.GUIDED, O.OREG, walls=True)
    want = O.run(O.init_equilibrium(p, *case.fields()), p, case.steps)
    with Lattice(case.nx, case.ny, case.tau, theta, "guided", "oreg", "f64", layout,
                 boundary="walls_x") as lat:
        lat.init_case(case)
        lat.step(case.steps)
        err = rel_linf(lat.populations(), want)
    assert err <= TOL["f64"], err


@pytest.mark.parametrize("storage,bound", [("f16", 2e-3), ("bf16", 1.6e-2)])
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_half_precision_with_walls(storage, bound, layout):
    """Shifted half storage against the FP64 oracle on a 20-step run with
    walls: the bound is a few hundred unit roundoffs of the format relative to
    max |f| (as for the periodic lattice)."""
    from paper_2501_16000_gb300.engine import Lattice
    nx, ny = 70, 9
    f0 = random_state(nx, ny, "guided", 1 / 3, seed=5)
    p = O.params(nx, ny, 0.8, 1 / 3, O.GUIDED, O.OREG, walls=True)
    want = O.run(f0, p, 20)
    with Lattice(nx, ny, 0.8, 1 / 3, "guided", "oreg", storage, layout,
                 boundary="walls_x") as lat:
        lat.set_populations(f0)
        lat.step(20)
        err = rel_linf(lat.populations(), want)
    assert err <= bound, err


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
def test_wall_mass_is_conserved(storage):
    """Bounce-back permutes populations: total mass over all nodes is
    conserved to the format's rounding of the collision (FP64: 1e-13)."""
    from paper_2501_16000_gb300.engine import Lattice
    case = W.shock_tube_walls(theta=0.35, nu=1e-5, nx=800, ny=4)
    bound = {"f64": 1e-13, "f32": 1e-6, "f16": 1e-4, "bf16": 1e-3}[storage]
    with Lattice(case.nx, case.ny, case.tau, case.theta, storage=storage, layout="aa",
                 boundary="walls_x") as lat:
        lat.init_case(case)
        m0 = lat.diagnostics()["mass"]
        lat.step(case.steps)
        m1 = lat.diagnostics()["mass"]
    assert abs(m1 / m0 - 1) <= bound, (m0, m1)


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_batch_with_walls_equals_alone(storage, layout):
    """Wall lattices advanced inside a batch, next to periodic ones, are
    bitwise those advanced alone."""
    from paper_2501_16000_gb300.batch import BatchEngine
    from paper_2501_16000_gb300.engine import Lattice
    cases = [W.shock_tube_walls(theta=0.35, nu=1e-5, nx=203, ny=3, steps=150),
             W.LatticeCase(nx=61, ny=40, tau=0.7, m=1, n=2, steps=150),
             W.shock_tube_walls(theta=0.4, nu=1e-3, nx=96, ny=17, coll="bgk", steps=150)]
    alone = []
    for c in cases:
        with Lattice(c.nx, c.ny, c.tau, c.theta, c.eq, c.coll, storage, layout,
                     boundary=c.boundary) as lat:
            lat.init_case(c)
            lat.step(c.steps)
            alone.append(lat.populations())
    with BatchEngine(storage, layout, max_lattices=8, max_items=1 << 14,
                     steps_per_launch=50) as eng:
        lats = [eng.new_lattice(c) for c in cases]
        for lat, c in zip(lats, cases):
            eng.add(lat, c.steps)
        eng.run(3)
        eng.wait()
        for lat, ref in zip(lats, alone):
            assert eng.remaining(lat) == 0
            assert np.array_equal(lat.populations(), ref)
        for lat in lats:
            lat.close()


def test_walls_reject_narrow_lattice():
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.engine import Lattice
    with pytest.raises(B.OregError) as e:
        Lattice(2, 8, 0.8, boundary="walls_x")
    assert e.value.status == B.OLB_ERR_INVALID
