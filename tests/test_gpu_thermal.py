"""GPU parity of the guided equilibrium at each node's own temperature
(olb_params.theta_mode = OLB_THETA_LOCAL) against the FP64 CPU oracle.

Tolerances: FP64 1e-12 and FP32 1e-5 relative L_inf over all 9 canonical
populations; half formats as in test_gpu_parity.py."""
import math

import numpy as np
import pytest

from oracle import oracle as O

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


def thermal_state(nx, ny, seed, theta0=1 / 3, noise=0.01):
    """Guided equilibria of random density, velocity and temperature fields
    (theta within 15% of theta0), plus a random non-equilibrium part."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.9, 1.1, (ny, nx))
    ux, uy = rng.uniform(-0.05, 0.05, (2, ny, nx))
    th = theta0 * rng.uniform(0.85, 1.15, (ny, nx))
    f = np.empty((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            f[:, y, x] = O.feq(O.GUIDED, th[y, x], rho[y, x], ux[y, x], uy[y, x])
    return f * (1 + noise * rng.standard_normal(f.shape))


def gpu_run(f0, nx, ny, tau, theta, coll, storage, layout, steps, boundary="periodic"):
    from paper_2501_16000_gb300.engine import Lattice
    with Lattice(nx, ny, tau, theta, "guided", coll, storage, layout, boundary=boundary,
                 theta_mode="local") as lat:
        lat.set_populations(f0)
        lat.step(steps)
        return lat.populations()


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("coll", ["oreg", "bgk"])
@pytest.mark.parametrize("nx,ny,theta", [(37, 13, 1 / 3), (70, 9, 0.3), (8, 5, 0.4)])
def test_random_thermal_states(nx, ny, theta, coll, layout, storage):
    f0 = thermal_state(nx, ny, seed=nx + 100 * ny, theta0=theta)
    p = O.params(nx, ny, 0.7, theta, O.GUIDED, O.OREG if coll == "oreg" else O.BGK,
                 theta_local=True)
    want = O.run(f0, p, 41)
    err = rel_linf(gpu_run(f0, nx, ny, 0.7, theta, coll, storage, layout, 41), want)
    assert err <= TOL[storage], err


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_thermal_with_walls(layout):
    nx, ny = 133, 6
    f0 = thermal_state(nx, ny, seed=7)
    p = O.params(nx, ny, 0.6, 1 / 3, O.GUIDED, O.OREG, walls=True, theta_local=True)
    want = O.run(f0, p, 60)
    err = rel_linf(gpu_run(f0, nx, ny, 0.6, 1 / 3, "oreg", "f64", layout, 60, "walls_x"), want)
    assert err <= TOL["f64"], err


@pytest.mark.parametrize("storage,bound", [("f16", 2e-3), ("bf16", 1.6e-2)])
def test_half_precision_thermal(storage, bound):
    nx, ny = 70, 9
    f0 = thermal_state(nx, ny, seed=3)
    p = O.params(nx, ny, 0.8, 1 / 3, O.GUIDED, O.OREG, theta_local=True)
    want = O.run(f0, p, 20)
    err = rel_linf(gpu_run(f0, nx, ny, 0.8, 1 / 3, "oreg", storage, "ab", 20), want)
    assert err <= bound, err


def test_adiabatic_sound_speed_and_energy_fp64():
    """An isentropic standing density wave travels at sqrt(2 theta) on the GPU
    as in the oracle (the speeds agree to 1e-9), and BGK keeps sum <f,c^2>."""
    from paper_2501_16000_gb300.engine import Lattice
    L, steps, theta = 64, 400, 1 / 3
    x = np.arange(L)
    cs = np.cos(2 * np.pi * x / L)
    rho, th = 1 + 1e-4 * cs, theta * (1 + 1e-4 * cs)
    f0 = np.stack([np.stack([O.feq(O.GUIDED, th[i], rho[i], 0.0, 0.0) for i in range(L)], 1)] * 2,
                  1)  # (9, 2, L): two identical rows
    c2 = (O.velocities() ** 2).sum(1).astype(float)
    speeds = {}
    for coll in ("oreg", "bgk"):
        with Lattice(L, 2, 0.6, theta, "guided", coll, "f64", "aa", theta_mode="local") as lat:
            lat.set_populations(f0)
            amp = []
            for _ in range(steps + 1):
                amp.append(np.sum((lat.moments()[0][0] - 1) * cs))
                lat.step(1)
            if coll == "bgk":
                e0 = np.einsum("i,iyx->", c2, f0)
                e1 = np.einsum("i,iyx->", c2, lat.populations())
                assert abs(e1 / e0 - 1) < 1e-13, (e0, e1)
        amp = np.array(amp)
        zc = [t + amp[t] / (amp[t] - amp[t + 1]) for t in range(steps) if amp[t] * amp[t + 1] < 0]
        speeds[coll] = L / (2 * np.mean(np.diff(zc)))
        assert abs(speeds[coll] / math.sqrt(2 * theta) - 1) < 1e-3, speeds
    p = O.params(L, 2, 0.6, theta, O.GUIDED, O.OREG, theta_local=True)
    f = f0
    amp = []
    for _ in range(steps + 1):
        amp.append(np.sum((O.fields(f)[0][0] - 1) * cs))
        f = O.step(f, p)
    amp = np.array(amp)
    zc = [t + amp[t] / (amp[t] - amp[t + 1]) for t in range(steps) if amp[t] * amp[t + 1] < 0]
    assert abs(L / (2 * np.mean(np.diff(zc))) / speeds["oreg"] - 1) < 1e-9


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_with_local_temperature_equals_alone(storage):
    from paper_2501_16000_gb300 import workloads as W
    from paper_2501_16000_gb300.batch import BatchEngine
    from paper_2501_16000_gb300.engine import Lattice
    cases = [W.LatticeCase(nx=70, ny=33, tau=0.7, m=1, n=1, steps=120, theta_mode="local"),
             W.LatticeCase(nx=61, ny=40, tau=0.7, m=1, n=2, steps=120),
             W.shock_tube_walls(theta=0.35, nu=1e-3, nx=96, ny=5, steps=120)]
    alone = []
    for c in cases:
        with Lattice(c.nx, c.ny, c.tau, c.theta, c.eq, c.coll, storage, "ab",
                     boundary=c.boundary, theta_mode=c.theta_mode) as lat:
            lat.init_case(c)
            lat.step(c.steps)
            alone.append(lat.populations())
    with BatchEngine(storage, "ab", max_lattices=8, max_items=1 << 14,
                     steps_per_launch=40) as eng:
        lats = [eng.new_lattice(c) for c in cases[1:]]
        for lat, c in zip(lats, cases[1:]):
            eng.add(lat, c.steps)
        eng.run(1)
        # a local-temperature member joins a batch whose graph lacks its kernels
        late = eng.new_lattice(cases[0])
        eng.add(late, cases[0].steps)
        eng.run(3)
        eng.wait()
        assert np.array_equal(late.populations(), alone[0])
        for lat, ref in zip(lats, alone[1:]):
            assert np.array_equal(lat.populations(), ref)
        for lat in lats + [late]:
            lat.close()


def test_local_temperature_needs_guided_equilibrium():
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.engine import Lattice
    with pytest.raises(B.OregError) as e:
        Lattice(16, 16, 0.8, eq="poly2", theta_mode="local")
    assert e.value.status == B.OLB_ERR_INVALID
