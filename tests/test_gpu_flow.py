"""GPU parity of the mean-flow shear wave, the first-order start of Eq. 5, the
two-quadrature mode projection and the Mach sweep of Sec. IV (Fig. 2),
against the FP64 CPU oracle.

Tolerances as in test_gpu_parity.py: FP64 1e-12 and FP32 1e-5 relative L_inf
over all 9 canonical populations."""
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


def _params(case):
    return O.params(case.nx, case.ny, case.tau, case.theta,
                    O.GUIDED if case.eq == "guided" else O.POLY2,
                    O.OREG if case.coll == "oreg" else O.BGK)


def oracle_state(case, steps):
    p = _params(case)
    rho, ux, uy = case.fields()
    if case.first_order:
        f = O.init_first_order(p, rho, ux, uy, case.gradients())
    else:
        f = O.init_equilibrium(p, rho, ux, uy)
    return O.run(f, p, steps) if steps else f


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


# ragged sizes (not multiples of any tile) with a mean flow in both axes
FLOW_CASES = [
    W.LatticeCase(nx=70, ny=37, tau=0.62, m=2, n=1, u0=0.04, ux_mean=0.05, uy_mean=-0.12,
                  first_order=True),
    W.LatticeCase(nx=70, ny=37, tau=0.62, coll="bgk", m=-1, n=2, u0=0.04, ux_mean=-0.08,
                  uy_mean=0.1, first_order=True),
    W.LatticeCase(nx=53, ny=64, tau=0.9, theta=0.3, m=1, n=1, u0=0.03, uy_mean=0.15,
                  first_order=True),
    W.LatticeCase(nx=53, ny=64, tau=0.55, eq="poly2", m=3, n=-1, u0=0.03, ux_mean=0.1,
                  first_order=True),
    W.LatticeCase(nx=64, ny=48, tau=0.7, m=1, n=2, u0=0.05, ux_mean=0.07, uy_mean=0.07),
]


def _id(c):
    return f"{c.nx}x{c.ny}-{c.eq}-{c.coll}-th{c.theta:.3f}-fo{int(c.first_order)}"


@pytest.mark.parametrize("case", FLOW_CASES, ids=_id)
def test_initial_state_matches_oracle(case):
    from paper_2501_16000_gb300.engine import Lattice
    for layout in ("ab", "aa"):
        with Lattice(case.nx, case.ny, case.tau, case.theta, case.eq, case.coll, "f64",
                     layout) as lat:
            lat.init_case(case)
            err = rel_linf(lat.populations(), oracle_state(case, 0))
            assert err <= 1e-14, (layout, err)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("case", FLOW_CASES, ids=_id)
def test_flow_runs_match_oracle(case, layout, storage):
    from paper_2501_16000_gb300.engine import Lattice
    steps = 301
    with Lattice(case.nx, case.ny, case.tau, case.theta, case.eq, case.coll, storage,
                 layout) as lat:
        lat.init_case(case)
        lat.step(steps)
        err = rel_linf(lat.populations(), oracle_state(case, steps))
    assert err <= TOL[storage], err


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
def test_wave_mode_matches_projection_of_oracle_fields(storage):
    """Both quadratures (2/N) sum u.e_perp {sin, cos}(k.x) of the GPU against the
    same sums over the oracle's velocity field, to the format's tolerance times
    the largest |u.e_perp| (the mean flow's share of each term cancels only in
    the sum, so the state's rounding enters at the scale of u, not of the
    wave amplitude)."""
    from paper_2501_16000_gb300.engine import Lattice
    case = FLOW_CASES[0]
    steps = 200
    _, vx, vy, _ = O.fields(oracle_state(case, steps))
    ph = 2 * np.pi * W.shear_wave_phase(case.nx, case.ny, case.m, case.n)
    ex, ey = W.shear_wave_direction(case.nx, case.ny, case.m, case.n)
    up = vx * ex + vy * ey
    want = (2 / case.nodes * np.sum(up * np.sin(ph)), 2 / case.nodes * np.sum(up * np.cos(ph)))
    scale = float(np.abs(up).max())
    tol = {"f64": 1e-12, "f32": 1e-5, "f16": 2e-3, "bf16": 2e-2}[storage]
    with Lattice(case.nx, case.ny, case.tau, case.theta, case.eq, case.coll, storage,
                 "aa") as lat:
        lat.init_case(case)
        lat.step(steps)
        got = lat.wave_mode(case.m, case.n)
        assert lat.wave_amplitude(case.m, case.n) == got[0]
    assert abs(got[0] - want[0]) <= tol * scale and abs(got[1] - want[1]) <= tol * scale, (
        got, want)


def test_mach_sweep_matches_oracle():
    """The GPU Mach sweep (FP64) reproduces the oracle's decay and phase rates of
    the same lattices (wavelength 64, 2000 steps) to 1e-9 relative."""
    from paper_2501_16000_gb300 import analysis
    rows = analysis.mach_sweep(machs=(0.0, 0.2, 0.4), length=64, steps=2000, every=10)
    assert len(rows) == 12
    for r in rows:
        case = W.mach_wave(r["geometry"], r["mach"], r["coll"], length=64, steps=2000)
        p = _params(case)
        f = oracle_state(case, 0)
        ph = 2 * np.pi * W.shear_wave_phase(case.nx, case.ny, case.m, case.n)
        sn, cs = np.sin(ph), np.cos(ph)
        ex, ey = W.shear_wave_direction(case.nx, case.ny, case.m, case.n)
        ts, a_s, a_c = [], [], []
        for t in range(0, case.steps + 1, 10):
            _, vx, vy, _ = O.fields(f)
            up = vx * ex + vy * ey
            ts.append(t)
            a_s.append(2 / case.nodes * np.sum(up * sn))
            a_c.append(2 / case.nodes * np.sum(up * cs))
            if t < case.steps:
                f = O.run(f, p, 10)
        gamma, omega = analysis.fit_wave(ts, a_s, a_c, case.tau)
        assert abs(r["gamma"] / gamma - 1) <= 1e-9, (r, gamma)
        assert abs(r["omega"] - omega) <= 1e-9 * max(abs(omega), 1e-6), (r, omega)
        if r["geometry"] == "axis":
            assert abs(r["nu_ratio"] - 1) < 2e-3, r


def test_init_shear_flow_rejects_bad_arguments():
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.engine import Lattice
    with Lattice(16, 16, 0.8) as lat:
        for args in ((1.0, 0.05, 0, 0, 0.0, 0.0, 0), (1.0, 0.05, 1, 0, float("nan"), 0.0, 0),
                     (1.0, 0.05, 1, 0, 0.0, 0.0, 2), (-1.0, 0.05, 1, 0, 0.0, 0.0, 1)):
            with pytest.raises(B.OregError) as e:
                B.call("olb_init_shear_flow", lat.handle, *args)
            assert e.value.status == B.OLB_ERR_INVALID
        with pytest.raises(B.OregError):
            B.call("olb_wave_mode", lat.handle, 1, 0, None, None)
