"""GPU parity: the CUDA stream-collide path (through the C ABI) against the
FP64 CPU oracle, element by element on the canonical populations.

Tolerances (relative L_inf over all 9 populations, normalised by max |f|):
FP64 1e-12 and FP32 1e-5 after the stated step counts; the half-precision
storage formats are checked against bounds derived from their unit roundoff
(see test docstrings)."""
import functools

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


def _oracle_params(case):
    return O.params(case.nx, case.ny, case.tau, case.theta,
                    O.GUIDED if case.eq == "guided" else O.POLY2,
                    O.OREG if case.coll == "oreg" else O.BGK)


@functools.lru_cache(maxsize=None)
def oracle_run(case, steps):
    p = _oracle_params(case)
    f0 = O.init_equilibrium(p, *case.fields())
    return O.run(f0, p, steps)


def gpu_run(case, steps, storage, layout, split=None, comp=None, f64_coll=None):
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.engine import Lattice
    with Lattice(case.nx, case.ny, case.tau, case.theta, case.eq, case.coll, storage,
                 layout) as lat:
        if comp is not None:
            lat.set_option(B.OLB_OPT_COMPENSATED, comp)
        if f64_coll is not None:
            lat.set_option(B.OLB_OPT_F64_COLLISION, f64_coll)
        lat.init_case(case)
        if split:
            for k in split:
                lat.step(k)
        else:
            lat.step(steps)
        assert lat.time == steps
        return lat.populations()


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


SHEAR_64 = [W.shear_64("oreg"), W.shear_64("bgk"), W.shear_64("oreg", 1, 1)]
SHOCK_2048X4 = [W.shock_2048x4("guided"), W.shock_2048x4("poly2")]


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("case", SHEAR_64, ids=lambda c: f"shear64-{c.coll}-{c.m}{c.n}")
def test_shear_wave_64x64_fp64(case, layout):
    err = rel_linf(gpu_run(case, case.steps, "f64", layout), oracle_run(case, case.steps))
    assert err <= TOL["f64"], err


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("case", SHOCK_2048X4, ids=lambda c: f"shock-{c.eq}")
def test_shock_tube_2048x4_fp64(case, layout):
    err = rel_linf(gpu_run(case, case.steps, "f64", layout), oracle_run(case, case.steps))
    assert err <= TOL["f64"], err


@pytest.mark.parametrize("case", SHEAR_64[:2], ids=lambda c: f"shear64-{c.coll}")
def test_shear_wave_64x64_fp32(case):
    err = rel_linf(gpu_run(case, case.steps, "f32", "ab"), oracle_run(case, case.steps))
    assert err <= TOL["f32"], err


# The FP32 shock tube at tau = 0.51 (nu = 3.3e-3) over 2000 steps, the
# weakest-damped case: FP32 storage with the default exact conserved sums
# (OLB_OPT_COMPENSATED = 1) must stay within 1e-5 of the FP64 oracle at
# t = 2000 and t = 500, both layouts.  Plain sums (option 0) end ~3e-5 away
# after 2000 steps (their rounding repeats identically over the uniform
# states); they are held to 1e-5 at t = 500 only, before the periodic waves
# meet.
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("case", SHOCK_2048X4, ids=lambda c: f"shock-{c.eq}")
def test_shock_tube_2048x4_fp32(case, layout):
    for steps in (case.steps, 500):
        err = rel_linf(gpu_run(case, steps, "f32", layout), oracle_run(case, steps))
        print(f"FP32 shock {case.eq} {layout} t={steps}: rel Linf {err:.3e}")
        assert err <= TOL["f32"], (steps, err)


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("case", SHOCK_2048X4, ids=lambda c: f"shock-{c.eq}")
def test_shock_tube_2048x4_fp32_plain_sums_t500(case, layout):
    err = rel_linf(gpu_run(case, 500, "f32", layout, comp=0), oracle_run(case, 500))
    print(f"FP32 plain sums shock {case.eq} {layout} t=500: rel Linf {err:.3e}")
    assert err <= TOL["f32"], err


# FP32 storage with the collision in FP64 (OLB_OPT_F64_COLLISION): the store
# is the only FP32 rounding of a step.  Emulating exactly that on the CPU (the
# oracle's FP64 step, then g = f - s rounded to FP32) gives 4.3e-6 (guided)
# and 4.4e-6 (polynomial) after 2000 steps, so this mode meets 1e-5 where the
# FP32 collision does not.
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("case", SHOCK_2048X4, ids=lambda c: f"shock-{c.eq}")
def test_shock_tube_2048x4_fp32_storage_fp64_collision(case, layout):
    err = rel_linf(gpu_run(case, case.steps, "f32", layout, f64_coll=1),
                   oracle_run(case, case.steps))
    print(f"FP32 storage / FP64 collision shock {case.eq} {layout} t=2000: rel Linf {err:.3e}")
    assert err <= TOL["f32"], err


@pytest.mark.parametrize("case", SHEAR_64, ids=lambda c: f"shear64-{c.coll}-{c.m}{c.n}")
def test_shear_wave_64x64_fp32_storage_fp64_collision(case):
    err = rel_linf(gpu_run(case, case.steps, "f32", "aa", f64_coll=1),
                   oracle_run(case, case.steps))
    assert err <= TOL["f32"], err


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("theta_mode", ["fixed", "local"])
def test_fp64_collision_random_states_every_kernel_kind(walls, theta_mode):
    """Random non-equilibrium states through the FP64-collision kernels with
    and without wall columns and local temperature, A-B and AA, switching the
    option on and off between steps (the stored state is the same), against
    the oracle after each call."""
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.engine import Lattice
    nx, ny, tau, theta = 131, 7, 0.7, 0.35
    f0 = random_state(nx, ny, "guided", theta, seed=11)
    p = O.params(nx, ny, tau, theta, O.GUIDED, O.OREG, walls=walls,
                 theta_local=theta_mode == "local")
    for layout in ("ab", "aa"):
        with Lattice(nx, ny, tau, theta, "guided", "oreg", "f32", layout,
                     boundary="walls_x" if walls else "periodic", theta_mode=theta_mode) as lat:
            lat.set_populations(f0, 0)
            ref = f0
            for steps, on in ((1, 1), (2, 0), (5, 1), (3, 1)):
                lat.set_option(B.OLB_OPT_F64_COLLISION, on)
                lat.step(steps)
                ref = O.run(ref, p, steps)
                err = rel_linf(lat.populations(), ref)
                assert err <= 1e-6, (layout, lat.time, on, err)


def test_fp64_collision_option_validation():
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.engine import Lattice
    for storage in ("f64", "f16", "bf16"):
        with Lattice(16, 8, 0.8, storage=storage) as lat:
            with pytest.raises(B.OregError) as e:
                lat.set_option(B.OLB_OPT_F64_COLLISION, 1)
            assert e.value.status == B.OLB_ERR_INVALID
            lat.set_option(B.OLB_OPT_F64_COLLISION, 0)
    with Lattice(16, 8, 0.8, storage="f32") as lat:
        with pytest.raises(B.OregError) as e:
            lat.set_option(B.OLB_OPT_F64_COLLISION, 2)
        assert e.value.status == B.OLB_ERR_INVALID


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
def test_block_size_does_not_change_results(storage, layout):
    """OLB_OPT_WARPS_PER_BLOCK only changes how warp passes map to blocks
    (and, for the half formats, whether the register-capped A-B kernel runs):
    results are bitwise the same for 1, 2, 4 and 8 warps per block."""
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.engine import Lattice
    nx, ny = 131, 23
    f0 = random_state(nx, ny, "guided", 1.0 / 3.0, seed=5)
    got = {}
    for w in (1, 2, 4, 8):
        with Lattice(nx, ny, 0.7, storage=storage, layout=layout) as lat:
            lat.set_option(B.OLB_OPT_WARPS_PER_BLOCK, w)
            lat.set_populations(f0, 0)
            lat.step(5)
            got[w] = lat.populations()
    for w in (1, 2, 8):
        assert np.array_equal(got[w], got[4]), w


def test_theta_off_reference_fp64():
    case = W.LatticeCase(nx=48, ny=40, tau=0.6, theta=0.3, case="shear", u0=0.05, m=2, n=1)
    err = rel_linf(gpu_run(case, 300, "f64", "aa"), oracle_run(case, 300))
    assert err <= TOL["f64"], err


# ---------------------------------------------------------------------------
# ragged sizes, odd and even step counts, random non-equilibrium states
# ---------------------------------------------------------------------------

def random_state(nx, ny, eq, theta, seed):
    """Equilibrium of a random smooth-ish field plus a random non-equilibrium
    part, all positive."""
    rng = np.random.default_rng(seed)
    p = O.params(nx, ny, 0.7, theta, O.GUIDED if eq == "guided" else O.POLY2, O.OREG)
    rho = 1.0 + 0.1 * rng.uniform(-1, 1, (ny, nx))
    ux = 0.08 * rng.uniform(-1, 1, (ny, nx))
    uy = 0.08 * rng.uniform(-1, 1, (ny, nx))
    f = O.init_equilibrium(p, rho, ux, uy)
    return f * (1.0 + 0.02 * rng.uniform(-1, 1, f.shape))


SIZES = [(1, 1), (1, 5), (5, 1), (3, 2), (37, 23), (131, 7), (257, 3), (520, 4)]


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_ragged_random_states(nx, ny, layout, storage):
    from paper_2501_16000_gb300.engine import Lattice
    for eq, coll, theta in (("guided", "oreg", 0.35), ("poly2", "bgk", 1.0 / 3.0)):
        f0 = random_state(nx, ny, eq, theta, seed=nx * 1000 + ny)
        p = O.params(nx, ny, 0.7, theta, O.GUIDED if eq == "guided" else O.POLY2,
                     O.OREG if coll == "oreg" else O.BGK)
        with Lattice(nx, ny, 0.7, theta, eq, coll, storage, layout) as lat:
            lat.set_populations(f0, 0)
            ref = f0
            for steps in (1, 1, 5, 2):      # even and odd times, AA parity both ways
                lat.step(steps)
                ref = O.run(ref, p, steps)
                err = rel_linf(lat.populations(), ref)
                assert err <= TOL[storage] * (1 if storage == "f64" else 0.1), \
                    (eq, coll, lat.time, err)


@pytest.mark.parametrize("storage,bound", [("f16", 2e-3), ("bf16", 1.6e-2)])
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_half_precision_storage_short_runs(storage, bound, layout):
    """Shifted half storage: each step rounds g = f - s to 11 (f16) or 8 (bf16)
    significant bits, |g| <= ~0.15 here, so a few steps stay within a few
    half-ulps of max|g| relative to max|f| (bound = 4 ulp * 0.15 / 0.44)."""
    from paper_2501_16000_gb300.engine import Lattice
    nx, ny = 131, 7
    f0 = random_state(nx, ny, "guided", 1.0 / 3.0, seed=3)
    p = O.params(nx, ny, 0.7, 1.0 / 3.0, O.GUIDED, O.OREG)
    with Lattice(nx, ny, 0.7, storage=storage, layout=layout) as lat:
        lat.set_populations(f0, 0)
        lat.step(3)
        err = rel_linf(lat.populations(), O.run(f0, p, 3))
    assert err <= bound, err


@pytest.mark.parametrize("storage,bound", [("f16", 2e-3), ("bf16", 1.6e-2)])
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_half_precision_ragged_sizes(nx, ny, layout, storage, bound):
    """The half formats on every ragged size (single nodes, single rows and
    columns, partial vectors, warp passes spanning rows) against the oracle, within the same
    few-ulp bounds as the short-run test above, at even and odd times."""
    from paper_2501_16000_gb300.engine import Lattice
    f0 = random_state(nx, ny, "guided", 1.0 / 3.0, seed=nx * 7 + ny)
    p = O.params(nx, ny, 0.7, 1.0 / 3.0, O.GUIDED, O.OREG)
    with Lattice(nx, ny, 0.7, storage=storage, layout=layout) as lat:
        lat.set_populations(f0, 0)
        ref = f0
        for steps in (1, 2):
            lat.step(steps)
            ref = O.run(ref, p, steps)
            err = rel_linf(lat.populations(), ref)
            assert err <= bound, (lat.time, err)


# ---------------------------------------------------------------------------
# state plumbing: round trips, checkpoint/resume, moments, diagnostics
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_set_get_roundtrip(storage, layout):
    from paper_2501_16000_gb300.engine import Lattice
    f0 = random_state(37, 11, "guided", 1.0 / 3.0, seed=1)
    with Lattice(37, 11, 0.8, storage=storage, layout=layout) as lat:
        for t in (0, 1):           # even and odd AA parity
            lat.set_populations(f0, t)
            got = lat.populations()
            if storage == "f64":
                assert np.array_equal(got, f0)
            else:
                eps = {"f32": 2 ** -24, "f16": 2 ** -11, "bf16": 2 ** -8}[storage]
                assert np.abs(got - f0).max() <= eps * 0.5 + 1e-12


def test_failed_allocation_is_reported_and_harmless():
    """A lattice larger than the GPU's memory (the library allocating its
    populations) and a batch with an impossible item table fail with
    OLB_ERR_NOMEM and a message; afterwards a normal lattice still steps and
    matches the oracle (the failed allocation leaves no error behind)."""
    import ctypes

    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.engine import make_params
    lib = B.load()
    p = make_params(nx=60000, ny=60000, tau=0.8, storage="f64")        # ~518 GB of populations
    h = ctypes.c_void_p()
    assert lib.olb_create_lattice(ctypes.byref(p), ctypes.byref(h)) == B.OLB_ERR_NOMEM
    assert "allocating" in lib.olb_last_error().decode()
    bp = B.olb_batch_params(B.OLB_F16_SHIFTED, B.OLB_LAYOUT_AB, 4, 1 << 40, 4, 4, 0, None, 0)
    hb = ctypes.c_void_p()
    assert lib.olb_batch_create(ctypes.byref(bp), ctypes.byref(hb)) == B.OLB_ERR_NOMEM
    case = SHEAR_64[0]
    err = rel_linf(gpu_run(case, 20, "f32", "ab"), oracle_run(case, 20))
    assert err <= TOL["f32"], err


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_checkpoint_resume_is_bitwise(layout):
    from paper_2501_16000_gb300.engine import Lattice
    case = W.shear_64("oreg")
    with Lattice(64, 64, case.tau, storage="f32", layout=layout) as a:
        a.init_case(case)
        a.step(37)
        ck = a.populations()
        a.step(20)
        straight = a.populations()
    with Lattice(64, 64, case.tau, storage="f32", layout=layout) as b:
        b.set_populations(ck, 37)
        b.step(20)
        assert np.array_equal(b.populations(), straight)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("variant", ["periodic", "walls", "local_theta", "poly2_bgk"])
def test_ab_and_aa_layouts_give_bitwise_the_same_states(storage, variant):
    """The layout is hidden behind the calls: the same state advanced with the
    two-buffer A-B kernels and with the in-place AA kernels (even and odd
    steps) is bitwise the same after an odd and after an even number of
    steps, on ragged sizes whose warp passes span rows."""
    from paper_2501_16000_gb300.engine import Lattice
    kw = dict(eq="poly2", coll="bgk") if variant == "poly2_bgk" else {}
    if variant == "walls":
        kw["boundary"] = "walls_x"
    if variant == "local_theta":
        kw["theta_mode"] = "local"
    for (nx, ny) in ((37, 23), (131, 7), (520, 4)):
        f0 = random_state(nx, ny, kw.get("eq", "guided"), 1.0 / 3.0, seed=3 * nx + ny)
        for steps in (7, 12):
            got = {}
            for layout in ("ab", "aa"):
                with Lattice(nx, ny, 0.6, storage=storage, layout=layout, **kw) as lat:
                    lat.set_populations(f0, 0)
                    lat.step(steps)
                    got[layout] = lat.populations()
            assert np.array_equal(got["ab"], got["aa"]), (nx, ny, steps)


def test_moments_and_diagnostics_match_oracle():
    from paper_2501_16000_gb300.engine import Lattice
    case = W.shear_64("oreg")
    ref = oracle_run(case, 100)
    rho_o, ux_o, uy_o, th_o = O.fields(ref)
    with Lattice(64, 64, case.tau, storage="f64", layout="aa") as lat:
        lat.init_case(case)
        lat.step(100)
        rho, ux, uy, th = lat.moments(theta_loc=True)
        d = lat.diagnostics()
        amp = lat.wave_amplitude(case.m, case.n)
    for a, b in ((rho, rho_o), (ux, ux_o), (uy, uy_o), (th, th_o)):
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())
    assert abs(d["mass"] - rho_o.sum()) <= 1e-11
    assert abs(d["mom_x"] - (rho_o * ux_o).sum()) <= 1e-11
    assert d["nonfinite"] == 0
    s = np.sin(2 * np.pi * W.shear_wave_phase(64, 64, case.m, case.n))
    ex, ey = W.shear_wave_direction(64, 64, case.m, case.n)
    amp_o = 2.0 / 4096 * np.sum((ux_o * ex + uy_o * ey) * s)
    assert abs(amp - amp_o) <= 1e-12


def test_init_fields_matches_analytic_init():
    from paper_2501_16000_gb300.engine import Lattice
    case = W.shear_64("oreg")
    with Lattice(64, 64, case.tau, storage="f64") as a, Lattice(64, 64, case.tau, storage="f64") as b:
        a.init_case(case)
        b.init_fields(*case.fields())
        assert rel_linf(a.populations(), b.populations()) <= 1e-15


def test_mass_conservation_fp64():
    from paper_2501_16000_gb300.engine import Lattice
    case = W.shock_2048x4()
    with Lattice(case.nx, case.ny, case.tau, storage="f64", layout="aa") as lat:
        lat.init_case(case)
        m0 = lat.diagnostics()["mass"]
        lat.step(1000)
        d = lat.diagnostics()
    assert abs(d["mass"] / m0 - 1) <= 1e-13
    assert abs(d["mom_y"]) <= 1e-10


# ---------------------------------------------------------------------------
# error paths made on the host (no GPU fault)
# ---------------------------------------------------------------------------

def test_error_paths():
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.engine import Lattice
    lat = Lattice(16, 8, 0.8, storage="f32")
    with pytest.raises(B.OregError) as e:
        lat.step(1)                      # before any init
    assert e.value.status == B.OLB_ERR_STATE
    lat.init_shear_wave(1.0, 0.05, 1, 0)
    with pytest.raises(B.OregError) as e:
        lat.step(-1)
    assert e.value.status == B.OLB_ERR_INVALID
    f = lat.populations()
    f[3, 2, 5] = np.nan                  # a non-finite value injected from the host
    lat.set_populations(f, 4)
    with pytest.raises(B.OregError) as e:
        lat.diagnostics()
    assert e.value.status == B.OLB_ERR_NONFINITE
    assert lat.diagnostics(raise_nonfinite=False)["nonfinite"] == 1
    lat.close()
