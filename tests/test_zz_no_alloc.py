"""olb_diagnostics_noalloc against olb_diagnostics, through the C ABI.

olb_diagnostics_noalloc serves callers that must not have the library
allocate device memory: they account the GPU memory budget themselves (for
example a serving loop admitting work against a fixed HBM budget) or cannot
afford the device synchronisation cudaMalloc/cudaFree bring into their loop.
It reads a population state from the caller's buffer and keeps its
reduction partials in a fixed static device array shared by all calls.

This file is collected last so that a failure here comes after every other
test has run.  It must pass alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# FP64 sums over the same nodes in a different order: tolerance of the FP64
# parity tests, relative to the total mass.
REL_TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16000_gb300 import binding, build
    build.build()
    return binding.load()


def _noalloc(lib, lat, d_out):
    import torch
    st = lib.olb_diagnostics_noalloc(ctypes.c_void_p(lat._buf.data_ptr()),
                                     ctypes.byref(lat.params), lat.time,
                                     ctypes.c_void_p(d_out.data_ptr()))
    assert st == 0, lib.olb_last_error().decode()
    torch.cuda.synchronize()
    return d_out.cpu().numpy()


def _check(got, want):
    scale = abs(want["mass"])
    assert abs(got[0] - want["mass"]) <= REL_TOL * scale
    assert abs(got[1] - want["mom_x"]) <= REL_TOL * scale
    assert abs(got[2] - want["mom_y"]) <= REL_TOL * scale
    assert int(round(got[3])) == want["nonfinite"]


def _two_calls(lib, storage, layout, t1, t2, **kw):
    """Call 1 on a taller lattice (150 rows) leaves row partials that call 2,
    on a shorter one (23 rows, one planted non-finite node), must not pick
    up; both against olb_diagnostics of the same state."""
    import torch

    from paper_2501_16000_gb300.engine import Lattice

    d_out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    with Lattice(200, 150, 0.6, storage=storage, layout=layout, torch_memory=True, **kw) as a:
        a.init_shear_wave(1.0, 0.05, 2, 3)
        a.step(t1)
        _check(_noalloc(lib, a, d_out), a.diagnostics())
    with Lattice(37, 23, 0.51, storage=storage, layout=layout, torch_memory=True, **kw) as b:
        b.init_shock_tube(1.5, 0.75, 18)
        b.step(t2)
        f = b.populations()
        f[5, 11, 30] = np.nan
        b.set_populations(f, b.time)
        want = b.diagnostics(raise_nonfinite=False)
        assert want["nonfinite"] == 1
        _check(_noalloc(lib, b, d_out), want)


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
def test_noalloc_matches_diagnostics_on_two_calls_in_a_row(lib, storage, layout):
    """Every storage format (FP16 stored as g * 2^8 and decoded with its
    scale; BF16 unscaled) and both layouts, one call at an odd and one at an
    even time (the A-B buffer and the AA parity each take both values)."""
    _two_calls(lib, storage, layout, 7, 4)
    _two_calls(lib, storage, layout, 4, 7)


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_noalloc_on_wall_and_local_temperature_lattices(lib, layout):
    """Lattices with bounce-back wall columns and with the local-temperature
    guided equilibrium hold their state in the same layout; the reduction
    reads it the same way."""
    _two_calls(lib, "f16", layout, 5, 6, boundary="walls_x")
    _two_calls(lib, "f32", layout, 6, 5, theta_mode="local")


def test_noalloc_rejects_more_rows_than_its_scratch_holds(lib):
    import torch

    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.engine import make_params

    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    d_out = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = make_params(nx=8, ny=16385, tau=0.8, storage="f32")
    st = lib.olb_diagnostics_noalloc(ctypes.c_void_p(buf.data_ptr()), ctypes.byref(p), 0,
                                     ctypes.c_void_p(d_out.data_ptr()))
    assert st == B.OLB_ERR_INVALID
    assert "16384" in lib.olb_last_error().decode()
