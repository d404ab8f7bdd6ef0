"""The C-ABI library builds, loads and exports every entry point that
include/oreg.h declares; host-side validation works without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2501_16000_gb300 import binding as B
from paper_2501_16000_gb300 import build as BUILD
from paper_2501_16000_gb300 import engine as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "oreg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(olb_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return B.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("olb_create_lattice", "olb_init_shear_wave", "olb_init_shock_tube",
                     "olb_step", "olb_moments", "olb_destroy", "olb_get_populations",
                     "olb_set_populations", "olb_diagnostics", "olb_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (olb_[a-z_0-9]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    # and the binding declares exactly the same names
    assert sorted(B.SIGNATURES) == declared_functions()


def test_abi_version(lib):
    assert lib.olb_abi_version() == 5


def _params(**kw):
    base = dict(nx=64, ny=32, tau=0.8, theta=1.0 / 3.0, eq="guided", coll="oreg",
                storage="f32", layout="ab", rho0=1.0)
    base.update(kw)
    return E.make_params(**base)


@pytest.mark.parametrize("storage,layout,elem,nbuf", [
    ("f64", "ab", 8, 2), ("f32", "ab", 4, 2), ("f16", "aa", 2, 1), ("bf16", "ab", 2, 2)])
def test_required_bytes(lib, storage, layout, elem, nbuf):
    p = _params(nx=37, ny=5, storage=storage, layout=layout)
    vec = 16 // elem
    pitch = (37 + vec - 1) // vec * vec
    assert lib.olb_required_bytes(ctypes.byref(p)) == nbuf * 9 * 5 * pitch * elem


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(ny=-1), dict(tau=0.5), dict(tau=float("nan")), dict(rho0=0.0),
    dict(theta=0.0), dict(theta=1.0), dict(eq="poly2", theta=0.3),
    dict(nx=1 << 20, ny=1 << 17),    # 2^37 nodes: beyond the 2^36 limit (no size_t overflow)
    dict(nx=200000, ny=200000, storage="f64")])   # 2e10 > 2^31 vectors per plane
def test_invalid_parameters_are_rejected_on_the_host(lib, bad):
    p = _params(**bad)
    assert lib.olb_required_bytes(ctypes.byref(p)) == 0
    h = ctypes.c_void_p()
    st = lib.olb_create_lattice(ctypes.byref(p), ctypes.byref(h))
    assert st == B.OLB_ERR_INVALID
    assert h.value is None
    assert lib.olb_last_error().decode()


def test_bad_enums_and_null_handles(lib):
    p = _params()
    p.storage = 7
    h = ctypes.c_void_p()
    assert lib.olb_create_lattice(ctypes.byref(p), ctypes.byref(h)) == B.OLB_ERR_INVALID
    assert lib.olb_create_lattice(None, ctypes.byref(h)) == B.OLB_ERR_INVALID
    assert lib.olb_step(None, 1) == B.OLB_ERR_INVALID
    assert lib.olb_destroy(None) == B.OLB_OK
    assert lib.olb_time(None) == -1


def test_header_compiles_as_c_and_struct_layouts_match_the_binding(tmp_path):
    """include/oreg.h is plain C99 (and C++), and the ctypes mirrors of
    olb_params / olb_batch_params have the C compiler's sizes and offsets."""
    fields = {"olb_params": [f[0] for f in B.olb_params._fields_],
              "olb_batch_params": [f[0] for f in B.olb_batch_params._fields_]}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "oreg.h"', "int main(void) {"]
    for st, names in fields.items():
        lines.append(f'    printf("{st} size %zu\\n", sizeof({st}));')
        for n in names:
            lines.append(f'    printf("{st} {n} %zu\\n", offsetof({st}, {n}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER),
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    subprocess.run(["g++", "-std=c++17", "-fsyntax-only", "-Wall", "-Werror", "-x", "c++",
                    "-I", os.path.dirname(HEADER), str(src)], check=True, capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True,
                               text=True).stdout.splitlines():
        st, name, val = line.split()
        got[(st, name)] = int(val)
    for st, cls in (("olb_params", B.olb_params), ("olb_batch_params", B.olb_batch_params)):
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for n in fields[st]:
            assert got[(st, n)] == getattr(cls, n).offset, (st, n)


@pytest.mark.parametrize("bad", [
    dict(boundary="walls_x", nx=2), dict(eq="poly2", theta_mode="local")])
def test_invalid_boundary_and_temperature_modes(lib, bad):
    p = _params(**bad)
    assert lib.olb_required_bytes(ctypes.byref(p)) == 0
    h = ctypes.c_void_p()
    assert lib.olb_create_lattice(ctypes.byref(p), ctypes.byref(h)) == B.OLB_ERR_INVALID
    p = _params()
    p.theta_mode = 5
    assert lib.olb_create_lattice(ctypes.byref(p), ctypes.byref(h)) == B.OLB_ERR_INVALID
    p = _params()
    p.boundary = -1
    assert lib.olb_create_lattice(ctypes.byref(p), ctypes.byref(h)) == B.OLB_ERR_INVALID


def test_header_enum_values_match_the_binding(tmp_path):
    """Every status, equilibrium, collision, storage, layout and option value
    the binding passes is the value the C compiler sees in include/oreg.h."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    names = re.findall(r"\b(OLB_[A-Z0-9_]+)\s*=", text)
    lines = ["#include <stdio.h>", '#include "oreg.h"', "int main(void) {"]
    lines += [f'    printf("{n} %d\\n", (int){n});' for n in names]
    lines += ["    return 0;", "}"]
    src = tmp_path / "enums.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "enums"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = dict(line.split() for line in subprocess.run(
        [str(exe)], check=True, capture_output=True, text=True).stdout.splitlines())
    mapped = {"OLB_BOUNDARY_PERIODIC": B.BOUNDARY["periodic"],
              "OLB_BOUNDARY_WALLS_X": B.BOUNDARY["walls_x"],
              "OLB_THETA_FIXED": B.THETA_MODE["fixed"], "OLB_THETA_LOCAL": B.THETA_MODE["local"]}
    for n in names:
        want = mapped[n] if n in mapped else getattr(B, n)
        assert int(got[n]) == want, n
