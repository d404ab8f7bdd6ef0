"""Builds liboreg.so (the CUDA library behind include/oreg.h) in-tree for sm_103a.

Translation units are compiled in parallel with nvcc and linked into
``paper_2501_16000_gb300/_build/liboreg.so``.  The FP64 unit is compiled
without fused multiply-add contraction: the FP64 path exists to match the
FP64 oracle, which is compiled the same way.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboreg.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
          "-I" + CSRC, "--expt-relaxed-constexpr"]
UNITS = {
    "oreg_api.cu": [],
    "oreg_st_f64.cu": ["-fmad=false"],
    "oreg_st_f32.cu": [],
    "oreg_st_f16.cu": [],
    "oreg_st_bf16.cu": [],
    "oreg_st_f32c64.cu": [],
    "oreg_batch.cu": [],
    "oreg_noalloc.cu": [],
    "oreg_compare.cu": [],
}


def nvcc() -> str:
    for cand in (os.environ.get("CUDACXX"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liboreg.so")


def _sources_newer_than(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "oreg.h")]
    return any(os.path.getmtime(f) > t for f in files if os.path.isfile(f))


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile and link liboreg.so; returns its path.  Rebuilds when any
    source is newer than the library (or when force is set)."""
    if not force and not _sources_newer_than(LIB):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    extra = list(extra or [])
    units = {u: f for u, f in UNITS.items() if os.path.exists(os.path.join(CSRC, u))}
    tmpdir = tempfile.mkdtemp(prefix="oreg_build_", dir=BUILD)
    try:
        procs = []
        objs = []
        for unit, flags in units.items():
            obj = os.path.join(tmpdir, unit.replace(".cu", ".o"))
            cmd = [cc, *ARCH, *COMMON, *flags, *extra, "-c", os.path.join(CSRC, unit), "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                 stderr=subprocess.STDOUT, text=True)))
            objs.append(obj)
        errors = []
        for unit, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                errors.append(f"--- {unit} ---\n{out}")
            elif verbose and out:
                print(out, file=sys.stderr)
        if errors:
            raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
        tmp_lib = os.path.join(tmpdir, "liboreg.so")
        link = [cc, *ARCH, "-shared", "-o", tmp_lib, *objs]
        r = subprocess.run(link, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp_lib, LIB)
    finally:
        shutil.rmtree(tmpdir, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
