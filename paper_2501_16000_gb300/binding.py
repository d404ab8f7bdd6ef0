"""ctypes binding of liboreg.so: the C ABI of include/oreg.h under the same names.

Argument marshalling only: every step of the computation runs in the CUDA
library.  ``load()`` raises when the library has not been built; there is no
fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

OLB_OK, OLB_ERR_INVALID, OLB_ERR_NOMEM, OLB_ERR_CUDA = 0, 1, 2, 3
OLB_ERR_NONFINITE, OLB_ERR_TIMEOUT, OLB_ERR_STATE = 4, 5, 6
OLB_EQ_GUIDED, OLB_EQ_POLY2 = 0, 1
OLB_COLL_OREG, OLB_COLL_BGK = 0, 1
OLB_F64, OLB_F32, OLB_F16_SHIFTED, OLB_BF16_SHIFTED = 0, 1, 2, 3
OLB_LAYOUT_AB, OLB_LAYOUT_AA = 0, 1
OLB_OPT_COMPENSATED, OLB_OPT_WARPS_PER_BLOCK, OLB_OPT_STOCHASTIC_ROUNDING = 1, 2, 3
OLB_OPT_F64_COLLISION = 4

STATUS_NAMES = {0: "OLB_OK", 1: "OLB_ERR_INVALID", 2: "OLB_ERR_NOMEM", 3: "OLB_ERR_CUDA",
                4: "OLB_ERR_NONFINITE", 5: "OLB_ERR_TIMEOUT", 6: "OLB_ERR_STATE"}


class OregError(RuntimeError):
    """A liboreg call returned a status other than OLB_OK."""

    def __init__(self, status: int, message: str, call: str):
        super().__init__(f"{call}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class OregLibraryMissing(RuntimeError):
    pass


class olb_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("tau", ctypes.c_double), ("theta", ctypes.c_double),
                ("rho0", ctypes.c_double),
                ("eq", ctypes.c_int32), ("coll", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("device_buffer", ctypes.c_void_p), ("buffer_bytes", ctypes.c_size_t),
                ("cuda_stream", ctypes.c_void_p), ("boundary", ctypes.c_int32),
                ("theta_mode", ctypes.c_int32)]


ABI_VERSION = 5
BOUNDARY = {"periodic": 0, "walls_x": 1}
THETA_MODE = {"fixed": 0, "local": 1}


class olb_batch_params(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("max_lattices", ctypes.c_int32), ("max_items", ctypes.c_int64),
                ("steps_per_launch", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p),
                ("item_passes", ctypes.c_int32)]


_P = ctypes.POINTER
_d = _P(ctypes.c_double)
_h = ctypes.c_void_p

# name -> (restype, argtypes); the ABI of include/oreg.h
SIGNATURES = {
    "olb_abi_version": (ctypes.c_int32, []),
    "olb_required_bytes": (ctypes.c_size_t, [_P(olb_params)]),
    "olb_create_lattice": (ctypes.c_int, [_P(olb_params), _P(_h)]),
    "olb_set_option": (ctypes.c_int, [_h, ctypes.c_int32, ctypes.c_int64]),
    "olb_set_stream": (ctypes.c_int, [_h, ctypes.c_void_p]),
    "olb_compare": (ctypes.c_int, [_h, _h, _d, _d]),
    "olb_init_shear_wave": (ctypes.c_int, [_h, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int32, ctypes.c_int32]),
    "olb_init_shear_flow": (ctypes.c_int, [_h, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int32]),
    "olb_init_shock_tube": (ctypes.c_int, [_h, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int32]),
    "olb_init_fields": (ctypes.c_int, [_h, _d, _d, _d]),
    "olb_step": (ctypes.c_int, [_h, ctypes.c_int64]),
    "olb_time": (ctypes.c_int64, [_h]),
    "olb_moments": (ctypes.c_int, [_h, _d, _d, _d, _d]),
    "olb_moments_device": (ctypes.c_int, [_h, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "olb_get_populations": (ctypes.c_int, [_h, _d]),
    "olb_get_region": (ctypes.c_int, [_h, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, _d]),
    "olb_set_populations": (ctypes.c_int, [_h, _d, ctypes.c_int64]),
    "olb_diagnostics": (ctypes.c_int, [_h, _d, _d, _d, _P(ctypes.c_int64)]),
    "olb_wave_amplitude": (ctypes.c_int, [_h, ctypes.c_int32, ctypes.c_int32, _d]),
    "olb_wave_mode": (ctypes.c_int, [_h, ctypes.c_int32, ctypes.c_int32, _d, _d]),
    "olb_diagnostics_noalloc": (ctypes.c_int, [ctypes.c_void_p, _P(olb_params), ctypes.c_int64,
                                               ctypes.c_void_p]),
    "olb_destroy": (ctypes.c_int, [_h]),
    "olb_batch_create": (ctypes.c_int, [_P(olb_batch_params), _P(_h)]),
    "olb_batch_add": (ctypes.c_int, [_h, _h, ctypes.c_int64]),
    "olb_batch_remove": (ctypes.c_int, [_h, _h]),
    "olb_batch_run": (ctypes.c_int, [_h, ctypes.c_int64]),
    "olb_batch_wait": (ctypes.c_int, [_h]),
    "olb_batch_wait_for": (ctypes.c_int, [_h, ctypes.c_double]),
    "olb_batch_remaining": (ctypes.c_int, [_h, _h, _P(ctypes.c_int64)]),
    "olb_batch_size": (ctypes.c_int32, [_h]),
    "olb_batch_work_items": (ctypes.c_int64, [_h]),
    "olb_batch_destroy": (ctypes.c_int, [_h]),
    "olb_last_error": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Opens liboreg.so (built by ``paper_2501_16000_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise OregLibraryMissing(
                    f"{path} does not exist: build it with "
                    "`python -m paper_2501_16000_gb300.build` (needs nvcc)")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            if lib.olb_abi_version() != ABI_VERSION:
                raise OregLibraryMissing(
                    f"{path} implements ABI {lib.olb_abi_version()}, this binding {ABI_VERSION}: "
                    "rebuild it with `python -m paper_2501_16000_gb300.build`")
            _lib = lib
        return _lib


def check(status: int, call: str) -> None:
    if status != OLB_OK:
        msg = load().olb_last_error()
        raise OregError(status, msg.decode() if msg else "", call)


def call(name: str, *args):
    """Calls an olb_* function that returns olb_status; raises OregError."""
    st = getattr(load(), name)(*args)
    check(st, name)
    return st


def __getattr__(name: str):
    # binding.olb_step(...) etc. resolve to the raw C functions
    if name.startswith("olb_"):
        return getattr(load(), name)
    raise AttributeError(name)
