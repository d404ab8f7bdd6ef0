"""Python handle on the plain FP64 CPU oracle (``oreg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg use this module; the product path never does.  It compiles
the C oracle with gcc (no floating-point contraction, OpenMP when available)
into ``oracle/_build/`` on first use and exposes numpy-level calls.

Each call restates one passage of arXiv 2501.16000:
  feq          Eq. 11 (guided) / Eq. 15 (polynomial, -u^2/(2 theta0) restored)
  foreg        Eq. 6
  collide      Eq. 7 (OReg) or Eq. 1 (BGK), one node (fixed or local temperature)
  stream       streaming of Eqs. 1/7 (x -> x + c_i, periodic)
  step / run   collide (or bounce back at wall nodes) + stream at every node
  first_order  Eq. 5, one node; init_first_order: S_0 = f^eq + f^(1)
  fields       rho, u and the local temperature of Eq. 2a
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oreg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboreg_oracle.so")

GUIDED, POLY2 = 0, 1
OREG, BGK = 0, 1

_lock = threading.Lock()
_lib = None


class OraParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("tau", ctypes.c_double), ("theta", ctypes.c_double),
                ("eq", ctypes.c_int32), ("coll", ctypes.c_int32),
                ("walls", ctypes.c_int32), ("theta_local", ctypes.c_int32)]


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the oracle shared library (``src`` -> ``out``); returns ``out``."""
    out_dir = os.path.dirname(out)
    os.makedirs(out_dir, exist_ok=True)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", src, "-lm"]
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=out_dir)
    os.close(fd)
    try:
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-o", tmp],
                           check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base + ["-o", tmp], check=True, capture_output=True)
        os.replace(tmp, out)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)
    return out


def load(path: str) -> ctypes.CDLL:
    """Opens an oracle library at ``path`` and declares its signatures."""
    L = ctypes.CDLL(path)
    d = ctypes.POINTER(ctypes.c_double)
    P = ctypes.POINTER(OraParams)
    L.ora_feq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                          ctypes.c_double, ctypes.c_double, d]
    L.ora_node_moments.argtypes = [d, d, d, d]
    L.ora_foreg.argtypes = [d, d, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, ctypes.c_double, d]
    L.ora_collide_node.argtypes = [P, d, d]
    L.ora_bounce_back_node.argtypes = [d, d]
    L.ora_node_theta.argtypes = [d, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.ora_node_theta.restype = ctypes.c_double
    L.ora_stream.argtypes = [ctypes.c_int32, ctypes.c_int32, d, d]
    L.ora_step.argtypes = [P, d, d]
    L.ora_run.argtypes = [P, d, d, ctypes.c_int64]
    L.ora_init_equilibrium.argtypes = [P, d, d, d, d]
    L.ora_first_order.argtypes = [ctypes.c_double, ctypes.c_double, d, ctypes.c_double,
                                  ctypes.c_double, d, d]
    L.ora_init_first_order.argtypes = [P, d, d, d, d, d]
    L.ora_fields.argtypes = [ctypes.c_int32, ctypes.c_int32, d, d, d, d, d]
    L.ora_velocities.argtypes = [ctypes.POINTER(ctypes.c_int32)]
    L.ora_set_threads.argtypes = [ctypes.c_int]
    L.ora_get_threads.restype = ctypes.c_int
    return L


def use(path: str) -> None:
    """Points every call of this module at another build of the oracle
    (the mutation tests load deliberately broken copies this way)."""
    global _lib
    with _lock:
        _lib = load(path)


def reset() -> None:
    """Returns to the committed oracle."""
    global _lib
    with _lock:
        _lib = None


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
        return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def velocities() -> np.ndarray:
    """The oracle's D2Q9 velocity table, shape (9, 2)."""
    out = np.zeros((9, 2), dtype=np.int32)
    lib().ora_velocities(out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return out.astype(np.int64)


def set_threads(n: int) -> None:
    lib().ora_set_threads(int(n))


def get_threads() -> int:
    return int(lib().ora_get_threads())


def params(nx, ny, tau, theta=1.0 / 3.0, eq=GUIDED, coll=OREG, walls=False,
           theta_local=False) -> OraParams:
    """walls: columns x = 0 and nx - 1 are full-way bounce-back walls.
    theta_local: the guided equilibrium and Eq. 6 use each node's temperature."""
    return OraParams(int(nx), int(ny), float(tau), float(theta), int(eq), int(coll),
                     1 if walls else 0, 1 if theta_local else 0)


def feq(eq: int, theta: float, rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    lib().ora_feq(int(eq), float(theta), float(rho), float(ux), float(uy), _p(out))
    return out


def node_moments(f) -> tuple[float, float, float]:
    f = _f64(f)
    r, ux, uy = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().ora_node_moments(_p(f), ctypes.byref(r), ctypes.byref(ux), ctypes.byref(uy))
    return r.value, ux.value, uy.value


def foreg(f, eq: int, theta: float) -> np.ndarray:
    """Eq. 6 for one node's populations f (predictor f^neq = f - f^eq)."""
    f = _f64(f)
    rho, ux, uy = node_moments(f)
    fe = feq(eq, theta, rho, ux, uy)
    theta_eff = theta if eq == GUIDED else 1.0 / 3.0
    out = np.zeros(9)
    lib().ora_foreg(_p(f), _p(fe), rho, ux, uy, float(theta_eff), _p(out))
    return out


def collide(f, tau: float, theta: float = 1.0 / 3.0, eq: int = GUIDED,
            coll: int = OREG, theta_local: bool = False) -> np.ndarray:
    f = _f64(f)
    out = np.zeros(9)
    p = params(1, 1, tau, theta, eq, coll, theta_local=theta_local)
    lib().ora_collide_node(ctypes.byref(p), _p(f), _p(out))
    return out


def stream(post: np.ndarray) -> np.ndarray:
    """Streaming only; post has shape (9, ny, nx)."""
    post = _f64(post)
    _, ny, nx = post.shape
    dst = np.zeros_like(post)
    lib().ora_stream(nx, ny, _p(post), _p(dst))
    return dst


def step(f: np.ndarray, p: OraParams) -> np.ndarray:
    f = _f64(f)
    assert f.shape == (9, p.ny, p.nx)
    dst = np.empty_like(f)
    lib().ora_step(ctypes.byref(p), _p(f), _p(dst))
    return dst


def run(f: np.ndarray, p: OraParams, nsteps: int) -> np.ndarray:
    """Returns S_{t+nsteps} from S_t (the input array is not modified)."""
    a = np.array(f, dtype=np.float64, copy=True, order="C")
    assert a.shape == (9, p.ny, p.nx)
    work = np.empty_like(a)
    lib().ora_run(ctypes.byref(p), _p(a), _p(work), int(nsteps))
    return a


def init_equilibrium(p: OraParams, rho, ux, uy) -> np.ndarray:
    rho, ux, uy = _f64(rho), _f64(ux), _f64(uy)
    assert rho.shape == (p.ny, p.nx)
    f = np.empty((9, p.ny, p.nx))
    lib().ora_init_equilibrium(ctypes.byref(p), _p(rho), _p(ux), _p(uy), _p(f))
    return f


def first_order(tau: float, eq: int, theta: float, rho: float, ux: float, uy: float,
                grad) -> np.ndarray:
    """Eq. 5 for one node; grad[a][b] = d_b u_a."""
    g = _f64(grad).reshape(4)
    fe = feq(eq, theta, rho, ux, uy)
    theta_eff = theta if eq == GUIDED else 1.0 / 3.0
    out = np.zeros(9)
    lib().ora_first_order(float(tau), float(theta_eff), _p(fe), float(ux), float(uy), _p(g),
                          _p(out))
    return out


def init_first_order(p: OraParams, rho, ux, uy, grad) -> np.ndarray:
    """S_0 = f^eq + f^(1) (Eq. 5); grad has shape (2, 2, ny, nx), grad[a, b] = d_b u_a."""
    rho, ux, uy, grad = _f64(rho), _f64(ux), _f64(uy), _f64(grad)
    assert rho.shape == (p.ny, p.nx) and grad.shape == (2, 2, p.ny, p.nx)
    f = np.empty((9, p.ny, p.nx))
    lib().ora_init_first_order(ctypes.byref(p), _p(rho), _p(ux), _p(uy), _p(grad), _p(f))
    return f


def fields(f: np.ndarray):
    """(rho, ux, uy, theta_local), each (ny, nx)."""
    f = _f64(f)
    _, ny, nx = f.shape
    rho, ux, uy, th = (np.empty((ny, nx)) for _ in range(4))
    lib().ora_fields(nx, ny, _p(f), _p(rho), _p(ux), _p(uy), _p(th))
    return rho, ux, uy, th
