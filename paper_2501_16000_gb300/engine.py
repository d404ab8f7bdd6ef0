"""Python-level ``Lattice`` over the C ABI (include/oreg.h).

PyTorch provides the device memory (the population buffer) and the CUDA
stream; all computation happens in liboreg.so.  Host arrays are numpy float64.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding as B

EQ = {"guided": B.OLB_EQ_GUIDED, "poly2": B.OLB_EQ_POLY2}
COLL = {"oreg": B.OLB_COLL_OREG, "bgk": B.OLB_COLL_BGK}
STORAGE = {"f64": B.OLB_F64, "f32": B.OLB_F32, "f16": B.OLB_F16_SHIFTED,
           "bf16": B.OLB_BF16_SHIFTED}
LAYOUT = {"ab": B.OLB_LAYOUT_AB, "aa": B.OLB_LAYOUT_AA}
ELEM_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}


def bytes_per_node_step(storage: str) -> int:
    """Algorithmic HBM traffic of one node update: 9 reads + 9 writes."""
    return 18 * ELEM_BYTES[storage]


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(nx, ny, tau, theta=1.0 / 3.0, eq="guided", coll="oreg", storage="f32",
                layout="ab", rho0=1.0, device_buffer=0, buffer_bytes=0, stream=0,
                boundary="periodic", theta_mode="fixed"):
    return B.olb_params(int(nx), int(ny), float(tau), float(theta), float(rho0), EQ[eq],
                        COLL[coll], STORAGE[storage], LAYOUT[layout], device_buffer or None,
                        int(buffer_bytes), stream or None, B.BOUNDARY[boundary],
                        B.THETA_MODE[theta_mode])


def required_bytes(**kw) -> int:
    p = make_params(**kw)
    return int(B.load().olb_required_bytes(ctypes.byref(p)))


class Lattice:
    """One D2Q9 lattice (periodic, or with bounce-back wall columns at x = 0
    and x = nx - 1) advanced by the OReg (or BGK) update.

    ``torch_memory=True`` places the populations in a torch CUDA tensor and
    runs on torch's current stream (the default when torch sees a GPU)."""

    def __init__(self, nx, ny, tau, theta=1.0 / 3.0, eq="guided", coll="oreg",
                 storage="f32", layout="ab", rho0=1.0, torch_memory=None, stream=None,
                 boundary="periodic", theta_mode="fixed"):
        self.nx, self.ny, self.tau, self.theta = int(nx), int(ny), float(tau), float(theta)
        self.eq, self.coll, self.storage, self.layout = eq, coll, storage, layout
        self.boundary, self.theta_mode = boundary, theta_mode
        self._buf = None
        self._handle = None
        self.stream = None  # torch stream the lattice runs on (torch memory only)
        kw = dict(nx=nx, ny=ny, tau=tau, theta=theta, eq=eq, coll=coll, storage=storage,
                  layout=layout, rho0=rho0, boundary=boundary, theta_mode=theta_mode)
        dev_ptr, nbytes, sptr = 0, 0, 0
        if torch_memory is None:
            try:
                import torch
                torch_memory = torch.cuda.is_available()
            except ImportError:
                torch_memory = False
        if torch_memory:
            import torch
            nbytes = required_bytes(**kw)
            if nbytes == 0:
                p = make_params(**kw)
                h = ctypes.c_void_p()
                B.check(B.load().olb_create_lattice(ctypes.byref(p), ctypes.byref(h)),
                        "olb_create_lattice")
            self._buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            dev_ptr = self._buf.data_ptr()
            s = stream if stream is not None else torch.cuda.current_stream()
            if s.cuda_stream == 0:
                # torch's legacy default stream has handle 0, which the C ABI
                # reads as "create a stream": give the lattice a torch stream
                # of its own instead, so callers can order work against it
                s = torch.cuda.Stream()
            self.stream = s
            sptr = s.cuda_stream
        self.params = make_params(**kw, device_buffer=dev_ptr, buffer_bytes=nbytes, stream=sptr)
        h = ctypes.c_void_p()
        B.check(B.load().olb_create_lattice(ctypes.byref(self.params), ctypes.byref(h)),
                "olb_create_lattice")
        self._handle = h

    # -- lifetime ---------------------------------------------------------
    @property
    def handle(self):
        if self._handle is None:
            raise RuntimeError("lattice is closed")
        return self._handle

    def close(self) -> None:
        if self._handle is not None:
            st = B.load().olb_destroy(self._handle)
            self._handle = None
            self._buf = None
            B.check(st, "olb_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if self._handle is not None:
                B.load().olb_destroy(self._handle)
                self._handle = None
        except Exception:
            pass

    # -- state --------------------------------------------------------------
    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    @property
    def time(self) -> int:
        return int(B.load().olb_time(self.handle))

    def set_option(self, option: int, value: int) -> None:
        B.call("olb_set_option", self.handle, int(option), int(value))

    def set_stream(self, stream) -> None:
        """Runs every later call of this lattice on the torch stream `stream`
        (olb_set_stream); the caller orders it after work already enqueued."""
        B.call("olb_set_stream", self.handle, ctypes.c_void_p(stream.cuda_stream))
        self.stream = stream

    def read_back_on(self, stream, keep_fields: bool = True):
        """Reads the state back on `stream` without the library allocating
        device memory: the FP64 diagnostics through olb_diagnostics_noalloc
        (its fixed scratch; callers must not overlap such calls on the GPU)
        and, if asked, rho and u through olb_moments_device into torch
        buffers copied to pinned host memory.  The lattice moves to `stream`;
        the caller orders `stream` after the lattice's last update.  Blocks
        until `stream` has run the readback.  Returns (mass, non-finite node
        count, (rho, ux, uy) or None); the fields are None for a state with
        non-finite nodes."""
        import torch
        if self._buf is None:
            raise RuntimeError("read_back_on needs torch memory")
        self.set_stream(stream)
        with torch.cuda.stream(stream):
            d_out = torch.empty(4, dtype=torch.float64, device="cuda")
            p = B.olb_params.from_buffer_copy(self.params)
            p.cuda_stream = stream.cuda_stream
            B.call("olb_diagnostics_noalloc", ctypes.c_void_p(self._buf.data_ptr()),
                   ctypes.byref(p), self.time, ctypes.c_void_p(d_out.data_ptr()))
            h_out = torch.empty(4, dtype=torch.float64, pin_memory=True)
            h_out.copy_(d_out, non_blocking=True)
            h = None
            if keep_fields:
                d = torch.empty((3, self.ny, self.nx), dtype=torch.float64, device="cuda")
                B.call("olb_moments_device", self.handle, ctypes.c_void_p(d[0].data_ptr()),
                       ctypes.c_void_p(d[1].data_ptr()), ctypes.c_void_p(d[2].data_ptr()), None)
                h = torch.empty((3, self.ny, self.nx), dtype=torch.float64, pin_memory=True)
                h.copy_(d, non_blocking=True)
        stream.synchronize()
        out = h_out.numpy()
        nonfinite = int(round(out[3]))
        fields = None
        if h is not None and nonfinite == 0:
            a = h.numpy()
            fields = (a[0].copy(), a[1].copy(), a[2].copy())
        return float(out[0]), nonfinite, fields

    def init_shear_wave(self, rho0=1.0, u0=0.05, m=1, n=0) -> None:
        B.call("olb_init_shear_wave", self.handle, float(rho0), float(u0), int(m), int(n))

    def init_shear_flow(self, rho0=1.0, u0=0.05, m=1, n=0, ux_mean=0.0, uy_mean=0.0,
                        first_order=False) -> None:
        """Shear wave on a uniform mean flow; ``first_order`` adds f^(1) of Eq. 5."""
        B.call("olb_init_shear_flow", self.handle, float(rho0), float(u0), int(m), int(n),
               float(ux_mean), float(uy_mean), 1 if first_order else 0)

    def init_shock_tube(self, rho_left=1.5, rho_right=0.75, x_split=None) -> None:
        xs = self.nx // 2 if x_split is None else int(x_split)
        B.call("olb_init_shock_tube", self.handle, float(rho_left), float(rho_right), xs)

    def init_fields(self, rho, ux, uy) -> None:
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy)]
        for a in arrs:
            assert a.shape == (self.ny, self.nx)
        B.call("olb_init_fields", self.handle, *[_dptr(a) for a in arrs])

    def init_case(self, case) -> None:
        """Initial condition of a ``workloads.LatticeCase``."""
        if case.case == "shear":
            if case.ux_mean or case.uy_mean or case.first_order:
                self.init_shear_flow(case.rho0, case.u0, case.m, case.n, case.ux_mean,
                                     case.uy_mean, case.first_order)
            else:
                self.init_shear_wave(case.rho0, case.u0, case.m, case.n)
        else:
            self.init_shock_tube(case.rho_left, case.rho_right, case.x_split)

    def step(self, n: int = 1) -> None:
        B.call("olb_step", self.handle, int(n))

    def moments(self, theta_loc: bool = False):
        rho, ux, uy = (np.empty((self.ny, self.nx)) for _ in range(3))
        th = np.empty((self.ny, self.nx)) if theta_loc else None
        B.call("olb_moments", self.handle, _dptr(rho), _dptr(ux), _dptr(uy),
               _dptr(th) if th is not None else None)
        return (rho, ux, uy, th) if theta_loc else (rho, ux, uy)

    def populations(self) -> np.ndarray:
        f = np.empty((9, self.ny, self.nx))
        B.call("olb_get_populations", self.handle, _dptr(f))
        return f

    def region(self, x0: int, y0: int, wx: int, wy: int) -> np.ndarray:
        """Canonical populations of a window, shape (9, wy, wx)."""
        f = np.empty((9, wy, wx))
        B.call("olb_get_region", self.handle, int(x0), int(y0), int(wx), int(wy), _dptr(f))
        return f

    def set_populations(self, f, t: int = 0) -> None:
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx)
        B.call("olb_set_populations", self.handle, _dptr(f), int(t))

    def diagnostics(self, raise_nonfinite: bool = True):
        m, jx, jy = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        nf = ctypes.c_int64()
        st = B.load().olb_diagnostics(self.handle, ctypes.byref(m), ctypes.byref(jx),
                                      ctypes.byref(jy), ctypes.byref(nf))
        if st != B.OLB_ERR_NONFINITE or raise_nonfinite:
            B.check(st, "olb_diagnostics")
        return {"mass": m.value, "mom_x": jx.value, "mom_y": jy.value, "nonfinite": nf.value}

    def compare(self, ref: "Lattice") -> tuple[float, float]:
        """(max |f - f_ref|, max |f_ref|) over all populations of the two
        lattices' canonical states (olb_compare, reduced on the GPU)."""
        d, r = ctypes.c_double(), ctypes.c_double()
        B.call("olb_compare", self.handle, ref.handle, ctypes.byref(d), ctypes.byref(r))
        return d.value, r.value

    def wave_amplitude(self, m: int, n: int) -> float:
        a = ctypes.c_double()
        B.call("olb_wave_amplitude", self.handle, int(m), int(n), ctypes.byref(a))
        return a.value

    def wave_mode(self, m: int, n: int) -> tuple[float, float]:
        """(a_sin, a_cos): both quadratures of the shear-mode projection."""
        a, b = ctypes.c_double(), ctypes.c_double()
        B.call("olb_wave_mode", self.handle, int(m), int(n), ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value
