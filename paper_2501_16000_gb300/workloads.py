"""Seeded synthetic inputs shaped like the benchmarks of arXiv 2501.16000 Sec. IV.

This module holds input generators only: lattice sizes, relaxation times,
wave vectors, initial density/velocity fields, batch mixes and arrival traces.
It holds none of the scheme's arithmetic (no equilibrium, no collision, no
streaming), so both the CUDA path's tests and the CPU oracle's tests may use it.

Initial conditions:
  * rotated decaying shear wave (Sec. IV, Eq. 18 generalised to any integer
    wave vector on a periodic lattice):
      k = 2 pi (m / nx, n / ny),  u(x) = U + u0 sin(k . x) e_perp,
      e_perp = (-k_y, k_x) / |k|,  rho = rho0, U a uniform mean flow (zero
    except in the Mach sweep of Fig. 2), and its analytic velocity gradient
    for the first-order start of Eq. 5;
  * isothermal shock tube (Sec. IV): rho = rho_left for x < x_split,
    rho_right otherwise, u = 0, periodic in both axes.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

THETA0 = 1.0 / 3.0


def shear_wave_phase(nx: int, ny: int, m: int, n: int) -> np.ndarray:
    """k . x / (2 pi) reduced exactly to [0, 1) as a float64 array (ny, nx).

    The integer numerator (m x ny + n y nx) mod (nx ny) is formed exactly, so
    the phase carries a single rounding.
    """
    x = np.arange(nx, dtype=np.int64)[None, :]
    y = np.arange(ny, dtype=np.int64)[:, None]
    num = np.mod(m * x * ny + n * y * nx, nx * ny)
    return num.astype(np.float64) / float(nx * ny)


def shear_wave_direction(nx: int, ny: int, m: int, n: int) -> tuple[float, float]:
    """Unit vector e_perp = (-k_y, k_x) / |k| for k = 2 pi (m / nx, n / ny)."""
    kx, ky = m / nx, n / ny
    norm = math.hypot(kx, ky)
    if norm == 0.0:
        raise ValueError("wave vector (m, n) must not be (0, 0)")
    return -ky / norm, kx / norm


def wave_number_sq(nx: int, ny: int, m: int, n: int) -> float:
    """|k|^2 for k = 2 pi (m / nx, n / ny)."""
    return (2.0 * math.pi) ** 2 * ((m / nx) ** 2 + (n / ny) ** 2)


def shear_wave_fields(nx, ny, rho0, u0, m, n, ux_mean=0.0, uy_mean=0.0):
    """(rho, ux, uy) float64 arrays (ny, nx) of the rotated shear wave,
    optionally carried by a uniform mean flow (ux_mean, uy_mean)."""
    ph = shear_wave_phase(nx, ny, m, n)
    s = np.sin(2.0 * np.pi * ph)
    ex, ey = shear_wave_direction(nx, ny, m, n)
    rho = np.full((ny, nx), float(rho0))
    return rho, ux_mean + u0 * ex * s, uy_mean + u0 * ey * s


def shear_wave_gradients(nx, ny, u0, m, n):
    """Analytic velocity gradient of the shear wave, shape (2, 2, ny, nx):
    grad[a, b] = d_b u_a = u0 cos(k . x) e_perp_a k_b (the mean flow drops out)."""
    ph = shear_wave_phase(nx, ny, m, n)
    c = np.cos(2.0 * np.pi * ph)
    e = shear_wave_direction(nx, ny, m, n)
    k = (2.0 * math.pi * m / nx, 2.0 * math.pi * n / ny)
    return np.stack([np.stack([u0 * e[a] * k[b] * c for b in range(2)]) for a in range(2)])


def shear_wave_window(nx, ny, rho0, u0, m, n, x0, y0, wx, wy):
    """(rho, ux, uy) of the nx x ny shear wave on the window of wx x wy nodes
    whose first node is the global node (x0, y0) (coordinates wrap)."""
    x = (x0 + np.arange(wx, dtype=np.int64))[None, :] % nx
    y = (y0 + np.arange(wy, dtype=np.int64))[:, None] % ny
    num = np.mod(m * x * ny + n * y * nx, nx * ny)
    s = np.sin(2.0 * np.pi * (num.astype(np.float64) / float(nx * ny)))
    ex, ey = shear_wave_direction(nx, ny, m, n)
    return np.full((wy, wx), float(rho0)), u0 * ex * s, u0 * ey * s


def shock_tube_fields(nx, ny, rho_left, rho_right, x_split):
    """(rho, ux, uy) of the isothermal shock tube, a density step at x_split."""
    x = np.arange(nx)[None, :]
    rho = np.where(x < x_split, float(rho_left), float(rho_right)) * np.ones((ny, 1))
    z = np.zeros((ny, nx))
    return rho, z, z.copy()


def wave_vector_from_angle(nx: int, ny: int, phi: float, wavelength: float = 64.0):
    """Integer (m, n) closest to a wave of the given wavelength at angle phi.

    (m, n) = round(nx cos(phi) / lambda, ny sin(phi) / lambda); at least one is
    nonzero.  Returns (m, n, realised angle in radians).
    """
    m = int(round(nx * math.cos(phi) / wavelength))
    n = int(round(ny * math.sin(phi) / wavelength))
    if m == 0 and n == 0:
        if math.cos(phi) >= math.sin(phi):
            m = 1
        else:
            n = 1
    return m, n, math.atan2(n / ny, m / nx)


# ---------------------------------------------------------------------------
# Benchmark configurations (Sec. IV shapes; synthetic, seeded)
# ---------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class LatticeCase:
    """One lattice problem: geometry, physics and initial condition."""
    nx: int
    ny: int
    tau: float
    theta: float = THETA0
    eq: str = "guided"          # "guided" (Eq. 11) or "poly2" (Eq. 15)
    coll: str = "oreg"          # "oreg" (Eq. 7) or "bgk" (Eq. 1)
    case: str = "shear"         # "shear" or "shock"
    rho0: float = 1.0
    u0: float = 0.05
    m: int = 1
    n: int = 0
    rho_left: float = 1.5
    rho_right: float = 0.75
    x_split: int = 0
    steps: int = 0
    ux_mean: float = 0.0        # uniform mean flow under the shear wave
    uy_mean: float = 0.0
    first_order: bool = False   # start from f^eq + f^(1) of Eq. 5 (shear only)
    boundary: str = "periodic"  # or "walls_x": bounce-back wall columns x = 0, nx - 1
    theta_mode: str = "fixed"   # or "local": guided equilibrium at each node's temperature

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    def fields(self):
        if self.case == "shear":
            return shear_wave_fields(self.nx, self.ny, self.rho0, self.u0, self.m, self.n,
                                     self.ux_mean, self.uy_mean)
        return shock_tube_fields(self.nx, self.ny, self.rho_left, self.rho_right, self.x_split)

    def gradients(self):
        """grad[a, b] = d_b u_a of the initial velocity field (shear only)."""
        if self.case != "shear":
            raise ValueError("analytic gradients exist for the shear wave only")
        return shear_wave_gradients(self.nx, self.ny, self.u0, self.m, self.n)


def shear_64(coll: str = "oreg", m: int = 2, n: int = 1) -> LatticeCase:
    """64 x 64 periodic rotated shear wave, theta = 1/3, tau = 0.8, 1000 steps."""
    return LatticeCase(nx=64, ny=64, tau=0.8, coll=coll, case="shear", u0=0.05,
                       m=m, n=n, steps=1000)


def shock_2048x4(eq: str = "guided", coll: str = "oreg") -> LatticeCase:
    """2048 x 4 isothermal shock tube, 1.5 | 0.75 split at x = 1024, tau = 0.51."""
    return LatticeCase(nx=2048, ny=4, tau=0.51, eq=eq, coll=coll, case="shock",
                       rho_left=1.5, rho_right=0.75, x_split=1024, steps=2000)


def shock_tube_walls(theta: float = 0.35, nu: float = 1e-5, nx: int = 800, ny: int = 1,
                     eq: str = "guided", coll: str = "oreg", rho_left: float = 1.5,
                     rho_right: float = 0.75, steps: int = 500) -> LatticeCase:
    """Isothermal shock tube between full-way bounce-back walls (Sec. IV,
    Figs. 3-4): nx x ny lattice, wall columns x = 0 and nx - 1, density step
    at the middle, tau = 1/2 + nu / theta.  The paper runs 800 x 1 for 500
    steps at (theta, nu) = (0.35, 1e-5) and (0.4, 1e-9) and does not state
    the two densities; 1.5 | 0.75 is used as for the periodic tube."""
    return LatticeCase(nx=nx, ny=ny, tau=0.5 + nu / theta, theta=theta, eq=eq, coll=coll,
                       case="shock", rho_left=rho_left, rho_right=rho_right, x_split=nx // 2,
                       steps=steps, boundary="walls_x")


def large_shear(theta: float = THETA0, seed: int = 0, side: int = 8192,
                steps: int = 500) -> LatticeCase:
    """side x side rotated shear wave at a seeded random angle, tau = 0.6."""
    rng = np.random.default_rng(seed)
    phi = float(rng.uniform(0.0, math.pi / 2))
    m, n, _ = wave_vector_from_angle(side, side, phi)
    return LatticeCase(nx=side, ny=side, tau=0.6, theta=theta, case="shear",
                       u0=0.05, m=m, n=n, steps=steps)


def mach_wave(geometry: str, mach: float, coll: str = "oreg", nu: float = 0.01,
              theta: float = THETA0, amplitude: float = 1e-3, length: int = 200,
              steps: int = 20000, first_order: bool = True) -> LatticeCase:
    """Decaying shear wave on a mean flow u_y = Ma sqrt(theta) (Sec. IV, Fig. 2).

    ``axis``: u_x = A0 sin(2 pi y / L) on a 4 x L lattice, wave vector along y.
    ``diagonal``: the pi/4 wave, u = (A0, A0) sin(k . x) with k along (-1, 1) on
    an M x M lattice, M = round(L sqrt 2), so the wavelength is L as in the
    axis case.  tau = 1/2 + nu / theta.  The shear-wave fields point along
    e_perp = (-k_y, k_x) / |k|, which is -x (axis) and -(1, 1) / sqrt 2
    (diagonal) here, so the amplitudes are negated to give the paper's signs."""
    tau = 0.5 + nu / theta
    if geometry == "axis":
        nx, ny, m, n, u0 = 4, length, 0, 1, -amplitude
    elif geometry == "diagonal":
        side = int(round(length * math.sqrt(2.0)))
        nx, ny, m, n, u0 = side, side, -1, 1, -amplitude * math.sqrt(2.0)
    else:
        raise ValueError(f"unknown geometry {geometry!r}")
    return LatticeCase(nx=nx, ny=ny, tau=tau, theta=theta, coll=coll, case="shear", u0=u0,
                       m=m, n=n, steps=steps, uy_mean=mach * math.sqrt(theta),
                       first_order=first_order)


def _log_uniform_int(rng, lo, hi):
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def batch_mix(count: int = 512, seed: int = 1, lo: int = 32, hi: int = 1024,
              steps: int = 1000) -> list[LatticeCase]:
    """Independent uneven lattices: sides log-uniform in [lo, hi] (non-square),
    tau ~ U[0.51, 1.0], u0 ~ U[0.01, 0.1], angle ~ U[0, pi/2), case 50/50."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx = _log_uniform_int(rng, lo, hi)
        ny = _log_uniform_int(rng, lo, hi)
        tau = float(rng.uniform(0.51, 1.0))
        u0 = float(rng.uniform(0.01, 0.1))
        phi = float(rng.uniform(0.0, math.pi / 2))
        shock = bool(rng.integers(0, 2))
        if shock:
            out.append(LatticeCase(nx=nx, ny=ny, tau=tau, case="shock",
                                   x_split=nx // 2, steps=steps))
        else:
            m, n, _ = wave_vector_from_angle(nx, ny, phi)
            out.append(LatticeCase(nx=nx, ny=ny, tau=tau, case="shear", u0=u0,
                                   m=m, n=n, steps=steps))
    return out


def batch_mix_classes(count: int = 512, seed: int = 1, steps: int = 1000) -> list[LatticeCase]:
    """The lattices of ``batch_mix`` spread over six kernel / constant
    classes: lattice j runs BGK for odd j (else OReg), the polynomial
    equilibrium (theta = 1/3) when j // 2 is odd, else the guided one at
    theta = 0.36 or 0.30 (j // 4 even or odd)."""
    out = []
    for j, c in enumerate(batch_mix(count, seed, steps=steps)):
        poly = (j // 2) % 2 == 1
        out.append(dataclasses.replace(
            c, coll="bgk" if j % 2 else "oreg", eq="poly2" if poly else "guided",
            theta=THETA0 if poly else (0.30 if (j // 4) % 2 else 0.36)))
    return out


@dataclasses.dataclass(frozen=True)
class Request:
    """One solve request of the serving trace."""
    rid: int
    arrival_s: float
    lattice: LatticeCase


def arrival_trace(count: int, rate_per_s: float, seed: int = 2, lo: int = 64,
                  hi: int = 2048, steps_lo: int = 100, steps_hi: int = 10000
                  ) -> list[Request]:
    """Poisson arrivals of square shear/shock solves, sides log-uniform in
    [lo, hi], step counts log-uniform in [steps_lo, steps_hi]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        side = _log_uniform_int(rng, lo, hi)
        steps = _log_uniform_int(rng, steps_lo, steps_hi)
        tau = float(rng.uniform(0.51, 1.0))
        u0 = float(rng.uniform(0.01, 0.1))
        phi = float(rng.uniform(0.0, math.pi / 2))
        if bool(rng.integers(0, 2)):
            lat = LatticeCase(nx=side, ny=side, tau=tau, case="shock",
                              x_split=side // 2, steps=steps)
        else:
            m, n, _ = wave_vector_from_angle(side, side, phi)
            lat = LatticeCase(nx=side, ny=side, tau=tau, case="shear", u0=u0,
                              m=m, n=n, steps=steps)
        out.append(Request(rid, t, lat))
    return out
