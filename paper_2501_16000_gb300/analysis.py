"""Decay-rate statistic of the rotated shear wave (Sec. IV).

The paper fits u_x^max(t) ~ exp(-|k|^2 nu~ t).  Here the amplitude is the
projection of the velocity on the initial mode,
A(t) = (2/N) sum_x u(x).e_perp sin(k.x), computed in FP64 on the GPU by
``olb_wave_amplitude``; the decay rate gamma is the least-squares slope of
ln A(t) over samples after the start-up transient (t >= max(20, 20 tau)),
and nu~ = gamma / |k|^2.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W


def fit_decay(ts, amps, tau, floor=0.05):
    """Decay rate from samples after the start-up transient, while the
    amplitude is still above `floor` times its value at the window start
    (later samples mostly measure rounding noise of the storage format)."""
    ts, amps = np.asarray(ts, float), np.asarray(amps, float)
    sel = (ts >= max(20.0, 20.0 * tau)) & (amps > 0)
    if sel.any():
        a0 = amps[np.argmax(sel)]
        sel &= amps >= floor * a0
    if sel.sum() < 3:
        raise ValueError("not enough samples after the start-up transient")
    slope = np.polyfit(ts[sel], np.log(amps[sel]), 1)[0]
    return -slope


def measure_decay(lat, case, steps, every=10):
    """Advances an initialised lattice `steps` steps, sampling A(t) every
    `every` steps; returns (gamma, nu_tilde, samples)."""
    ts, amps = [], []
    t = 0
    while True:
        ts.append(t)
        amps.append(lat.wave_amplitude(case.m, case.n))
        if t >= steps:
            break
        k = min(every, steps - t)
        lat.step(k)
        t += k
    gamma = fit_decay(ts, amps, case.tau)
    return gamma, gamma / W.wave_number_sq(case.nx, case.ny, case.m, case.n), (ts, amps)


def fit_wave(ts, a_sin, a_cos, tau, floor=0.05):
    """(gamma, omega) of an advected wave a_sin + i a_cos ~ A0 exp(-gamma t - i omega t):
    the decay rate from the amplitude hypot(a_sin, a_cos) (as fit_decay) and the
    phase rate from the least-squares slope of the unwrapped phase
    atan2(a_cos, a_sin), so omega = U.k for a wave carried by a mean flow U."""
    ts = np.asarray(ts, float)
    a_sin, a_cos = np.asarray(a_sin, float), np.asarray(a_cos, float)
    amps = np.hypot(a_sin, a_cos)
    gamma = fit_decay(ts, amps, tau, floor)
    phase = np.unwrap(np.arctan2(a_cos, a_sin))
    sel = ts >= max(20.0, 20.0 * tau)
    omega = -np.polyfit(ts[sel], phase[sel], 1)[0]
    return gamma, omega


def measure_wave(lat, case, steps, every=100):
    """Advances an initialised lattice `steps` steps sampling both quadratures of
    the shear mode every `every` steps.  Returns a dict with gamma, nu~ = gamma /
    |k|^2, nu~/nu (nu = theta (tau - 1/2), Eq. 14a), the phase rate omega and the
    advection rate U.k of the case's mean flow."""
    ts, a_s, a_c = [], [], []
    t = 0
    while True:
        s, c = lat.wave_mode(case.m, case.n)
        ts.append(t)
        a_s.append(s)
        a_c.append(c)
        if t >= steps:
            break
        k = min(every, steps - t)
        lat.step(k)
        t += k
    gamma, omega = fit_wave(ts, a_s, a_c, case.tau)
    k2 = W.wave_number_sq(case.nx, case.ny, case.m, case.n)
    theta = case.theta if case.eq == "guided" else W.THETA0
    kx, ky = 2 * np.pi * case.m / case.nx, 2 * np.pi * case.n / case.ny
    return {"gamma": gamma, "nu_tilde": gamma / k2,
            "nu_ratio": gamma / k2 / (theta * (case.tau - 0.5)),
            "omega": omega, "omega_advect": case.ux_mean * kx + case.uy_mean * ky}


def mach_sweep(machs=(0.0, 0.1, 0.2, 0.3, 0.4), geometries=("axis", "diagonal"),
               colls=("oreg", "bgk"), storage="f64", layout="ab", length=200, steps=20000,
               every=200):
    """nu~/nu of the decaying shear wave on a mean flow u_y = Ma sqrt(theta)
    (Sec. IV, Fig. 2): one GPU lattice per (geometry, Ma, collision), started
    from the first-order populations of Eq. 5.  Returns a list of row dicts; a
    run that turns non-finite is reported with ``unstable`` set."""
    from . import binding as B
    from .engine import Lattice
    rows = []
    for geom in geometries:
        for ma in machs:
            for coll in colls:
                case = W.mach_wave(geom, ma, coll, length=length, steps=steps)
                row = {"geometry": geom, "mach": ma, "coll": coll, "nx": case.nx,
                       "ny": case.ny, "tau": case.tau}
                with Lattice(case.nx, case.ny, case.tau, case.theta, case.eq, case.coll,
                             storage, layout) as lat:
                    lat.init_case(case)
                    try:
                        row.update(measure_wave(lat, case, steps, every))
                    except B.OregError as e:
                        if e.status != B.OLB_ERR_NONFINITE:
                            raise
                        row["unstable"] = True
                rows.append(row)
    return rows
