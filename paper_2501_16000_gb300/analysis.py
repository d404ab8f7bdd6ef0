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
