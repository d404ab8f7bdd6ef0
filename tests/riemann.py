"""Exact solution of the isothermal Riemann problem (textbook gas dynamics).

For an isothermal ideal gas p = theta rho (sound speed c = sqrt(theta)), a
density step rho_l > rho_r at rest splits into a left rarefaction and a right
shock around a uniform star state (rho*, u*):
  rarefaction (Riemann invariant u + c ln rho):   u* = -c ln(rho* / rho_l)
  shock (Rankine-Hugoniot, mass flux c sqrt(rho* rho_r)):
                                                  u* = c (rho* - rho_r) / sqrt(rho* rho_r)
  shock speed s = c sqrt(rho* / rho_r); fan from -c to u* - c, where
  u = xi + c and rho = rho_l exp(-u / c).
Used to check the oracle on the shock-tube benchmark of Sec. IV.
"""
import math

import numpy as np
from scipy.optimize import brentq


def star_state(rho_l: float, rho_r: float, theta: float):
    c = math.sqrt(theta)
    g = lambda rs: -c * math.log(rs / rho_l) - c * (rs - rho_r) / math.sqrt(rs * rho_r)
    rs = brentq(g, rho_r, rho_l, xtol=1e-15, rtol=1e-15)
    us = -c * math.log(rs / rho_l)
    return rs, us, c * math.sqrt(rs / rho_r)


def solution(xi: np.ndarray, rho_l: float, rho_r: float, theta: float):
    """(rho, u) at similarity coordinate xi = (x - x0) / t."""
    c = math.sqrt(theta)
    rs, us, s = star_state(rho_l, rho_r, theta)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.where(xi < -c, rho_l, np.where(xi < s, rs, rho_r)).astype(np.float64)
    u = np.where((xi >= -c) & (xi < s), us, 0.0)
    fan = (xi >= -c) & (xi < us - c)
    u = np.where(fan, xi + c, u)
    rho = np.where(fan, rho_l * np.exp(-(xi + c) / c), rho)
    return rho, u
