"""Rounding check of the FP64 oracle: the same update evaluated in exact
rational arithmetic on a tiny lattice (Eq. 11 product form, Eq. 6, Eq. 7,
push streaming).  This restates the scheme, so it is not a pin of the
formulas (those are in pins.py); it bounds the oracle's rounding error."""
from fractions import Fraction as Fr

import numpy as np

from oracle import oracle as O


def _psi(c, u, th):
    return {0: 1 - th - u * u, 1: (th + u + u * u) / 2, -1: (th - u + u * u) / 2}[c]


def _exact_step(f, C, nx, ny, tau, th):
    out = [[[None] * nx for _ in range(ny)] for _ in range(9)]
    for y in range(ny):
        for x in range(nx):
            g = [f[i][y][x] for i in range(9)]
            rho = sum(g)
            ux = sum(C[i][0] * g[i] for i in range(9)) / rho
            uy = sum(C[i][1] * g[i] for i in range(9)) / rho
            feq = [rho * _psi(C[i][0], ux, th) * _psi(C[i][1], uy, th) for i in range(9)]
            neq = [g[i] - feq[i] for i in range(9)]
            sxx = sum(Fr(C[k][0] ** 2 - C[k][1] ** 2, 2) * neq[k] for k in range(9))
            sxy = sum(C[k][0] * C[k][1] * neq[k] for k in range(9))
            for i in range(9):
                cx, cy = C[i][0] - ux, C[i][1] - uy
                fo = feq[i] / (2 * rho * th * th) * ((cx * cx - cy * cy) * sxx + 2 * cx * cy * sxy)
                out[i][(y + C[i][1]) % ny][(x + C[i][0]) % nx] = feq[i] + (1 - 1 / tau) * fo
    return out


def test_oracle_matches_exact_rationals():
    rng = np.random.default_rng(5)
    nx, ny = 4, 3
    C = [tuple(int(v) for v in c) for c in O.velocities()]
    num = rng.integers(50, 150, size=(9, ny, nx))
    f = [[[Fr(int(num[i, y, x]), 900) for x in range(nx)] for y in range(ny)] for i in range(9)]
    tau, th = Fr(4, 5), Fr(1, 3)
    f64 = np.array([[[float(v) for v in row] for row in pl] for pl in f])
    p = O.params(nx, ny, 0.8, 1 / 3, O.GUIDED, O.OREG)
    for _ in range(2):
        f = _exact_step(f, C, nx, ny, tau, th)
        f64 = O.step(f64, p)
        exact = np.array([[[float(v) for v in row] for row in pl] for pl in f])
        assert np.max(np.abs(f64 - exact)) / np.max(np.abs(exact)) < 1e-14
