"""Checks that pin the FP64 oracle to what arXiv 2501.16000 and the mathematics fix.

Each ``check_*`` raises AssertionError on failure.  They are used twice: by
``test_oracle_pins.py`` against the committed oracle, and by
``test_oracle_mutations.py`` against deliberately broken copies of it (every
broken copy must fail at least one check).

The expected values below are closed forms, textbook special cases or exact
invariants.  None is produced by re-running the oracle's own formula:

* Eq. 2a/2b (moment constraints of the equilibrium) and the heat-flux defect
  the paper states for the guided equilibrium (Sec. III.C, "six out of eight").
* Rest weights of Eq. 11 / Eq. 15: (1-theta)^2, theta(1-theta)/2, theta^2/4;
  the textbook D2Q9 weights 4/9, 1/9, 1/36 at theta = 1/3.
* Eq. 13a / Eq. 16a (mass compatibility of f^OReg is zero).
* Eq. 13b / Eq. 16b (momentum source of f^OReg), Eq. 12b/12c and Eq. 17
  (stress of f^OReg), rewritten with the trace-free non-equilibrium stress S
  in place of the strain rate (S = -tau rho theta (grad u + grad u^T - div u I)
  at first order), for populations built with a prescribed S.
* Eq. 1 vs Eq. 7: at rest and theta = 1/3 the OReg projection is the identity
  on the stress Hermite modes, so both updates coincide there.
* Streaming of Eqs. 1/7: a lone population moves by c_i and wraps.
* Conservation under periodic boundaries; the viscous decay of a shear wave
  exp(-nu k^2 t), nu = theta (tau - 1/2) (Eq. 14a, Sec. IV); the isothermal
  Riemann problem (Sec. IV shock tube, textbook solution in riemann.py).
* Eq. 5 (first-order populations from a velocity gradient): their mass,
  momentum and stress are the paper's Eqs. 12-13 / 16-17; a wave started
  from them decays at the viscous rate from the first step.
* Fig. 2a: an axis-aligned shear wave on a mean flow along its wave vector
  decays at the imposed viscosity and is advected at U.k.
* Local temperature: BGK conserves <f, c^2> at every node (Eq. 2a energy of
  the guided equilibrium), OReg changes it by (1 - 1/tau) x the trace of
  Eq. 12b; sound travels at sqrt(theta) (isothermal) and at sqrt(2 theta)
  (gamma = 2 for D = 2) with the local temperature.
* Full-way bounce-back walls: exact mass, the rest state as a fixed point,
  the slowest viscous mode between no-slip walls placed halfway between wall
  and fluid columns, and the Sec. IV shock tube between walls against the
  Riemann solution at the paper's temperatures and viscosities.

Values the paper prints (the weight factors after Eq. 15, the Sec. IV
shock-tube grid, steps, temperatures, viscosities and L2 accuracies) are read
from ``tests/golden/paper_values.json``, each with its citation.
"""
from __future__ import annotations

import itertools
import json
import math
import os

import numpy as np

from oracle import oracle as O
from paper_2501_16000_gb300 import workloads as W

from . import riemann

RNG_SEED = 20250127

with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                       "paper_values.json")) as _f:
    GOLDEN = json.load(_f)


# ---------------------------------------------------------------------------
# helpers that only take moments (sums of c-polynomials), never the scheme
# ---------------------------------------------------------------------------

def _c():
    return O.velocities().astype(np.float64)


def _moments(f):
    """rho, j, Pi (2x2), q (heat flux vector) of 9 populations."""
    c = _c()
    rho = f.sum()
    j = c.T @ f
    Pi = np.einsum("ia,ib,i->ab", c, c, f)
    c2 = (c ** 2).sum(1)
    q = 0.5 * np.einsum("i,ia,i->a", c2, c, f)
    return rho, j, Pi, q


def _basis():
    """9 x 9 moment matrix with rows 1, cx, cy, (cx^2-cy^2)/2, cx cy,
    cx^2+cy^2, cx^2 cy, cx cy^2, cx^2 cy^2 (invertible on D2Q9)."""
    c = _c()
    cx, cy = c[:, 0], c[:, 1]
    return np.stack([np.ones(9), cx, cy, 0.5 * (cx ** 2 - cy ** 2), cx * cy,
                     cx ** 2 + cy ** 2, cx ** 2 * cy, cx * cy ** 2, cx ** 2 * cy ** 2])


def _with_stress(eq, theta, rho, ux, uy, sxx, sxy, ghosts):
    """Populations with density rho, velocity u, trace-free non-equilibrium
    stress (S_xx, S_xy) and arbitrary higher (ghost) moments."""
    M = _basis()
    g = np.linalg.solve(M, np.array([0.0, 0.0, 0.0, sxx, sxy, *ghosts]))
    return O.feq(eq, theta, rho, ux, uy) + g


def _close(a, b, tol, what):
    a, b = np.asarray(a, float), np.asarray(b, float)
    err = np.max(np.abs(a - b)) if a.size else 0.0
    assert err <= tol, f"{what}: |{a} - {b}| = {err:.3e} > {tol:.1e}"


# ---------------------------------------------------------------------------
# velocity set
# ---------------------------------------------------------------------------

def check_velocity_set():
    c = O.velocities()
    assert c.shape == (9, 2)
    want = sorted(itertools.product((-1, 0, 1), repeat=2))
    assert sorted(map(tuple, c.tolist())) == want, "not the D2Q9 set (Fig. 1a)"
    assert tuple(c[0]) == (0, 0)


# ---------------------------------------------------------------------------
# equilibria: Eq. 2a/2b, rest weights, heat-flux defect
# ---------------------------------------------------------------------------

def check_guided_rest_weights():
    c = O.velocities()
    for theta in (1.0 / 3.0, 0.3, 0.4):
        f = O.feq(O.GUIDED, theta, 1.7, 0.0, 0.0)
        nz = (c != 0).sum(1)
        want = np.where(nz == 0, (1 - theta) ** 2,
                        np.where(nz == 1, theta * (1 - theta) / 2, theta ** 2 / 4)) * 1.7
        _close(f, want, 1e-15, f"guided rest weights theta={theta}")
    f = O.feq(O.GUIDED, 1.0 / 3.0, 1.0, 0.0, 0.0)
    nz = (c != 0).sum(1)
    _close(f, np.where(nz == 0, 4 / 9, np.where(nz == 1, 1 / 9, 1 / 36)), 1e-15,
           "textbook D2Q9 weights")


def check_poly2_rest_weights():
    c = O.velocities()
    nz = (c != 0).sum(1)
    f = O.feq(O.POLY2, 0.3, 1.3, 0.0, 0.0)   # theta argument is ignored: theta0 = 1/3
    _close(f, 1.3 * np.where(nz == 0, 4 / 9, np.where(nz == 1, 1 / 9, 1 / 36)), 1e-15,
           "polynomial weights W_i")
    # the paper's own statement (after Eq. 15): tensor products of
    # W_0 = 1 - theta0 and W_+-1 = theta0 / 2
    g = GOLDEN["polynomial_equilibrium_weights"]
    th0 = g["theta0"][0] / g["theta0"][1]
    w1 = {0: 1 - th0, 1: th0 / 2, -1: th0 / 2}
    _close(f, np.array([1.3 * w1[int(cx)] * w1[int(cy)] for cx, cy in c]), 1e-15,
           "polynomial weights as tensor products (after Eq. 15)")


def check_equilibrium_moments():
    rng = np.random.default_rng(RNG_SEED)
    for _ in range(50):
        rho = rng.uniform(0.5, 2.0)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        for eq in (O.GUIDED, O.POLY2):
            theta = rng.uniform(0.2, 0.5) if eq == O.GUIDED else 1.0 / 3.0
            f = O.feq(eq, theta, rho, ux, uy)
            r, j, Pi, q = _moments(f)
            u = np.array([ux, uy])
            _close(r, rho, 1e-14, "Eq. 2a mass")
            _close(j, rho * u, 1e-14, "Eq. 2a momentum")
            _close(Pi, rho * theta * np.eye(2) + rho * np.outer(u, u), 1e-14,
                   "Eq. 2b pressure tensor")
            E = (2 * rho * theta + rho * u @ u) / 2
            _close(0.5 * np.trace(Pi), E, 1e-14, "energy E")
            if eq == O.GUIDED:
                # heat flux misses Eq. 2c by -rho u_a (3 theta + u_a^2 - 1)/2
                q_mb = u * (E + rho * theta)
                _close(q - q_mb, -rho * u * (3 * theta + u ** 2 - 1) / 2, 1e-14,
                       "guided heat-flux defect")
            else:
                q_mb = u * (E + rho * theta)
                _close(q - q_mb, -rho * u * (u @ u) / 2, 1e-14, "poly2 heat-flux defect")


# ---------------------------------------------------------------------------
# Eq. 6 against Eqs. 12, 13, 16, 17
# ---------------------------------------------------------------------------

def _foreg_cases(eq):
    rng = np.random.default_rng(RNG_SEED + eq)
    for k in range(40):
        rho = rng.uniform(0.6, 1.8)
        ux, uy = (0.0, 0.0) if k < 4 else rng.uniform(-0.25, 0.25, 2)
        theta = (rng.uniform(0.25, 0.45) if k % 2 else 1.0 / 3.0) if eq == O.GUIDED else 1.0 / 3.0
        sxx, sxy = rng.uniform(-0.02, 0.02, 2)
        ghosts = rng.uniform(-0.02, 0.02, 4)
        yield rho, ux, uy, theta, sxx, sxy, ghosts


def check_foreg_mass_zero():
    for eq in (O.GUIDED, O.POLY2):
        for rho, ux, uy, th, sxx, sxy, gh in _foreg_cases(eq):
            f = _with_stress(eq, th, rho, ux, uy, sxx, sxy, gh)
            _close(O.foreg(f, eq, th).sum(), 0.0, 1e-15, "Eq. 13a/16a <f^OReg,1> = 0")


def check_foreg_guided_closed_forms():
    c = _c()
    for rho, ux, uy, th, sxx, sxy, gh in _foreg_cases(O.GUIDED):
        f = _with_stress(O.GUIDED, th, rho, ux, uy, sxx, sxy, gh)
        fo = O.foreg(f, O.GUIDED, th)
        mom = c.T @ fo
        # Eq. 13b: <f^OReg, c_a> = -S_aa u_a (3 theta + u_a^2 - 1) / (2 theta^2), S_yy = -S_xx
        _close(mom[0], -sxx * ux * (3 * th + ux ** 2 - 1) / (2 * th ** 2), 1e-15, "Eq. 13b x")
        _close(mom[1], sxx * uy * (3 * th + uy ** 2 - 1) / (2 * th ** 2), 1e-15, "Eq. 13b y")
        Pi = np.einsum("ia,ib,i->ab", c, c, fo)
        # Eq. 12b diagonal viscosity: (theta - u_a^2)(1 - theta - u_a^2) / (2 theta^2)
        _close(Pi[0, 0], sxx * (th - ux ** 2) * (1 - th - ux ** 2) / (2 * th ** 2), 1e-15,
               "Eq. 12b xx")
        _close(Pi[1, 1], -sxx * (th - uy ** 2) * (1 - th - uy ** 2) / (2 * th ** 2), 1e-15,
               "Eq. 12b yy")
        # Eq. 12b off-diagonal (viscosity tau rho theta) plus the Eq. 12c error
        _close(Pi[0, 1], sxy - sxx * ux * uy * (ux ** 2 - uy ** 2) / (2 * th ** 2), 1e-15,
               "Eq. 12a/12c xy")


def check_foreg_poly2_closed_forms():
    c = _c()
    for rho, ux, uy, th, sxx, sxy, gh in _foreg_cases(O.POLY2):
        f = _with_stress(O.POLY2, th, rho, ux, uy, sxx, sxy, gh)
        fo = O.foreg(f, O.POLY2, th)
        mom = c.T @ fo
        # Eq. 16b: <f^OReg, c_a> = -u_a [(u_x^2 - u_y^2) S_xx + 2 u_x u_y S_xy] / (2 theta0^2)
        br = (ux ** 2 - uy ** 2) * sxx + 2 * ux * uy * sxy
        phi = np.array([-4.5 * ux * br, -4.5 * uy * br])
        _close(mom, phi, 1e-15, "Eq. 16b")
        Pi = np.einsum("ia,ib,i->ab", c, c, fo)
        # Eq. 17: off-diagonal error -u_b phi_a; diagonal -u_a phi_a plus the
        # O(u^4) term -(9/2) u_a^2 S_aa
        _close(Pi[0, 1], sxy - uy * phi[0], 1e-15, "Eq. 17 xy")
        _close(Pi[0, 0], sxx - ux * phi[0] - 4.5 * ux ** 2 * sxx, 1e-15, "Eq. 17 xx")
        _close(Pi[1, 1], -sxx - uy * phi[1] + 4.5 * uy ** 2 * sxx, 1e-15, "Eq. 17 yy")


def _first_order_cases(eq):
    rng = np.random.default_rng(RNG_SEED + 11 + eq)
    for k in range(40):
        rho = rng.uniform(0.6, 1.8)
        ux, uy = (0.0, 0.0) if k < 4 else rng.uniform(-0.25, 0.25, 2)
        theta = (rng.uniform(0.25, 0.45) if k % 2 else 1.0 / 3.0) if eq == O.GUIDED else 1.0 / 3.0
        tau = rng.uniform(0.51, 2.0)
        grad = rng.uniform(-0.01, 0.01, (2, 2))
        yield rho, ux, uy, theta, tau, grad


def check_first_order_closed_forms():
    """Eq. 5 populations against the paper's own moments of them: Eq. 12 is
    the pressure tensor and Eq. 13 the mass/momentum of f^(1) with the guided
    equilibrium, Eqs. 16-17 with the polynomial one.  With the strain rate
    written as the trace-free stress S = -tau rho theta (grad u + grad u^T -
    div u I): S_xx = -tau rho theta (d_x u_x - d_y u_y),
    S_xy = -tau rho theta (d_x u_y + d_y u_x)."""
    c = _c()
    for eq in (O.GUIDED, O.POLY2):
        for rho, ux, uy, th, tau, g in _first_order_cases(eq):
            f1 = O.first_order(tau, eq, th, rho, ux, uy, g)
            te = th if eq == O.GUIDED else 1.0 / 3.0
            sxx = -tau * rho * te * (g[0, 0] - g[1, 1])
            sxy = -tau * rho * te * (g[1, 0] + g[0, 1])
            _close(f1.sum(), 0.0, 1e-16, "Eq. 13a/16a <f^(1),1> = 0")
            mom = c.T @ f1
            Pi = np.einsum("ia,ib,i->ab", c, c, f1)
            if eq == O.GUIDED:
                _close(mom[0], -sxx * ux * (3 * th + ux ** 2 - 1) / (2 * th ** 2), 1e-16,
                       "Eq. 13b x of f^(1)")
                _close(mom[1], sxx * uy * (3 * th + uy ** 2 - 1) / (2 * th ** 2), 1e-16,
                       "Eq. 13b y of f^(1)")
                _close(Pi[0, 0], sxx * (th - ux ** 2) * (1 - th - ux ** 2) / (2 * th ** 2), 1e-16,
                       "Eq. 12b xx of f^(1)")
                _close(Pi[1, 1], -sxx * (th - uy ** 2) * (1 - th - uy ** 2) / (2 * th ** 2),
                       1e-16, "Eq. 12b yy of f^(1)")
                _close(Pi[0, 1], sxy - sxx * ux * uy * (ux ** 2 - uy ** 2) / (2 * th ** 2), 1e-16,
                       "Eq. 12a/12c xy of f^(1)")
            else:
                br = (ux ** 2 - uy ** 2) * sxx + 2 * ux * uy * sxy
                phi = np.array([-4.5 * ux * br, -4.5 * uy * br])
                _close(mom, phi, 1e-16, "Eq. 16b of f^(1)")
                _close(Pi[0, 1], sxy - uy * phi[0], 1e-16, "Eq. 17 xy of f^(1)")
                _close(Pi[0, 0], sxx - ux * phi[0] - 4.5 * ux ** 2 * sxx, 1e-16,
                       "Eq. 17 xx of f^(1)")
                _close(Pi[1, 1], -sxx - uy * phi[1] + 4.5 * uy ** 2 * sxx, 1e-16,
                       "Eq. 17 yy of f^(1)")


def check_foreg_vanishes_without_stress():
    rng = np.random.default_rng(RNG_SEED + 7)
    for eq in (O.GUIDED, O.POLY2):
        for _ in range(10):
            th = rng.uniform(0.25, 0.45) if eq == O.GUIDED else 1.0 / 3.0
            f = _with_stress(eq, th, rng.uniform(0.7, 1.5), *rng.uniform(-0.2, 0.2, 2),
                             0.0, 0.0, rng.uniform(-0.03, 0.03, 4))
            _close(O.foreg(f, eq, th), np.zeros(9), 1e-16, "f^OReg without stress")


# ---------------------------------------------------------------------------
# Eq. 7 vs Eq. 1
# ---------------------------------------------------------------------------

def check_collision_special_cases():
    rng = np.random.default_rng(RNG_SEED + 11)
    c = _c()
    nz = (c != 0).sum(1)
    w = np.where(nz == 0, 4 / 9, np.where(nz == 1, 1 / 9, 1 / 36))
    for eq in (O.GUIDED, O.POLY2):
        # tau = 1: both collisions return the equilibrium
        f = _with_stress(eq, 1 / 3, 1.2, 0.05, -0.07, 0.01, -0.004, rng.uniform(-0.01, 0.01, 4))
        fe = O.feq(eq, 1 / 3, *O.node_moments(f))
        for coll in (O.OREG, O.BGK):
            _close(O.collide(f, 1.0, 1 / 3, eq, coll), fe, 1e-15, "tau = 1 gives f^eq")
        # at rest, theta = 1/3 and a pure stress Hermite mode the OReg
        # projection is the identity, so Eq. 7 equals Eq. 1
        a, b = rng.uniform(-0.05, 0.05, 2)
        rho = 1.1
        g = w * ((c[:, 0] ** 2 - c[:, 1] ** 2) * a + c[:, 0] * c[:, 1] * b)
        f = rho * w + g
        for tau in (0.55, 0.8, 1.7):
            _close(O.collide(f, tau, 1 / 3, eq, O.OREG), O.collide(f, tau, 1 / 3, eq, O.BGK),
                   1e-15, "OReg == BGK on stress modes at rest")
        # BGK relaxes the whole non-equilibrium by (1 - 1/tau)
        tau = 0.7
        f = _with_stress(eq, 1 / 3, 0.9, 0.1, 0.03, 0.01, 0.006, rng.uniform(-0.01, 0.01, 4))
        fe = O.feq(eq, 1 / 3, *O.node_moments(f))
        _close(O.collide(f, tau, 1 / 3, eq, O.BGK) - fe, (1 - 1 / tau) * (f - fe), 1e-15,
               "Eq. 1 non-equilibrium relaxation")
        # OReg: mass is conserved; momentum changes by (1 - 1/tau) <f^OReg, c>
        post = O.collide(f, tau, 1 / 3, eq, O.OREG)
        _close(post.sum(), f.sum(), 1e-15, "OReg collision mass")
        _close(c.T @ post - c.T @ f, (1 - 1 / tau) * (c.T @ O.foreg(f, eq, 1 / 3)), 1e-15,
               "OReg collision momentum change")


# ---------------------------------------------------------------------------
# streaming and lattice-level invariants
# ---------------------------------------------------------------------------

def check_streaming_translation():
    c = O.velocities()
    nx, ny = 7, 5
    for i in range(9):
        for (x0, y0) in ((0, 0), (6, 4), (3, 2), (6, 0), (0, 4)):
            post = np.zeros((9, ny, nx))
            post[i, y0, x0] = 1.0
            out = O.stream(post)
            want = np.zeros_like(post)
            want[i, (y0 + c[i, 1]) % ny, (x0 + c[i, 0]) % nx] = 1.0
            assert np.array_equal(out, want), f"population {i} from ({x0},{y0})"


def check_uniform_state_is_fixed():
    for eq in (O.GUIDED, O.POLY2):
        for coll in (O.OREG, O.BGK):
            p = O.params(6, 5, 0.7, 0.35 if eq == O.GUIDED else 1 / 3, eq, coll)
            rho = np.full((5, 6), 1.3)
            f0 = O.init_equilibrium(p, rho, np.full((5, 6), 0.04), np.full((5, 6), -0.03))
            f = O.run(f0, p, 20)
            _close(f, f0, 2e-15, "uniform equilibrium is a fixed point")


def _totals(f):
    c = _c()
    return f.sum(), np.einsum("ia,iyx->a", c, f)


def check_conservation():
    for eq in (O.GUIDED, O.POLY2):
        for coll in (O.OREG, O.BGK):
            p = O.params(24, 16, 0.62, 1 / 3, eq, coll)
            rho, ux, uy = W.shear_wave_fields(24, 16, 1.0, 0.08, 2, 1)
            rho = rho + 0.1 * (np.arange(24)[None, :] < 12)
            ux = ux + 0.03                       # net momentum
            f0 = O.init_equilibrium(p, rho, ux, uy)
            m0, j0 = _totals(f0)
            f = f0
            for _ in range(5):
                g = O.run(f, p, 1)
                m1, j1 = _totals(g)
                _close(m1 / m0, 1.0, 2e-15, "mass per step")
                if coll == O.BGK:
                    _close(j1, j0, 1e-13, "BGK momentum per step")
                else:
                    # momentum change = (1 - 1/tau) sum_x <f^OReg(x), c>; the
                    # per-node source is pinned by Eq. 13b / 16b above
                    src = np.zeros(2)
                    c = _c()
                    for y in range(p.ny):
                        for x in range(p.nx):
                            src += c.T @ O.foreg(f[:, y, x], eq, 1 / 3)
                    _close(j1 - _totals(f)[1], (1 - 1 / p.tau) * src, 1e-13,
                           "OReg momentum change per step")
                f = g
            f = O.run(f, p, 500)
            _close(_totals(f)[0] / m0, 1.0, 1e-13, "mass over 500 steps")


def _decay_ratio(nx, ny, m, n, tau, theta, coll, steps, u0=0.05, eq=O.GUIDED):
    p = O.params(nx, ny, tau, theta, eq, coll)
    f = O.init_equilibrium(p, *W.shear_wave_fields(nx, ny, 1.0, u0, m, n))
    s = np.sin(2 * np.pi * W.shear_wave_phase(nx, ny, m, n))
    ex, ey = W.shear_wave_direction(nx, ny, m, n)
    ts, amps = [], []
    every = max(1, steps // 100)
    for t in range(0, steps + 1, every):
        _, vx, vy, _ = O.fields(f)
        ts.append(t)
        amps.append(2.0 / (nx * ny) * np.sum((vx * ex + vy * ey) * s))
        if t < steps:
            f = O.run(f, p, every)
    ts, amps = np.array(ts), np.array(amps)
    sel = ts >= max(20, 20 * tau)
    with np.errstate(invalid="ignore", divide="ignore"):   # a planted mistake may flip the sign
        gamma = -np.polyfit(ts[sel], np.log(amps[sel]), 1)[0]
    return gamma / W.wave_number_sq(nx, ny, m, n) / (theta * (tau - 0.5))


def check_shear_wave_decay():
    # nu = theta (tau - 1/2) at theta = 1/3 (Eq. 14a, Sec. IV), OReg and BGK
    for coll in (O.OREG, O.BGK):
        for (m, n) in ((2, 1), (1, 1)):
            r = _decay_ratio(64, 64, m, n, 0.8, 1 / 3, coll, 1000)
            assert abs(r - 1) < 2e-3, f"coll={coll} (m,n)=({m},{n}) nu~/nu={r}"
    # second-order lattice: the error falls ~4x when the wave is resolved 2x finer
    e32 = abs(_decay_ratio(32, 32, 2, 1, 0.8, 1 / 3, O.OREG, 250) - 1)
    e64 = abs(_decay_ratio(64, 64, 2, 1, 0.8, 1 / 3, O.OREG, 1000) - 1)
    assert 3.0 < e32 / e64 < 6.0, (e32, e64)


def check_shear_wave_decay_off_reference_temperature():
    """theta != 1/3: the normal-stress response of Eq. 6 at rest is
    kappa = (1 - theta)/(2 theta) times the shear response (Eq. 12b at u = 0).
    Linear theory then gives the decay of a wave at angle phi as
    nu~/nu = cos^2(2 phi) + sin^2(2 phi) r, with r = kappa (tau_n - 1/2)/(tau - 1/2)
    and 1 - 1/tau_n = kappa (1 - 1/tau) for OReg, r = kappa for BGK."""
    theta, tau = 0.3, 0.6
    kappa = (1 - theta) / (2 * theta)
    tau_n = 1.0 / (1.0 - kappa * (1 - 1 / tau))
    phi = math.atan2(1, 2)
    c2, s2 = math.cos(2 * phi) ** 2, math.sin(2 * phi) ** 2
    want = {O.OREG: c2 + s2 * kappa * (tau_n - 0.5) / (tau - 0.5), O.BGK: c2 + s2 * kappa}
    for coll in (O.OREG, O.BGK):
        r = _decay_ratio(64, 64, 2, 1, tau, theta, coll, 1000)
        assert abs(r / want[coll] - 1) < 1e-2, f"coll={coll}: {r} vs linear theory {want[coll]}"


def _wave_series(case, steps, every):
    """Oracle run of a shear-wave case; samples t, and both quadratures of the
    mode projection (2/N) sum u.e_perp {sin, cos}(k.x)."""
    p = O.params(case.nx, case.ny, case.tau, case.theta,
                 O.GUIDED if case.eq == "guided" else O.POLY2,
                 O.OREG if case.coll == "oreg" else O.BGK)
    rho, ux, uy = case.fields()
    if case.first_order:
        f = O.init_first_order(p, rho, ux, uy, case.gradients())
    else:
        f = O.init_equilibrium(p, rho, ux, uy)
    ph = 2 * np.pi * W.shear_wave_phase(case.nx, case.ny, case.m, case.n)
    sn, cs = np.sin(ph), np.cos(ph)
    ex, ey = W.shear_wave_direction(case.nx, case.ny, case.m, case.n)
    ts, a_s, a_c = [], [], []
    for t in range(0, steps + 1, every):
        _, vx, vy, _ = O.fields(f)
        up = vx * ex + vy * ey
        ts.append(t)
        a_s.append(2.0 / case.nodes * np.sum(up * sn))
        a_c.append(2.0 / case.nodes * np.sum(up * cs))
        if t < steps:
            f = O.run(f, p, every)
    return np.array(ts, float), np.array(a_s), np.array(a_c)


def check_first_order_start():
    """Starting from f^eq + f^(1) (Eq. 5) puts the wave on its viscous decay
    exp(-nu k^2 t) (Eq. 14a) from the first step; an equilibrium start (no
    stress) first jumps by O(1e-3) of the amplitude before it settles."""
    k2 = W.wave_number_sq(64, 64, 2, 1)
    for coll in ("oreg", "bgk"):
        for tau in (0.53, 0.8):
            nu = (tau - 0.5) / 3.0
            dev = {}
            for first_order in (False, True):
                case = W.LatticeCase(nx=64, ny=64, tau=tau, coll=coll, m=2, n=1, u0=0.05,
                                     first_order=first_order)
                ts, a_s, _ = _wave_series(case, 20, 1)
                dev[first_order] = np.max(np.abs(a_s / (a_s[0] * np.exp(-nu * k2 * ts)) - 1))
            assert dev[True] < 2e-4, (coll, tau, dev)
            assert dev[False] > 2e-3, (coll, tau, dev)


def check_mean_flow_axis_wave():
    """Sec. IV, Fig. 2a: a shear wave whose wave vector is along a lattice axis,
    carried along that axis by a mean flow u_y = Ma sqrt(theta), decays at the
    imposed viscosity for OReg and BGK alike, and is advected rigidly: its
    phase turns at U.k (Galilean invariance of the Navier-Stokes limit)."""
    for ma in (0.0, 0.2, 0.4):
        for coll in ("oreg", "bgk"):
            case = W.mach_wave("axis", ma, coll, length=64, steps=2000)
            ts, a_s, a_c = _wave_series(case, case.steps, 10)
            gamma = -np.polyfit(ts, np.log(np.hypot(a_s, a_c)), 1)[0]
            ratio = gamma / W.wave_number_sq(case.nx, case.ny, case.m, case.n) / (
                case.theta * (case.tau - 0.5))
            assert abs(ratio - 1) < 2e-3, (ma, coll, ratio)
            omega = -np.polyfit(ts, np.unwrap(np.arctan2(a_c, a_s)), 1)[0]
            want = case.uy_mean * 2 * np.pi * case.n / case.ny
            assert abs(omega - want) <= 1e-4 * abs(want) + 1e-12, (ma, coll, omega, want)


def check_mean_flow_diagonal_wave():
    """Sec. IV, Fig. 2b, read with the paper's own Eq. 12b.  The pi/4 wave
    (wave vector along (-1, 1), velocity along (1, 1)) carried by a mean flow
    u = (0, U), U = Ma sqrt(theta), lives in the normal stresses
    (S_xx = -S_yy, S_xy = 0).  Eq. 12b gives the diagonal stress that f^OReg
    carries the factor phi_a = (theta - u_a^2)(1 - theta - u_a^2) / (2 theta^2):
    phi_x = (1 - theta) / (2 theta) = 1 and phi_y < 1 here, so the normal-stress
    difference S_xx - S_yy is carried with the mean factor (phi_x + phi_y) / 2
    and relaxed per step by (1 - 1/tau)(phi_x + phi_y) / 2 instead of
    (1 - 1/tau), an effective tau' = 1 / (1 - (1 - 1/tau)(phi_x + phi_y) / 2)
    and viscosity theta (tau' - 1/2).  BGK keeps (1 - 1/tau) and carries the
    equilibrium's own O(Ma^2) error, which OReg shares, so the ratio of the
    OReg to the BGK decay rate is predicted as (tau' - 1/2) / (tau - 1/2)
    = 1 + 6.2 Ma^2 + O(Ma^4) at tau = 0.53: the oracle must show that excess
    within 1.5% at Ma <= 0.1 and 4% at Ma = 0.2 (measured -0.8% and -2.9%; the
    remainder grows to -7% of the excess at Ma = 0.3 and -12% at Ma = 0.4,
    where the literal Eqs. 6-7 give nu~/nu = 1.65 rather than Fig. 2b's 1).  Axis-aligned waves, which live in
    the shear stress (factor 1), stay at 1 (check_mean_flow_axis_wave)."""
    th = 1.0 / 3.0
    for ma, tol in ((0.05, 0.015), (0.1, 0.015), (0.2, 0.04)):
        rate = {}
        for coll in ("oreg", "bgk"):
            case = W.mach_wave("diagonal", ma, coll, length=32, steps=2000)
            ts, a_s, a_c = _wave_series(case, case.steps, 20)
            rate[coll] = -np.polyfit(ts, np.log(np.hypot(a_s, a_c)), 1)[0]
        u2 = case.uy_mean ** 2
        phi = 0.5 * ((1 - th) / (2 * th) + (th - u2) * (1 - th - u2) / (2 * th * th))
        lam = 1 - 1 / case.tau
        tau_eff = 1 / (1 - lam * phi)
        want = (tau_eff - 0.5) / (case.tau - 0.5)
        got = rate["oreg"] / rate["bgk"]
        assert want > 1 and abs((got - 1) / (want - 1) - 1) < tol, (ma, got, want)


def check_shock_tube():
    """Sec. IV shock tube at theta = 1/3 vs the exact isothermal Riemann
    solution; OReg shows no post-shock oscillation, BGK does."""
    case = W.shock_2048x4()
    nx, t = case.nx, 500
    x = np.arange(nx)
    win = (x > 600) & (x < 1500)
    rho_ex, u_ex = riemann.solution((x - (case.x_split - 0.5)) / t, 1.5, 0.75, 1 / 3)
    tv_exact = np.abs(np.diff(rho_ex[win])).sum()
    tv = {}
    for coll in (O.OREG, O.BGK):
        p = O.params(nx, case.ny, case.tau, 1 / 3, O.GUIDED, coll)
        f = O.run(O.init_equilibrium(p, *case.fields()), p, t)
        rho, ux, uy, _ = O.fields(f)
        l2 = np.sqrt(((rho[0, win] - rho_ex[win]) ** 2).sum() / (rho_ex[win] ** 2).sum())
        tv[coll] = np.abs(np.diff(rho[0, win])).sum()
        if coll == O.OREG:
            assert l2 < 0.01, f"OReg density L2 error {l2}"
            assert abs(tv[coll] / tv_exact - 1) < 0.01, (tv[coll], tv_exact)
            assert abs(rho[0, 1100] - riemann.star_state(1.5, 0.75, 1 / 3)[0]) < 2e-3
            assert np.abs(uy).max() < 1e-14
    assert tv[O.BGK] > 3 * tv[O.OREG], tv


# ---------------------------------------------------------------------------
# local temperature (the guided equilibrium taking each node's own theta)
# ---------------------------------------------------------------------------

def check_local_theta_energy():
    """With the node's own temperature theta = (<f,c^2> - rho u^2)/(2 rho), the
    guided equilibrium carries the node's energy (Eq. 2a: <f^eq, c^2/2> = E),
    so BGK conserves <f, c^2> at every node, and OReg changes it by exactly
    (1 - 1/tau) times the trace of Eq. 12b's stress of f^OReg,
    S_xx [(theta - u_x^2)(1 - theta - u_x^2) - (theta - u_y^2)(1 - theta - u_y^2)]
    / (2 theta^2).  A uniform state at any temperature is a fixed point."""
    c = _c()
    c2 = (c ** 2).sum(1)
    rng = np.random.default_rng(RNG_SEED + 31)
    for _ in range(40):
        rho = rng.uniform(0.7, 1.4)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        th = rng.uniform(0.25, 0.45)
        sxx, sxy = rng.uniform(-0.02, 0.02, 2)
        f = _with_stress(O.GUIDED, th, rho, ux, uy, sxx, sxy, [0.0, 0.0, 0.0, 0.0])
        # a zero non-equilibrium trace keeps the node's temperature at th
        tau = rng.uniform(0.52, 1.5)
        post_b = O.collide(f, tau, 0.3, O.GUIDED, O.BGK, theta_local=True)
        _close(c2 @ post_b, c2 @ f, 1e-15, "BGK energy with the local temperature")
        post_o = O.collide(f, tau, 0.3, O.GUIDED, O.OREG, theta_local=True)
        tr = sxx * ((th - ux ** 2) * (1 - th - ux ** 2) - (th - uy ** 2) * (1 - th - uy ** 2)) / (
            2 * th ** 2)
        _close(c2 @ post_o - c2 @ f, (1 - 1 / tau) * tr, 1e-15,
               "OReg energy change with the local temperature (Eq. 12b trace)")
        _close(post_o.sum(), f.sum(), 1e-15, "mass with the local temperature")
    for th in (0.2, 0.3, 0.45):
        f = O.feq(O.GUIDED, th, 1.2, 0.03, -0.05)
        for coll in (O.OREG, O.BGK):
            _close(O.collide(f, 0.7, 1 / 3, O.GUIDED, coll, theta_local=True), f, 1e-15,
                   "uniform state at its own temperature")


def _density_wave_speed(coll, theta_local, isentropic, L=64, tau=0.6, th0=1 / 3, steps=400):
    """Sound speed from the zero crossings of the density mode of a standing
    wave rho = 1 + eps cos(k x), u = 0 (temperature perturbed adiabatically
    if isentropic)."""
    x = np.arange(L)
    cs = np.cos(2 * np.pi * x / L)
    eps = 1e-4
    rho = 1 + eps * cs
    th = th0 * (1 + eps * cs) if isentropic else np.full(L, th0)
    f = np.zeros((9, 1, L))
    for i in range(L):
        f[:, 0, i] = O.feq(O.GUIDED, th[i], rho[i], 0.0, 0.0)
    p = O.params(L, 1, tau, th0, O.GUIDED, coll, theta_local=theta_local)
    amp = []
    for _ in range(steps + 1):
        amp.append(np.sum((O.fields(f)[0][0] - 1) * cs))
        f = O.step(f, p)
    amp = np.array(amp)
    zc = [t + amp[t] / (amp[t] - amp[t + 1]) for t in range(steps) if amp[t] * amp[t + 1] < 0]
    return (2 * np.pi / (2 * np.mean(np.diff(zc)))) / (2 * np.pi / L)


def check_local_theta_sound_speed():
    """Sound speed c_s = sqrt(gamma theta): gamma = 1 in the isothermal scheme
    (fixed theta) and gamma = (D + 2)/D = 2 for the two-dimensional monatomic
    gas once each node's equilibrium carries its own temperature (adiabatic
    sound; the guided equilibrium's heat-flux defect, Sec. III, vanishes to
    first order in u at theta = 1/3)."""
    for coll in (O.OREG, O.BGK):
        c_iso = _density_wave_speed(coll, False, False)
        assert abs(c_iso / math.sqrt(1 / 3) - 1) < 1e-3, (coll, c_iso)
        c_ad = _density_wave_speed(coll, True, True)
        assert abs(c_ad / math.sqrt(2 / 3) - 1) < 1e-3, (coll, c_ad)


# ---------------------------------------------------------------------------
# full-way bounce-back wall columns (Sec. IV shock tube)
# ---------------------------------------------------------------------------

def check_walls_conservation():
    """Bounce-back only permutes populations: the mass summed over all nodes
    (walls included) stays exact, and a uniform fluid at rest, whose
    populations are symmetric under c -> -c, is a fixed point."""
    rng = np.random.default_rng(RNG_SEED + 21)
    nx, ny = 19, 5
    for coll in (O.OREG, O.BGK):
        p = O.params(nx, ny, 0.7, 1 / 3, O.GUIDED, coll, walls=True)
        f = O.init_equilibrium(p, rng.uniform(0.8, 1.2, (ny, nx)),
                               rng.uniform(-0.05, 0.05, (ny, nx)),
                               rng.uniform(-0.05, 0.05, (ny, nx)))
        g = O.run(f, p, 300)
        _close(g.sum() / f.sum() - 1, 0.0, 1e-13, "mass with walls")
        rest = O.init_equilibrium(p, np.full((ny, nx), 1.1), np.zeros((ny, nx)),
                                  np.zeros((ny, nx)))
        assert np.array_equal(O.run(rest, p, 7), rest), "rest state with walls moved"
    post = np.zeros(9)
    f = rng.uniform(0.1, 0.5, 9)
    O.lib().ora_bounce_back_node(O._p(f), O._p(post))
    c = _c()
    for i in range(9):
        k = [j for j in range(9) if (c[j] == -c[i]).all()][0]
        assert post[i] == f[k], "bounce-back must return f_opp(i) along c_i"


def check_walls_shear_decay():
    """No-slip walls halfway between the wall columns and the first fluid
    columns: u_y = A sin(pi (x - 1/2) / L), L = nx - 2, is the slowest
    Navier-Stokes mode between walls at x = 1/2 and x = nx - 3/2 and decays
    as exp(-nu (pi / L)^2 t), nu = theta (tau - 1/2)."""
    nx, ny = 66, 2
    L = nx - 2
    x = np.arange(nx)
    prof = np.sin(np.pi * (x - 0.5) / L)
    prof[0] = prof[-1] = 0.0
    for coll in (O.OREG, O.BGK):
        for tau in (0.6, 0.8):
            p = O.params(nx, ny, tau, 1 / 3, O.GUIDED, coll, walls=True)
            f = O.init_equilibrium(p, np.ones((ny, nx)), np.zeros((ny, nx)),
                                   1e-3 * prof[None, :] * np.ones((ny, 1)))
            ts, amps = [], []
            for t in range(0, 4001, 100):
                vy = O.fields(f)[2]
                if t >= 200:
                    ts.append(t)
                    amps.append(np.sum(vy[0, 1:-1] * prof[1:-1]))
                f = O.run(f, p, 100)
            gamma = -np.polyfit(ts, np.log(amps), 1)[0]
            ratio = gamma / ((tau - 0.5) / 3 * (np.pi / L) ** 2)
            assert abs(ratio - 1) < 1e-3, (coll, tau, ratio)


def check_walls_shock_tube():
    """Sec. IV, Figs. 3-4: the shock tube between bounce-back walls on 800 x 1
    cells, 500 steps, at (theta, nu) = (0.35, 1e-5) and (0.4, 1e-9).  OReg
    matches the exact isothermal Riemann solution (c_s = sqrt(theta)) to the
    paper's ~98-99% L2 accuracy with no spurious oscillation (total
    variation within 1% of the exact profile's); BGK oscillates."""
    g = GOLDEN["walled_shock_tube"]
    for gc, acc in zip(g["cases"], (0.985, 0.98)):
        theta, nu = gc["theta"], gc["nu"]
        case = W.shock_tube_walls(theta=theta, nu=nu, nx=g["grid"][0], ny=g["grid"][1],
                                  steps=g["steps"])
        x = np.arange(case.nx)
        rho_ex, _ = riemann.solution((x - (case.x_split - 0.5)) / case.steps,
                                     case.rho_left, case.rho_right, theta)
        fluid = (x >= 1) & (x <= case.nx - 2)
        tv_exact = np.abs(np.diff(rho_ex[fluid])).sum()
        tv = {}
        for coll in (O.OREG, O.BGK):
            p = O.params(case.nx, case.ny, case.tau, theta, O.GUIDED, coll, walls=True)
            rho = O.fields(O.run(O.init_equilibrium(p, *case.fields()), p, case.steps))[0][0]
            tv[coll] = np.abs(np.diff(rho[fluid])).sum() / tv_exact
            if coll == O.OREG:
                l2 = np.sqrt(((rho[fluid] - rho_ex[fluid]) ** 2).sum() / (rho_ex[fluid] ** 2).sum())
                assert 1 - l2 >= acc, (theta, nu, l2)
                # the paper's printed accuracy (its initial densities are not
                # stated; 1.5 | 0.75 is read): within one percentage point
                assert abs((1 - l2) - gc["oreg_density_l2_accuracy"]) <= 0.01, (theta, nu, l2)
                assert abs(tv[coll] - 1) < 0.01, (theta, nu, tv)
        assert tv[O.BGK] > 10, (theta, nu, tv)


FAST_CHECKS = [
    check_velocity_set, check_guided_rest_weights, check_poly2_rest_weights,
    check_equilibrium_moments, check_foreg_mass_zero, check_foreg_guided_closed_forms,
    check_foreg_poly2_closed_forms, check_first_order_closed_forms,
    check_foreg_vanishes_without_stress,
    check_collision_special_cases, check_streaming_translation,
    check_uniform_state_is_fixed, check_conservation,
]
LATTICE_CHECKS = [check_shear_wave_decay, check_shear_wave_decay_off_reference_temperature,
                  check_first_order_start, check_mean_flow_axis_wave,
                  check_mean_flow_diagonal_wave, check_shock_tube,
                  check_walls_conservation, check_walls_shear_decay, check_walls_shock_tube,
                  check_local_theta_energy, check_local_theta_sound_speed]
